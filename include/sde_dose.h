/*
 * sde_dose.h -- C ABI of the GB300 (sm_103a) jump-SDE proton dose engine.
 *
 * The engine advances pencil-beam protons through a voxelised phantom with the
 * Euler-Maruyama scheme of the jump SDE of arXiv 2511.03115 (Sec. 2.1.2,
 * Eq. VSDE): Bethe stopping drift, clamped Gaussian straggling, a spherical
 * Brownian direction increment from the Lynch-Dahl width, and Poisson-clocked
 * large-angle elastic and non-elastic nuclear jumps (Secs. 2.1.3-2.1.5).  The
 * energy lost in each step is tallied per voxel as 64-bit fixed-point integers
 * (one unit = 2^-S MeV), assigned at the step midpoint (Sec. 2.2.2) or split
 * along the step's chord, so the tally of a given seed is bit-identical run
 * to run.  Dose is dose-to-medium: deposited energy over voxel mass
 * (Sec. 2.2.2).
 *
 * Conventions for every call:
 *  - Return value: SDE_OK (0) or a negative SDE_E* code; sde_last_error()
 *    then describes the failure (thread-local string owned by the library).
 *  - Host pointers are read during the call only; the caller keeps ownership.
 *    The library owns all device memory it allocates; sde_dose_destroy frees it.
 *  - Device work is enqueued on the handle's stream (default: the legacy
 *    default stream; see sde_dose_set_stream) and is asynchronous unless the
 *    call says otherwise.  Errors raised on the device (step cap, invalid
 *    device-resident spot) are reported by the next sde_dose_sync /
 *    sde_dose_fetch* call as SDE_EDEVICE.
 *  - Arrays of voxels are x-fastest: index = ix + nx*(iy + ny*iz).
 *  - Coordinates are mm; energies MeV; densities g/cm^3.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef SDE_DOSE_H
#define SDE_DOSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDE_OK 0
#define SDE_EINVAL (-1)  /* bad argument (null pointer, size, range)      */
#define SDE_ENOMEM (-2)  /* device or pinned host allocation failed       */
#define SDE_ECUDA (-3)   /* a CUDA runtime call failed                     */
#define SDE_EDEVICE (-4) /* the device flagged an error (see message)      */

/* physics_mask bits (a set bit switches the term of Eq. VSDE on) */
#define SDE_PHYS_STRAGGLING 1 /* clamped Gaussian term of the energy line       */
#define SDE_PHYS_MCS 2        /* spherical Brownian increment Xi_n              */
#define SDE_PHYS_ELASTIC 4    /* large-angle elastic jumps (sigma_e, pi_e)      */
#define SDE_PHYS_INELASTIC 8  /* non-elastic jumps (sigma_ne, pi_ne)            */
#define SDE_PHYS_ALL 15

#define SDE_MAX_ELEMENTS 16
#define SDE_MAX_MATERIALS 16

typedef struct sde_dose sde_dose; /* opaque engine handle */

/* One element of a material: atomic number and mass fraction (fractions are
 * renormalised to sum to one).  Supported Z: 1,2,6,7,8,9,11-20,22,26,29,30. */
typedef struct {
    int Z;
    double mass_fraction;
} sde_element_frac;

/* A material composition (Sec. 2.1.1: materials enter through their chemical
 * composition and mean excitation energy).  I_eV <= 0 selects Bragg additivity
 * of ln I over the elements. */
typedef struct {
    const sde_element_frac* el;
    int n_el; /* 1..SDE_MAX_ELEMENTS */
    double I_eV;
} sde_material;

/* A beam spot (Sec. 2.2.2): mean energy and Gaussian energy spread, entry
 * point, direction (normalised by the library), Gaussian lateral sigma in the
 * plane perpendicular to the direction, Gaussian angular sigma (per axis),
 * and the number of histories to run from it. */
typedef struct {
    double E_MeV, sigma_E_MeV;
    double x_mm, y_mm, z_mm;
    double ux, uy, uz;
    double sigma_xy_mm, sigma_angle_rad;
    uint64_t n_hist;
} sde_spot;

/* Free parameters of the model and of the engine.  Defaults
 * (sde_default_params) are the paper's values, Sec. 2.2.2. */
typedef struct {
    double step_cm;         /* Delta of Eq. VSDE (0.05 cm)                          */
    double msc_z_cm;        /* z of the Lynch-Dahl width, m = sigma/sqrt(z) (0.05)  */
    double F;               /* Lynch-Dahl central fraction (0.98)                   */
    double theta_cut_rad;   /* large-angle elastic cut-off, CM frame (0.02)         */
    double backscatter_rad; /* hydrogen backscatter limit (0.04)                    */
    double e_min_MeV;       /* absorption energy (0.05)                             */
    double K;               /* Bethe prefactor of Eq. bethbloch (0.3072)            */
    double inel_u_lo;       /* non-elastic energy-loss fraction u ~ U(lo, hi) (0,1)  */
    double inel_u_hi;
    double km_r;            /* Kalbach-Mann pre-equilibrium fraction r (0.5)        */
    double e_max_MeV;       /* top of the physics-table energy grid (300)           */
    int tally_mode;         /* 0: midpoint deposit; 1: split along the chord (DDA)  */
    int fixed_point_shift;  /* S: one tally unit = 2^-S MeV (24)                    */
    int max_steps;          /* step cap per history; exceeding it is SDE_EDEVICE    */
    int physics_mask;       /* SDE_PHYS_* (SDE_PHYS_ALL)                            */
    int table_points;       /* points of the ln-E table grid, 64..4096 (256)        */
    double theta_cut_sigmas;/* 0: fixed theta_cut_rad (the paper's runs); k in (0, 100]: the
                               energy-dependent cut-off theta_c = k sigma(E) of Sec. 2.1.3
                               (k = 2.5), sigma the Lynch-Dahl width over z at the step's
                               energy and density, clamped to [1e-4, 1] rad; it sets the
                               large-angle elastic rates and the jump's CM angle range   */
    double secondary_fraction; /* 0: the paper's model, one proton per history (default).
                               kappa in (0, 1]: branching SDE (Sec. 2.1.1 names it as the
                               extension of the model): every non-elastic event of a primary
                               also emits a secondary proton with energy kappa u E' (E' = the
                               energy after the step's continuous loss, u the event's loss
                               fraction), from the event point, at a Kalbach-Mann CM angle of
                               its own (slope at emission fraction kappa u) about the incoming
                               direction, with uniform azimuth; it is transported by the same
                               SDE and emits no secondaries itself.  Its energy moves from
                               "removed" to the tally or "escaped".  Secondaries wait in a
                               device queue between two launches per chunk of histories; an
                               overflow is SDE_EDEVICE (the balance stays exact)           */
} sde_params;

/* Energy balance in tally units: incident == deposited + escaped + removed
 * holds exactly (escaped: carried out of the phantom; removed: lost in
 * non-elastic events and not tallied, Sec. 2.1.1). */
typedef struct {
    uint64_t incident, deposited, escaped, removed;
    uint64_t histories, steps, jumps_elastic, jumps_inelastic;
} sde_balance;

/* Launch shape of the transport kernel.  Zero fields keep the current value.
 * blocks_per_sm * warps_per_block warps run persistently; each warp claims
 * batch histories at a time from the shared work queue and refills its idle
 * lanes once at least refill_min of them are idle (or all lanes are idle).
 * The tally does not depend on these settings. */
typedef struct {
    int blocks_per_sm;   /* 1..8 (default: as many as fit)                 */
    int warps_per_block; /* 1..8 (default 8)                                */
    int batch;           /* 32..4096, multiple of 32 (default 32)           */
    int refill_min;      /* 1..32 (default 32: refill whole warps)          */
    int table_smem;      /* 1: stage the physics tables in shared memory;
                            2: read them through the L1 cache (default 2)   */
    int aggregate;       /* midpoint tally: 1 one atomic per lane and step
                            (default); 2 lanes of a warp that hit the same
                            voxel sum their deposits first                  */
    int graph;           /* 1: launch the kernels directly (default);
                            2: launch them as one CUDA graph                */
} sde_tuning;

/* Fill p with the defaults listed above.  Returns SDE_OK or SDE_EINVAL (p NULL). */
int sde_default_params(sde_params* p);

/* Message of the last failing call on this host thread (never NULL). */
const char* sde_last_error(void);

/* Create an engine for a phantom of nx*ny*nz voxels of size voxel_mm with its
 * first corner at origin_mm.  density_g_cm3 (>= 0) and material_id (< n_mats)
 * are x-fastest host arrays; mats[n_mats] are the compositions.  p may be
 * NULL (defaults).  Copies the phantom to the device, builds the FP32 physics
 * tables (FP64 evaluation on the device) and the CSDA range table.
 * Synchronous.  Errors: SDE_EINVAL, SDE_ENOMEM, SDE_ECUDA. */
int sde_dose_create(sde_dose** out, int nx, int ny, int nz, const double voxel_mm[3],
                    const double origin_mm[3], const float* density_g_cm3,
                    const uint8_t* material_id, const sde_material* mats, int n_mats,
                    const sde_params* p);

/* Use this CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) for all later work of the handle.  The caller keeps the stream
 * alive while the handle uses it. */
int sde_dose_set_stream(sde_dose* d, void* cuda_stream);

/* Set the transport launch shape (see sde_tuning). */
int sde_dose_set_tuning(sde_dose* d, const sde_tuning* t);
int sde_dose_get_tuning(const sde_dose* d, sde_tuning* t);

/* Autotuner: run the plan spots[0..n_spots) (host array), scaled down to at
 * most max_histories histories, under a fixed set of candidate launch shapes
 * (warps per block, refill threshold, batch, table placement, tally
 * aggregation, blocks per SM), keep the fastest (CUDA-event timing, best of
 * two timed runs after a warm-up) as the handle's tuning and return it in
 * best_out (may be NULL).  The results do not depend on the tuning.  The
 * tuning runs go through the tally: the call ends with sde_dose_reset, so
 * tune before accumulating.  Synchronous. */
int sde_dose_autotune(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed,
                      uint64_t max_histories, sde_tuning* best_out);

/* Transport the histories of spots[0..n_spots) (host array) with the given
 * seed and add their deposits to the tally (accumulates until reset).  History
 * ids run 0..sum(n_hist)-1 in spot order; the random stream of history h is
 * keyed by (seed, h), so a run is reproducible bit for bit.  The spots are
 * copied before the call returns; the transport itself is asynchronous.
 * Errors: SDE_EINVAL (bad spot, energy above e_max/1.05), SDE_ECUDA. */
int sde_dose_run(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed);

/* As sde_dose_run for the histories with global ids in [first_history,
 * first_history + n_histories) of the plan only (ids beyond the plan's total
 * are ignored).  Because every history's random stream is keyed by its global
 * id, disjoint ranges run with one seed -- on one handle, or on several GPUs
 * whose integer tallies are then summed -- give exactly the tally and balance
 * of the whole run: the multi-GPU split of a plan (the paper has no
 * counterpart; its histories are independent, Sec. 2.2.3).  Errors as
 * sde_dose_run. */
int sde_dose_run_range(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed, uint64_t first_history,
                       uint64_t n_histories);

/* As sde_dose_run, with spots already in device memory (d_spots, device
 * pointer to n_spots sde_spot records, caller-owned, must stay valid until
 * the work completes).  Fully asynchronous: invalid spots are reported as
 * SDE_EDEVICE by the next sync/fetch and their histories are not run. */
int sde_dose_run_device(sde_dose* d, const sde_spot* d_spots, int n_spots, uint64_t seed);

/* sde_dose_run_range with device-resident spots (as sde_dose_run_device). */
int sde_dose_run_device_range(sde_dose* d, const sde_spot* d_spots, int n_spots, uint64_t seed,
                              uint64_t first_history, uint64_t n_histories);

/* Wait for the handle's work; SDE_EDEVICE if the device flagged an error
 * (the flag is cleared by the call). */
int sde_dose_sync(sde_dose* d);

/* Copy results to host buffers (any may be NULL): dose_Gy[n_vox] (dose to
 * medium, 0 where density is 0), edep_fixed[n_vox] (tally units), bal.
 * Synchronous. */
int sde_dose_fetch(sde_dose* d, double* dose_Gy, uint64_t* edep_fixed, sde_balance* bal);

/* As sde_dose_fetch with device output buffers d_dose_Gy / d_edep_fixed
 * (caller-owned device memory, n_vox elements; either may be NULL).  The
 * conversion runs on the device; bal (host, may be NULL) is read back.
 * Synchronous when bal is non-NULL, else asynchronous. */
int sde_dose_fetch_device(sde_dose* d, double* d_dose_Gy, uint64_t* d_edep_fixed,
                          sde_balance* bal);

/* As sde_dose_fetch_device for the dose only, written as FP32 (n_vox floats,
 * caller-owned device memory).  Asynchronous. */
int sde_dose_fetch_device_f32(sde_dose* d, float* d_dose_Gy);

/* Zero the tally and the balance counters (asynchronous). */
int sde_dose_reset(sde_dose* d);

/* Release all device and host memory of the handle (synchronises first). */
void sde_dose_destroy(sde_dose* d);

/* Grid and table facts: n_vox, the number of table points, the ln-E grid
 * (e_min, e_max) and the number of materials.  Any output may be NULL. */
int sde_dose_info(const sde_dose* d, uint64_t* n_vox, int* table_points, double* e_min_MeV,
                  double* e_max_MeV, int* n_mats);

/* Copy the FP32 per-step physics tables of material m to host memory.
 * out[table_points * 5] receives, per grid energy E_k = e_min (e_max/e_min)^(k/(N-1)):
 * varsigma_1/rho (MeV cm^2/g), varsigma_2^2/rho (MeV^2 cm^2/g), chi_c^2/rho
 * (rad^2 cm^3/g, over the path z), 1/(2 chi_alpha^2 (1-F)) (rad^-2) and
 * (sigma_e + sigma_ne)/rho (cm^2/g).  rates_out[table_points * 2 * n_el]
 * (may be NULL) receives the per-element elastic then non-elastic rates per
 * unit density.  csda_out[table_points] (may be NULL) receives the CSDA range
 * at unit density (g/cm^2, FP64 quadrature).  Synchronous. */
int sde_dose_tables(const sde_dose* d, int m, float* out, float* rates_out, double* csda_out);

/* Single-step probe: for n independent histories h0..h0+n-1 at energy E (MeV)
 * along +z in an unbounded medium of material m and density rho, take one
 * step of the transport kernel's step function (same tables, same random
 * stream: step 0 of history h, exponential jump clock started from the
 * history's source draw) and write (each may be NULL) E_out (energy after the
 * step), cos_out (new direction . old), jump_out (0 none, 1 elastic,
 * 2 non-elastic), ux_out/uy_out.  All outputs are HOST arrays of n elements.
 * Synchronous.  For tests of the step against the oracle. */
int sde_dose_probe_steps(sde_dose* d, int m, double rho, double E, uint64_t seed, uint64_t h0,
                         int n, float* E_out, float* cos_out, int* jump_out, float* ux_out,
                         float* uy_out);

/* ---- learned denoiser building blocks (tensor-core kernels) ----
 * The denoiser is a 3D convolutional encoder-decoder that maps a low-history
 * dose and the density map to a high-history dose (it has no counterpart in
 * the paper; the plain high-history transport remains its reference).  Its
 * kernels use the tcgen05 tensor core (BF16 operands, FP32 accumulation in
 * tensor memory).  Completion waits are bounded; a wait that times out leaves
 * the output unwritten and the call returns SDE_EDEVICE.  Synchronous. */

/* D[M x N] = A[M x K] x B[N x K]^T.  A, B: device BF16, row-major, 16-byte
 * aligned; D: device FP32, row-major.  N a multiple of 16 in [16, 256], K a
 * multiple of 16.  stream: cudaStream_t or NULL. */
int sde_gemm_bf16(const void* d_A, const void* d_B, float* d_D, int M, int N, int K, void* stream);

/* Activation layout of the convolutions, "padded channel-group-major" BF16: a tensor of
 * C channels (C a multiple of 8) on a D x H x W grid is [batch][C/8][D+2][H+2][W+2][8],
 * channel 8 g + e of voxel (z, y, x) at ((((n C/8 + g)(D+2) + z+1)(H+2) + y+1)(W+2) + x+1) 8 + e.
 * The one-voxel border holds zeros (the convolution's zero padding): the caller zeroes
 * it once and these calls never write it.
 *
 * 3x3x3 convolution, stride 1, zero padding 1:
 * y[n][v][y_coffset + co] = (relu?) (bias[co] + sum_{tap,ci} x[n][v + off(tap)][ci] w[co][tap][ci]),
 * tap = 9 kz + 3 ky + kx, off = (kz-1, ky-1, kx-1).  d_x padded channel-group-major with Cin
 * channels; d_w [Cout][27][Cin] BF16 (the call packs it for the tensor core in
 * stream-ordered scratch memory); d_bias [Cout] FP32 or NULL.  The output has y_cstride
 * channels written from channel y_coffset on (so two producers can fill the parts of a
 * concatenation): padded channel-group-major BF16, or with y_fp32 != 0 plain
 * channels-last FP32 [batch][D*H*W][y_cstride].  Requires W <= 256, Cin a multiple of
 * 16 in [16, 192], Cout a multiple of 16 in [16, 256], 16-byte aligned d_x, d_y and
 * d_bias (SDE_EINVAL otherwise).  The data gradient of the convolution is this call on dy with
 * the weights of sde_conv3d_flip_weights.  Asynchronous; sde_denoise_status reports a
 * timed-out wait. */
int sde_conv3d_forward(const void* d_x, int batch, int D, int H, int W, int Cin, const void* d_w,
                       const float* d_bias, int Cout, void* d_y, int y_cstride, int y_coffset, int y_fp32,
                       int relu, void* stream);

/* Weight gradient of sde_conv3d_forward: d_dw[co][tap][ci] += sum over voxels of
 * dy[v][co] x[v + off(tap)][ci] (FP32 accumulation into d_dw; d_x and d_dy padded
 * channel-group-major BF16 with Cin and Cout channels; Cout <= 128; shape limits as
 * sde_conv3d_forward).  Asynchronous. */
int sde_conv3d_wgrad(const void* d_x, const void* d_dy, float* d_dw, int batch, int D, int H, int W, int Cin,
                     int Cout, void* stream);

/* d_wd[ci][26 - tap][co] = d_w[co][tap][ci] (BF16): weights of the data-gradient convolution. */
int sde_conv3d_flip_weights(const void* d_w, void* d_wd, int Cin, int Cout, void* stream);

/* Host-only inspection of the work decompositions the two convolution kernels launch
 * (no CUDA call: usable without a GPU, e.g. to check a shape's shared-memory and
 * tensor-memory layout before running it).
 * sde_conv3d_plan: the plan of sde_conv3d_forward for this shape, as 17 ints in the
 * order Ty, tiles, rowtile, fold, nyb, P, Yb, Cp, nsplit, plane, w_off, wres, stage,
 * nacc, xch, tcols, items (rows per work item, 128-position M tiles per item, row
 * tiles, x-tap fold, row blocks, brick row pitch W + 2, brick rows Ty + 2, output
 * channels per part, parts, bytes between the two 8-channel planes of a chunk,
 * weight offset in a stage, resident weights, bytes per stage, accumulators,
 * offset of the fold's exchange buffer, tensor-memory columns, work items), and
 * its dynamic shared memory in bytes.
 * sde_conv3d_wgrad_plan: the plan of sde_conv3d_wgrad on a GPU with `sms`
 * multiprocessors, as 14 ints: Ty, nyb, P, Yb, Nc, ntap, ngroups, kst, plane_dy,
 * plane_x, x_off, stage, items, G (input channels and taps per pass, tap groups,
 * 16-position K steps per item, plane pitches of the output-gradient rows and of
 * the input brick, brick offset in a stage, CTAs per pass), and its dynamic shared
 * memory.  Both fill min(n_fields, count) ints; SDE_EINVAL for a shape the
 * convolution rejects or has no plan for. */
int sde_conv3d_plan(int batch, int D, int H, int W, int Cin, int Cout, int32_t* fields, int n_fields,
                    uint64_t* smem_bytes);
int sde_conv3d_wgrad_plan(int batch, int D, int H, int W, int Cin, int Cout, int sms, int32_t* fields,
                          int n_fields, uint64_t* smem_bytes);

/* Wait for the stream and report (and clear) a timed-out tensor-core wait of any
 * denoiser kernel since the last call: SDE_EDEVICE, else SDE_OK. */
int sde_denoise_status(void* stream);

/* The denoiser network: a 3-level 3D convolutional encoder-decoder (32/64/128
 * channels, 3x3x3 kernels, average-pool down, nearest-neighbour up, skip
 * concatenations, leaky ReLU with slope 0.1), BF16 weights and activations with FP32 accumulation,
 * trained with Adam on FP32 master weights.  Inputs on a D x H x W grid (x
 * fastest, device FP32): the low-history dose (Gy) and the density (g/cm^3);
 * the output is the dose (Gy).  Internally the dose is scaled by 1/max of the
 * low-history dose of each sample and the network predicts a correction that
 * is added to it; the output layer starts at zero, so an untrained network
 * returns its input.  D, H, W must be multiples of 4, W <= 256 and
 * (D+2)(H+2)(W+2) batch_max below 2^31 / 24 (SDE_EINVAL otherwise).  The handle
 * owns its device memory (weights, optimiser state, and the activations and
 * gradients of batch_max samples in the convolutions' padded channel-group-major
 * layout). */
typedef struct sde_denoiser sde_denoiser;
int sde_denoiser_create(sde_denoiser** out, int D, int H, int W, int batch_max, uint64_t seed);
void sde_denoiser_destroy(sde_denoiser* d);
int sde_denoiser_set_stream(sde_denoiser* d, void* cuda_stream);
int sde_denoiser_num_params(const sde_denoiser* d, uint64_t* n);
/* Inference: d_dose_low and d_dose_out [batch][D*H*W], d_density [D*H*W] (one
 * density map for the batch), device FP32.  Asynchronous. */
int sde_denoiser_infer(sde_denoiser* d, const float* d_dose_low, const float* d_density, int batch,
                       float* d_dose_out);
/* One Adam step on the squared error between the prediction and t =
 * target_scale * d_dose_high (target_scale: e.g. the ratio of the history counts
 * of the low and high runs, so that both are doses of the same fluence), both
 * scaled as the input, weighted by 1/(t + 0.05) and summed over voxels (Adam
 * works on the sum; loss_out, host, may be NULL, receives the mean over voxels,
 * which makes the call synchronous). */
int sde_denoiser_train_step(sde_denoiser* d, const float* d_dose_low, const float* d_density,
                            const float* d_dose_high, float target_scale, int batch, float lr,
                            float* loss_out);
/* Gradient of the summed loss for all parameters without an update (host FP32
 * vector, same order as sde_denoiser_get_params; loss_out gets the mean loss);
 * synchronous. */
int sde_denoiser_gradients(sde_denoiser* d, const float* d_dose_low, const float* d_density,
                           const float* d_dose_high, float target_scale, int batch, float* host_grad,
                           uint64_t n, float* loss_out);
/* All parameters as one FP32 host vector: per layer the weights [Cout][27][Cin]
 * then the biases [Cout].  Synchronous. */
int sde_denoiser_get_params(const sde_denoiser* d, float* host, uint64_t n);
int sde_denoiser_set_params(sde_denoiser* d, const float* host, uint64_t n);

/* d_x[i] *= factor for i < n (device FP32).  Asynchronous. */
int sde_scale_f32(float* d_x, uint64_t n, float factor, void* stream);

/* 3D gamma index (local dose normalisation): reference voxels with dose >=
 * threshold * max(ref) are evaluated; one passes when an evaluated position within
 * dta_mm (searched on a grid of step dta_mm/steps, trilinear interpolation of
 * d_eval) has |dr|^2/dta^2 + (De - Dr)^2/(dd Dr)^2 <= 1.  Device FP32 grids of
 * nx*ny*nz (x fastest).  Synchronous; returns the counts. */
int sde_gamma3d(const float* d_ref, const float* d_eval, int nx, int ny, int nz, const double voxel_mm[3],
                double dd, double dta_mm, double threshold, int steps, uint64_t* n_eval, uint64_t* n_pass,
                void* stream);

/* Transport without any memory allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory -- code
 * running inside a framework that owns every device allocation through its own
 * pool, and services that forbid allocation after start-up because cudaMalloc
 * can block or fail at an arbitrary moment.
 *
 * It runs the same kernels as sde_dose_run_device on caller-owned device
 * inputs and output: d_vox[nx*ny*nz] packed voxel words (the FP32 density with
 * its low 4 mantissa bits replaced by the material id: word =
 * ((bits(density) + 8) & ~15) | material_id, material_id < n_mats), d_spots
 * (n_spots sde_spot records) and d_edep (nx*ny*nz 64-bit tally, ADDED to).
 * mats, params (not NULL) and bal (may be NULL) are host memory; d_status (may
 * be NULL) is one caller-owned device word.  Every other buffer (physics
 * tables, device spot records, history prefix, work-queue cursor, balance
 * counters) lives in one static 1 MiB device array inside the library, which
 * each GPU that loads the library holds until the process exits.  Limits set by
 * that array: n_mats <= 4, params->table_points <= 256, n_spots <= 4096; larger
 * inputs fail with SDE_EINVAL.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 *
 * The voxel words are checked on the device before the transport uses them:
 * a material id >= n_mats or a density that is not finite in [0, 1e3) g/cm^3
 * raises device error bit 8 and no history runs (d_edep is left as it was).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The array keeps the last call's contents; each
 * call clears what must start at zero.  All calls share the one array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and corrupt each other: serialise them.  Work is enqueued on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream).  Device-side
 * errors of the call (bits: 1 step cap reached, 2 invalid spot, 8 bad voxel
 * word; 0 = none) are written to *d_status when it is not NULL.  With bal !=
 * NULL the call waits for its work and fills the balance of this call alone
 * (deposited = the increase of the tally's sum, so a tally that already held
 * earlier deposits still balances: incident = deposited + escaped + removed),
 * and returns SDE_EDEVICE when a device error bit was raised; with bal == NULL
 * it returns without waiting and only d_status reports device-side errors. */
int sde_transport_noalloc(int nx, int ny, int nz, const double voxel_mm[3], const double origin_mm[3],
                          const uint32_t* d_vox, const sde_material* mats, int n_mats,
                          const sde_params* params, const sde_spot* d_spots, int n_spots,
                          uint64_t seed, unsigned long long* d_edep, sde_balance* bal,
                          unsigned int* d_status, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
