// sde_internal.cuh -- shared definitions of the GB300 jump-SDE proton dose
// engine (arXiv 2511.03115): device data layouts, kernel parameter block,
// Philox4x32-10 stream, and the device-side samplers of the large-angle laws.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sde_dose.h"

namespace sde {

// ----------------------------------------------------------------- constants
// CODATA 2018 (MeV, cm, fm).
constexpr double kProtonMass = 938.27208816;
constexpr double kElectronMass = 0.51099895000;
constexpr double kAtomicMassUnit = 931.49410242;
constexpr double kAvogadro = 6.02214076e23;
constexpr double kFineStructure = 1.0 / 137.035999084;
constexpr double kHbarcMeVfm = 197.3269804;
constexpr double kJoulePerMeV = 1.602176634e-13;
constexpr double kPi = 3.14159265358979323846;
constexpr float kTwoPiF = 6.28318530717958648f;

// Random stream tags (second counter word of Philox).
enum : uint32_t { kTagStep = 0, kTagJumpA = 1, kTagJumpB = 2, kTagSrcA = 3, kTagSrcB = 4 };

// Error flag bits raised on the device.
enum : uint32_t { kErrStepCap = 1u, kErrBadSpot = 2u, kErrNaN = 4u, kErrSecQueue = 16u };

// A secondary proton of the branching model waiting for transport: its history, its
// segment index (the j-th non-elastic event of the primary; it selects the random
// streams through the upper bits of the Philox tag word), and its initial state.
struct SecRec {
    unsigned long long h;
    uint32_t seg;
    float E, px, py, pz, ux, uy, uz, tau;
    uint32_t pad;
};
static_assert(sizeof(SecRec) == 48, "secondary record is 48 bytes");

// Hot table row per (material, energy point E_k): three float4 =
//   {f1, df1, f2, df2}  f1 = varsigma_1 beta^2 Delta / rho, f2 = sqrt(varsigma_2^2 Delta / rho)
//   {bt, dbt, fe, dfe}  bt = 1/(2 chi_alpha^2 (1-F) p^2), fe = sigma_e E^2 Delta / rho
//   {fn, dfn, cw, ct}   fn = sigma_ne Delta / rho; material constants
//                       cw = chi_c^2 (p beta)^2 / rho, ct = cw Delta / (z (1+F^2))
// Value at fractional grid position k + f is v + f dv (linear in ln E).  The
// fields are scaled by kinematic factors so that they are nearly linear in
// ln E; the kernel multiplies the factors back from E.
constexpr int kRowFloat4 = 3;
constexpr int kRawFields = 5;
// Hydrogen (Mott) inversion table of the fixed cut-off: knots in log2 of the no-sine root s0
// from log2(1 - cos theta_cut) to 0.
constexpr int kMottKnots = 64;

// Element data of a material as seen by the jump sampler.
struct MatJump {
    int n_el;
    int Z[SDE_MAX_ELEMENTS];
    float A[SDE_MAX_ELEMENTS];   // standard atomic weight
    float m2[SDE_MAX_ELEMENTS];  // target rest energy, MeV
};

// Beam spot in device form: position relative to the phantom origin in voxel units
// (mm over the voxel size of each axis), unit direction, and the two unit vectors
// spanning the lateral plane times the lateral sigma, in voxel units per axis.
struct SpotDev {
    float E, sE, sxy, sang;
    float px, py, pz, pad0;
    float ux, uy, uz, pad1;
    float e1x, e1y, e1z, pad2;
    float e2x, e2y, e2z, pad3;
};

// Balance counters (device, u64) in this order, then the work-queue cursor.
enum { kCntIncident = 0, kCntDeposited, kCntEscaped, kCntRemoved, kCntHistories, kCntSteps,
       kCntJumpEl, kCntJumpInel, kCntCursor, kCntWords };

// Everything the transport kernel reads, passed by value (constant bank).
struct KParams {
    int nx, ny, nz, n_mats;
    float inv_hx, inv_hy, inv_hz;
    float step_mm, half_step_mm;
    // Positions are kept in voxel units: one step and half a step along each axis
    // (x and y as a pair for the packed FP32x2 multiply-add).
    float2 sv_xy, hv_xy;
    float sv_z, hv_z;
    float inv_delta_cm;  // 1 / Delta (1/cm): jump rates x Delta back to rates
    float e_min, e_max;
    float qscale;  // 2^S
    int max_steps, mask, tally_mode, N;
    float lg2_emin, inv_dlg2;  // grid position = (log2 E - lg2_emin) * inv_dlg2
    float s_cut;               // 1 - cos(theta_cut)
    float ruth_span;           // 1/s_cut - 1/2
    float s_back;              // 1 - cos(backscatter limit)
    float inel_lo, inel_span, km_r;
    int batch, refill_min, aggregate;
    uint32_t rk0[10], rk1[10];  // Philox round keys
    float strag_on, mcs_on;  // 1 or 0 (physics_mask)
    const uint32_t* __restrict__ vox;  // packed voxel words (density | material id)
    unsigned long long* __restrict__ edep;
    const float4* __restrict__ table;  // [n_mats][N][kRowFloat4]
    const float* __restrict__ jrates;  // [n_mats][N][2*SDE_MAX_ELEMENTS] per unit density
    const float4* __restrict__ cut;    // [n_mats][N][2] Coulomb coefficients (variable cut-off)
    const float2* __restrict__ pick;   // [n_mats][N][2*SDE_MAX_ELEMENTS] cumulative rates {value, slope}:
                                       // elastic (x E^2 Delta / rho), then non-elastic (Delta / rho)
    const float4* __restrict__ mott_g;  // [N] {G(s_cut), slope, -G(s_back), slope} of the hydrogen primitive
    const float2* __restrict__ mott_r;  // [N][kMottKnots] {rho_j, rho_j+1}: exact root / no-sine root
    float mott_lg2_lo, mott_inv_dj;     // knot position = (log2 s0 - lo) * inv_dj
    float cut_k2;                      // k^2 z / Delta, or 0: fixed cut-off s_cut
    const MatJump* __restrict__ mats;
    const SpotDev* __restrict__ spots;
    const unsigned long long* __restrict__ prefix;  // [n_spots+1]
    unsigned long long h_end;  // histories with global id >= h_end are not run (range runs)
    int n_spots;
    unsigned long long* counters;  // kCntWords
    unsigned int* err;
    // branching model: 0 plain transport; 1 primaries that queue their secondaries;
    // 2 the queued secondaries.  sec_ctl[0] = records pushed, sec_ctl[1] = records claimed.
    int branch;
    float sec_frac;  // kappa
    SecRec* sec_q;
    unsigned long long* sec_ctl;
    unsigned long long sec_cap;
};

// ------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11.  Counter (n, tag, h_lo, h_hi); the ten round keys of
// the seed are precomputed on the host (Weyl sequence 0x9E3779B9, 0xBB67AE85).
// Each round's two 32x32 -> 64-bit products are formed as 64-bit multiplies (one
// wide integer multiply-add each, high and low halves together).
__device__ __forceinline__ uint4 philox(const KParams& P, uint32_t n, uint32_t tag, uint64_t h) {
    uint32_t c0 = n, c1 = tag, c2 = (uint32_t)h, c3 = (uint32_t)(h >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u, p1 = (uint64_t)c2 * 0xCD9E8D57u;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ P.rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ P.rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// (x + 1/2) 2^-32 as a float in (0, 1]: full relative precision near 0, where
// ln U is taken (the value rounds to 1 only for the top 2^7 words, where ln U = 0
// is harmless).
__device__ __forceinline__ float u01(uint32_t x) {
    return fmaf(__uint2float_rn(x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

__device__ __forceinline__ unsigned long long qfix(const KParams& P, float E) {
    return __float2ull_rn(E * P.qscale);
}

// Square root of the per-step quantities (x >= 0): the PTX approximate form, relative
// error at most 2^-23, exact at 0, without the IEEE-rounding fix-up sequence of sqrtf
// (measured 4 % of the transport kernel).
__device__ __forceinline__ float step_sqrt(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// cos and sin of a small polar angle given theta^2 (series when small).
__device__ __forceinline__ void cos_sin_from_sq(float th2, float& c, float& s) {
    if (th2 < 0.05f) {
        // Taylor series of cos and sin/theta in theta^2
        c = 1.f + th2 * (-0.5f + th2 * (1.f / 24.f + th2 * (-1.f / 720.f)));
        float so = 1.f + th2 * (-1.f / 6.f + th2 * (1.f / 120.f + th2 * (-1.f / 5040.f)));
        s = so * step_sqrt(th2);
    } else {
        __sincosf(step_sqrt(th2), &s, &c);
    }
}

// Rotate unit vector u by polar angle (cos_t, sin_t) and azimuth (cos_p, sin_p)
// about itself, with the branch-free orthonormal basis of Duff et al. (JCGT
// 2017); renormalised.
__device__ __forceinline__ void rotate(float& ux, float& uy, float& uz, float cos_t, float sin_t,
                                       float cos_p, float sin_p) {
    float sg = copysignf(1.f, uz);
    float a = __fdividef(-1.f, sg + uz);  // |sg + uz| >= 1
    float b = ux * uy * a;
    float e1x = 1.f + sg * ux * ux * a, e1y = sg * b, e1z = -sg * ux;
    float e2x = b, e2y = sg + uy * uy * a, e2z = -uy;
    float tx = cos_p * e1x + sin_p * e2x;
    float ty = cos_p * e1y + sin_p * e2y;
    float tz = cos_p * e1z + sin_p * e2z;
    float nx = cos_t * ux + sin_t * tx;
    float ny = cos_t * uy + sin_t * ty;
    float nz = cos_t * uz + sin_t * tz;
    float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
    ux = nx * inv;
    uy = ny * inv;
    uz = nz * inv;
}

}  // namespace sde
