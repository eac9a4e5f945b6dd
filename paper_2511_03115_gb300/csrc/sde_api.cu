// sde_api.cu -- the C ABI of the GB300 jump-SDE proton dose engine
// (declarations and contracts in include/sde_dose.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sde_internal.cuh"
#include "sde_tables.h"
#include "sde_transport.h"

using namespace sde;

static thread_local char g_err[512] = "";

static int set_err(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(e_ == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA,        \
                           "%s failed: %s", #call, cudaGetErrorString(e_));                 \
    } while (0)

struct sde_dose {
    int device = 0;
    int num_sms = 0;
    int nx = 0, ny = 0, nz = 0;
    size_t nvox = 0;
    double h[3] = {0, 0, 0}, o[3] = {0, 0, 0};
    sde_params p{};
    int n_mats = 0;
    MatHost mats[SDE_MAX_MATERIALS];
    MatJump mj[SDE_MAX_MATERIALS];
    cudaStream_t stream = nullptr;
    sde_tuning tune{};
    // device memory owned by the handle
    float* d_rho = nullptr;
    uint32_t* d_vox = nullptr;  // packed density | material id
    unsigned long long* d_edep = nullptr;
    MatHost* d_mats = nullptr;
    MatJump* d_mj = nullptr;
    float* d_raw = nullptr;
    float* d_jrates = nullptr;
    double* d_csda = nullptr;
    float4* d_table = nullptr;
    float4* d_cut = nullptr;  // [n_mats][N][2] Coulomb coefficients of the variable cut-off
    float2* d_pick = nullptr;  // [n_mats][N][2*SDE_MAX_ELEMENTS] cumulative rates for the event pick
    float4* d_mott_g = nullptr;  // [N] hydrogen primitive at the ends of the sampled range
    float2* d_mott_r = nullptr;  // [N][kMottKnots] hydrogen inversion ratios
    unsigned long long* d_counters = nullptr;
    unsigned int* d_err = nullptr;
    sde_spot* d_raw_spots = nullptr;
    SpotDev* d_spots = nullptr;
    unsigned long long* d_prefix = nullptr;
    int spot_cap = 0;
    double* d_dose = nullptr;
    // pinned host staging
    sde_spot* h_stage = nullptr;
    int stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    unsigned long long* h_counters = nullptr;  // kCntWords + 1 (error flag)
    size_t table_bytes = 0;
    // graph launch: [spot prep, transport] captured on a private stream and
    // updated in place when only kernel arguments change
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // branching model: the secondary queue (allocated on first use) and its two counters
    SecRec* d_secq = nullptr;
    unsigned long long* d_secctl = nullptr;
};

// Queue capacity of the branching model, in secondaries; histories run in chunks of this
// many, so the queue overflows only if a chunk's primaries average more than one
// non-elastic event each (about 0.1-0.4 do in water and bone at 70-230 MeV).
static constexpr unsigned long long kSecQueueCap = 1ull << 21;

extern "C" int sde_default_params(sde_params* p) {
    if (!p) return set_err(SDE_EINVAL, "params pointer is NULL");
    p->step_cm = 0.05;
    p->msc_z_cm = 0.05;
    p->F = 0.98;
    p->theta_cut_rad = 0.02;
    p->backscatter_rad = 0.04;
    p->e_min_MeV = 0.05;
    p->K = 0.3072;
    p->inel_u_lo = 0.0;
    p->inel_u_hi = 1.0;
    p->km_r = 0.5;
    p->e_max_MeV = 300.0;
    p->tally_mode = 0;
    p->fixed_point_shift = 24;
    p->max_steps = 100000;
    p->physics_mask = SDE_PHYS_ALL;
    p->theta_cut_sigmas = 0.0;
    p->table_points = 256;
    p->secondary_fraction = 0.0;
    return SDE_OK;
}

extern "C" const char* sde_last_error(void) { return g_err; }

namespace sde {
// Lets other translation units of the library report through sde_last_error.
void set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace sde

static int check_params(const sde_params& p) {
    bool ok = p.step_cm > 0.0 && p.step_cm <= 1.0 && p.msc_z_cm > 0.0 && p.F > 0.0 && p.F < 1.0 &&
              p.theta_cut_rad > 0.0 && p.theta_cut_rad < 3.0 && p.backscatter_rad > 0.0 &&
              p.backscatter_rad < 1.5 && p.e_min_MeV > 0.0 && p.K > 0.0 && p.inel_u_lo >= 0.0 &&
              p.inel_u_hi <= 1.0 && p.inel_u_lo <= p.inel_u_hi && p.km_r >= 0.0 && p.km_r < 1.0 &&
              p.e_max_MeV > 2.0 * p.e_min_MeV && p.e_max_MeV <= 1000.0 &&
              (p.tally_mode == 0 || p.tally_mode == 1) && p.fixed_point_shift >= 0 &&
              p.fixed_point_shift <= 30 && p.max_steps > 0 && p.physics_mask >= 0 &&
              p.physics_mask <= SDE_PHYS_ALL && p.table_points >= 64 && p.table_points <= 4096 &&
              p.theta_cut_sigmas >= 0.0 && p.theta_cut_sigmas <= 100.0 && p.secondary_fraction >= 0.0 &&
              p.secondary_fraction <= 1.0;
    return ok ? SDE_OK : set_err(SDE_EINVAL, "invalid sde_params");
}

static void free_all(sde_dose* d) {
    void* ptrs[] = {d->d_rho,   d->d_vox,      d->d_edep,   d->d_mats,        d->d_mj,
                    d->d_raw,   d->d_jrates,   d->d_csda,   d->d_table,       d->d_counters,
                    d->d_err,   d->d_raw_spots, d->d_spots, d->d_prefix,      d->d_dose,
                    d->d_cut,   d->d_secq,      d->d_secctl, d->d_pick,       d->d_mott_g,
                    d->d_mott_r};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (d->graph_exec) cudaGraphExecDestroy(d->graph_exec);
    if (d->capture_stream) cudaStreamDestroy(d->capture_stream);
    if (d->h_stage) cudaFreeHost(d->h_stage);
    if (d->h_counters) cudaFreeHost(d->h_counters);
    if (d->stage_ev) cudaEventDestroy(d->stage_ev);
}

extern "C" int sde_dose_create(sde_dose** out, int nx, int ny, int nz, const double voxel_mm[3],
                               const double origin_mm[3], const float* density,
                               const uint8_t* material_id, const sde_material* mats, int n_mats,
                               const sde_params* p) {
    if (!out) return set_err(SDE_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !voxel_mm || !origin_mm || !density || !material_id || !mats)
        return set_err(SDE_EINVAL, "bad grid arguments");
    if (n_mats < 1 || n_mats > SDE_MAX_MATERIALS)
        return set_err(SDE_EINVAL, "n_mats must be 1..%d", SDE_MAX_MATERIALS);
    size_t nvox = (size_t)nx * ny * nz;
    if (nvox > (size_t)INT32_MAX) return set_err(SDE_EINVAL, "grid has more than 2^31-1 voxels");
    for (int a = 0; a < 3; ++a)
        if (!(voxel_mm[a] > 0.0) || !isfinite(voxel_mm[a]) || !isfinite(origin_mm[a]))
            return set_err(SDE_EINVAL, "voxel size must be > 0 and origin finite");
    sde_params prm;
    if (p)
        prm = *p;
    else
        sde_default_params(&prm);
    if (check_params(prm)) return SDE_EINVAL;
    for (size_t v = 0; v < nvox; ++v) {
        if (material_id[v] >= n_mats) return set_err(SDE_EINVAL, "material id %d out of range at voxel %zu", (int)material_id[v], v);
        if (!(density[v] >= 0.f) || !(density[v] < 1e3f)) return set_err(SDE_EINVAL, "bad density at voxel %zu", v);
    }
    sde_dose* d = new (std::nothrow) sde_dose();
    if (!d) return set_err(SDE_ENOMEM, "out of host memory");
    char msg[256];
    for (int i = 0; i < n_mats; ++i) {
        int rc = resolve_material(mats[i], &d->mats[i], msg, sizeof msg);
        if (rc) {
            delete d;
            return set_err(rc, "material %d: %s", i, msg);
        }
        MatJump& j = d->mj[i];
        memset(&j, 0, sizeof j);
        j.n_el = d->mats[i].n_el;
        for (int e = 0; e < j.n_el; ++e) {
            j.Z[e] = d->mats[i].Z[e];
            j.A[e] = (float)d->mats[i].A[e];
            j.m2[e] = (float)(j.Z[e] == 1 ? kProtonMass : d->mats[i].A[e] * kAtomicMassUnit);
        }
    }
    d->nx = nx;
    d->ny = ny;
    d->nz = nz;
    d->nvox = nvox;
    for (int a = 0; a < 3; ++a) {
        d->h[a] = voxel_mm[a];
        d->o[a] = origin_mm[a];
    }
    d->p = prm;
    d->n_mats = n_mats;
    d->tune.blocks_per_sm = 0;  // 0: occupancy maximum
    d->tune.warps_per_block = 8;
    d->tune.batch = 32;
    d->tune.refill_min = 32;
    d->tune.table_smem = 2;
    d->tune.aggregate = 1;
    d->tune.graph = 1;

    auto fail = [&](int rc) {
        free_all(d);
        delete d;
        return rc;
    };
#define TRY(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(set_err(e_ == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA,           \
                                "%s failed: %s", #call, cudaGetErrorString(e_)));                   \
    } while (0)

    TRY(cudaGetDevice(&d->device));
    TRY(cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, d->device));
    const int N = prm.table_points;
    TRY(cudaMalloc(&d->d_rho, nvox * sizeof(float)));
    TRY(cudaMalloc(&d->d_vox, nvox * sizeof(uint32_t)));
    TRY(cudaMalloc(&d->d_edep, nvox * sizeof(unsigned long long)));
    TRY(cudaMalloc(&d->d_mats, n_mats * sizeof(MatHost)));
    TRY(cudaMalloc(&d->d_mj, n_mats * sizeof(MatJump)));
    TRY(cudaMalloc(&d->d_raw, (size_t)n_mats * N * kRawFields * sizeof(float)));
    TRY(cudaMalloc(&d->d_jrates, (size_t)n_mats * N * 2 * SDE_MAX_ELEMENTS * sizeof(float)));
    TRY(cudaMalloc(&d->d_csda, (size_t)n_mats * N * sizeof(double)));
    d->table_bytes = (size_t)n_mats * N * kRowFloat4 * sizeof(float4);
    TRY(cudaMalloc(&d->d_table, d->table_bytes));
    TRY(cudaMalloc(&d->d_cut, (size_t)n_mats * N * 2 * sizeof(float4)));
    TRY(cudaMalloc(&d->d_pick, (size_t)n_mats * N * 2 * SDE_MAX_ELEMENTS * sizeof(float2)));
    TRY(cudaMalloc(&d->d_mott_g, (size_t)N * sizeof(float4)));
    TRY(cudaMalloc(&d->d_mott_r, (size_t)N * kMottKnots * sizeof(float2)));
    TRY(cudaMalloc(&d->d_counters, kCntWords * sizeof(unsigned long long)));
    TRY(cudaMalloc(&d->d_err, sizeof(unsigned int)));
    TRY(cudaMallocHost(&d->h_counters, (kCntWords + 1) * sizeof(unsigned long long)));
    TRY(cudaEventCreateWithFlags(&d->stage_ev, cudaEventDisableTiming));
    TRY(cudaMemcpy(d->d_rho, density, nvox * sizeof(float), cudaMemcpyHostToDevice));
    {
        // One 32-bit word per voxel for the transport kernel: the density rounded to
        // 19 mantissa bits (relative change < 1e-6) with the material id in the low
        // 4 bits.  The dose conversion keeps the exact densities.
        uint32_t* packed = (uint32_t*)malloc(nvox * sizeof(uint32_t));
        if (!packed) return fail(set_err(SDE_ENOMEM, "out of host memory"));
        for (size_t v = 0; v < nvox; ++v) {
            uint32_t bits;
            memcpy(&bits, &density[v], sizeof bits);
            packed[v] = ((bits + 8u) & ~15u) | (uint32_t)material_id[v];
        }
        cudaError_t e = cudaMemcpy(d->d_vox, packed, nvox * sizeof(uint32_t), cudaMemcpyHostToDevice);
        free(packed);
        TRY(e);
    }
    TRY(cudaMemcpy(d->d_mats, d->mats, n_mats * sizeof(MatHost), cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(d->d_mj, d->mj, n_mats * sizeof(MatJump), cudaMemcpyHostToDevice));
    TRY(cudaMemset(d->d_edep, 0, nvox * sizeof(unsigned long long)));
    TRY(cudaMemset(d->d_counters, 0, kCntWords * sizeof(unsigned long long)));
    TRY(cudaMemset(d->d_err, 0, sizeof(unsigned int)));

    TableBuild tb;
    tb.N = N;
    tb.n_mats = n_mats;
    tb.e_min = prm.e_min_MeV;
    tb.e_max = prm.e_max_MeV;
    tb.K = prm.K;
    tb.F = prm.F;
    tb.z = prm.msc_z_cm;
    tb.step = prm.step_cm;
    tb.theta_cut = prm.theta_cut_rad;
    tb.theta_back = prm.backscatter_rad;
    tb.mask = prm.physics_mask;
    tb.d_mats = d->d_mats;
    tb.d_raw = d->d_raw;
    tb.d_jrates = d->d_jrates;
    tb.d_csda = d->d_csda;
    tb.d_table = d->d_table;
    tb.d_cut = d->d_cut;
    tb.d_pick = d->d_pick;
    tb.d_mott_g = d->d_mott_g;
    tb.d_mott_r = d->d_mott_r;
    TRY(build_tables(tb, nullptr));
    TRY(cudaDeviceSynchronize());
#undef TRY
    *out = d;
    return SDE_OK;
}

extern "C" int sde_dose_set_stream(sde_dose* d, void* s) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    d->stream = (cudaStream_t)s;
    return SDE_OK;
}

extern "C" int sde_dose_set_tuning(sde_dose* d, const sde_tuning* t) {
    if (!d || !t) return set_err(SDE_EINVAL, "null argument");
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 8 || t->warps_per_block < 0 ||
        t->warps_per_block > kMaxWarpsPerBlock || t->batch < 0 || t->batch > 4096 || (t->batch % 32) != 0 ||
        t->refill_min < 0 || t->refill_min > 32 || t->table_smem < 0 || t->table_smem > 2 || t->aggregate < 0 ||
        t->aggregate > 2 || t->graph < 0 || t->graph > 2)
        return set_err(SDE_EINVAL,
                       "tuning out of range (blocks_per_sm 0..8, warps_per_block 0..%d, batch multiple of 32 <= 4096, "
                       "refill_min 0..32, table_smem 0..2, aggregate 0..2, graph 0..2)",
                       kMaxWarpsPerBlock);
    if (t->blocks_per_sm) d->tune.blocks_per_sm = t->blocks_per_sm;
    if (t->warps_per_block) d->tune.warps_per_block = t->warps_per_block;
    if (t->batch) d->tune.batch = t->batch;
    if (t->refill_min) d->tune.refill_min = t->refill_min;
    if (t->table_smem) d->tune.table_smem = t->table_smem;
    if (t->aggregate) d->tune.aggregate = t->aggregate;
    if (t->graph) d->tune.graph = t->graph;
    return SDE_OK;
}

extern "C" int sde_dose_get_tuning(const sde_dose* d, sde_tuning* t) {
    if (!d || !t) return set_err(SDE_EINVAL, "null argument");
    *t = d->tune;
    return SDE_OK;
}

static int ensure_spot_capacity(sde_dose* d, int n) {
    if (n <= d->spot_cap) return SDE_OK;
    int cap = std::max(n, 2 * d->spot_cap);
    if (d->d_raw_spots) cudaFree(d->d_raw_spots);
    if (d->d_spots) cudaFree(d->d_spots);
    if (d->d_prefix) cudaFree(d->d_prefix);
    d->d_raw_spots = nullptr;
    d->d_spots = nullptr;
    d->d_prefix = nullptr;
    d->spot_cap = 0;
    CUDA_TRY(cudaMalloc(&d->d_raw_spots, (size_t)cap * sizeof(sde_spot)));
    CUDA_TRY(cudaMalloc(&d->d_spots, (size_t)cap * sizeof(SpotDev)));
    CUDA_TRY(cudaMalloc(&d->d_prefix, ((size_t)cap + 1) * sizeof(unsigned long long)));
    d->spot_cap = cap;
    return SDE_OK;
}

static KParams make_kparams(const sde_dose* d, int n_spots, uint64_t seed) {
    KParams P;
    memset(&P, 0, sizeof P);
    P.nx = d->nx;
    P.ny = d->ny;
    P.nz = d->nz;
    P.n_mats = d->n_mats;
    P.inv_hx = (float)(1.0 / d->h[0]);
    P.inv_hy = (float)(1.0 / d->h[1]);
    P.inv_hz = (float)(1.0 / d->h[2]);
    P.step_mm = (float)(d->p.step_cm * 10.0);
    P.half_step_mm = (float)(d->p.step_cm * 5.0);
    P.sv_xy = make_float2((float)(d->p.step_cm * 10.0 / d->h[0]), (float)(d->p.step_cm * 10.0 / d->h[1]));
    P.sv_z = (float)(d->p.step_cm * 10.0 / d->h[2]);
    P.hv_xy = make_float2((float)(d->p.step_cm * 5.0 / d->h[0]), (float)(d->p.step_cm * 5.0 / d->h[1]));
    P.hv_z = (float)(d->p.step_cm * 5.0 / d->h[2]);
    P.inv_delta_cm = (float)(1.0 / d->p.step_cm);
    P.e_min = (float)d->p.e_min_MeV;
    P.e_max = (float)d->p.e_max_MeV;
    P.qscale = (float)ldexp(1.0, d->p.fixed_point_shift);
    P.max_steps = d->p.max_steps;
    P.mask = d->p.physics_mask;
    P.tally_mode = d->p.tally_mode;
    P.N = d->p.table_points;
    P.lg2_emin = (float)log2(d->p.e_min_MeV);
    P.inv_dlg2 = (float)((d->p.table_points - 1) / (log2(d->p.e_max_MeV) - log2(d->p.e_min_MeV)));
    double s_cut = 2.0 * sin(0.5 * d->p.theta_cut_rad) * sin(0.5 * d->p.theta_cut_rad);
    P.s_cut = (float)s_cut;
    P.ruth_span = (float)(1.0 / s_cut - 0.5);
    P.s_back = (float)(2.0 * sin(0.5 * d->p.backscatter_rad) * sin(0.5 * d->p.backscatter_rad));
    P.inel_lo = (float)d->p.inel_u_lo;
    P.inel_span = (float)(d->p.inel_u_hi - d->p.inel_u_lo);
    P.km_r = (float)d->p.km_r;
    P.batch = d->tune.batch;
    P.refill_min = d->tune.refill_min;
    P.aggregate = d->tune.aggregate == 2 ? 1 : 0;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.rk0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        P.rk1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.strag_on = (d->p.physics_mask & SDE_PHYS_STRAGGLING) ? 1.f : 0.f;
    P.mcs_on = (d->p.physics_mask & SDE_PHYS_MCS) ? 1.f : 0.f;
    P.vox = d->d_vox;
    P.edep = d->d_edep;
    P.table = d->d_table;
    P.jrates = d->d_jrates;
    P.cut = d->d_cut;
    P.pick = d->d_pick;
    P.mott_g = d->d_mott_g;
    P.mott_r = d->d_mott_r;
    P.mott_lg2_lo = (float)mott_knot_lo(d->p.theta_cut_rad);
    P.mott_inv_dj = (float)((kMottKnots - 1) / -mott_knot_lo(d->p.theta_cut_rad));
    // theta_c^2 = k^2 sigma^2 = k^2 (z / Delta) t, t the step's Brownian time
    P.cut_k2 = d->p.theta_cut_sigmas > 0.0
                   ? (float)(d->p.theta_cut_sigmas * d->p.theta_cut_sigmas * d->p.msc_z_cm / d->p.step_cm)
                   : 0.f;
    P.mats = d->d_mj;
    P.spots = d->d_spots;
    P.prefix = d->d_prefix;
    P.h_end = ~0ull;
    P.n_spots = n_spots;
    P.counters = d->d_counters;
    P.err = d->d_err;
    P.branch = 0;
    P.sec_frac = (float)d->p.secondary_fraction;
    P.sec_q = d->d_secq;
    P.sec_ctl = d->d_secctl;
    P.sec_cap = kSecQueueCap;
    return P;
}

// Branching model: per chunk of at most kSecQueueCap history ids, one launch of the
// primaries (each non-elastic event queues a secondary) and one of the queued secondaries.
// The spot preparation runs once; the plan's history count is read back to size the chunks.
static int enqueue_branching(sde_dose* d, KParams P, const sde_spot* raw, int n, uint64_t h_begin, uint64_t h_end,
                             int grid, int block) {
    if (!d->d_secq) {
        CUDA_TRY(cudaMalloc(&d->d_secq, kSecQueueCap * sizeof(SecRec)));
        CUDA_TRY(cudaMalloc(&d->d_secctl, 2 * sizeof(unsigned long long)));
    }
    P.sec_q = d->d_secq;
    P.sec_ctl = d->d_secctl;
    CUDA_TRY(launch_prep(raw, n, d->d_spots, d->d_prefix, d->d_counters, d->d_err, d->o, d->h, d->p.e_min_MeV,
                         d->p.e_max_MeV, d->stream, h_begin));
    unsigned long long total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, d->d_prefix + n, sizeof total, cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    const uint64_t end = std::min<uint64_t>(h_end, total);
    for (uint64_t b = h_begin; b < end; b += kSecQueueCap) {
        const uint64_t e = std::min<uint64_t>(end, b + kSecQueueCap);
        CUDA_TRY(launch_branch_chunk(d->d_counters, d->d_secctl, b, d->stream));
        P.branch = 1;
        P.h_end = e;
        CUDA_TRY(launch_transport(P, grid, block, 0, false, d->stream));
        P.branch = 2;
        CUDA_TRY(launch_transport(P, grid, block, 0, false, d->stream));
    }
    return SDE_OK;
}

// Histories with global ids in [h_begin, h_end) of the plan are transported.
static int enqueue_transport(sde_dose* d, const sde_spot* raw, int n, uint64_t seed, uint64_t h_begin = 0,
                             uint64_t h_end = ~0ull) {
    KParams P = make_kparams(d, n, seed);
    P.h_end = h_end;
    int warps = d->tune.warps_per_block;
    int block = warps * 32;
    bool smem = d->tune.table_smem == 1 && d->table_bytes <= 96 * 1024;
    const bool cut = P.cut_k2 > 0.f;  // own kernels: no shared-memory tables or tally aggregation
    const bool branching = d->p.secondary_fraction > 0.0;  // so has the branching model
    if (cut || branching) smem = false;
    int per_sm = transport_max_blocks_per_sm(block, smem ? d->table_bytes : 0, smem, d->p.tally_mode,
                                             d->tune.aggregate == 2, cut, branching ? 1 : 0);
    if (per_sm < 1) return set_err(SDE_ECUDA, "transport kernel cannot be resident with %d warps per block", warps);
    if (d->tune.blocks_per_sm > 0) per_sm = std::min(per_sm, d->tune.blocks_per_sm);
    int grid = d->num_sms * per_sm;
    if (branching) return enqueue_branching(d, P, raw, n, h_begin, h_end, grid, block);
    if (d->tune.graph != 2) {
        CUDA_TRY(launch_prep(raw, n, d->d_spots, d->d_prefix, d->d_counters, d->d_err, d->o, d->h, d->p.e_min_MeV,
                             d->p.e_max_MeV, d->stream, h_begin));
        CUDA_TRY(launch_transport(P, grid, block, d->table_bytes, smem, d->stream));
        return SDE_OK;
    }
    // Graph launch: capture the two launches on the private stream, update the
    // instantiated graph in place (only kernel arguments differ between runs of
    // the same shape) or re-instantiate, then launch it on the handle's stream.
    if (!d->capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&d->capture_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(d->capture_stream, cudaStreamCaptureModeRelaxed));
    cudaError_t e1 = launch_prep(raw, n, d->d_spots, d->d_prefix, d->d_counters, d->d_err, d->o, d->h, d->p.e_min_MeV,
                                 d->p.e_max_MeV, d->capture_stream, h_begin);
    cudaError_t e2 = e1 == cudaSuccess
                         ? launch_transport(P, grid, block, d->table_bytes, smem, d->capture_stream)
                         : e1;
    cudaGraph_t g = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(d->capture_stream, &g);
    if (e2 != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_err(SDE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
    }
    if (d->graph_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(d->graph_exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(d->graph_exec);
            d->graph_exec = nullptr;
        }
    }
    cudaError_t e4 = d->graph_exec ? cudaSuccess : cudaGraphInstantiate(&d->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) return set_err(SDE_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e4));
    CUDA_TRY(cudaGraphLaunch(d->graph_exec, d->stream));
    return SDE_OK;
}

static int check_spots_host(const sde_dose* d, const sde_spot* spots, int n) {
    for (int i = 0; i < n; ++i) {
        const sde_spot& s = spots[i];
        double un = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
        if (!(s.E_MeV > d->p.e_min_MeV) || !(s.E_MeV + 5.0 * s.sigma_E_MeV <= d->p.e_max_MeV) ||
            !(s.sigma_E_MeV >= 0.0) || !(s.sigma_xy_mm >= 0.0 && s.sigma_xy_mm < 1e4) ||
            !(s.sigma_angle_rad >= 0.0 && s.sigma_angle_rad < 1.0) || !(un > 0.0) || !isfinite(un) ||
            !isfinite(s.x_mm) || !isfinite(s.y_mm) || !isfinite(s.z_mm))
            return set_err(SDE_EINVAL, "spot %d is invalid (energy must lie in (e_min, e_max - 5 sigma_E], sigmas >= 0, direction non-zero)", i);
    }
    return SDE_OK;
}

static int stage_spots(sde_dose* d, const sde_spot* spots, int n_spots);

extern "C" int sde_dose_run(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed) {
    int rc = stage_spots(d, spots, n_spots);
    return rc ? rc : enqueue_transport(d, d->d_raw_spots, n_spots, seed);
}

extern "C" int sde_dose_run_range(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed,
                                  uint64_t first_history, uint64_t n_histories) {
    int rc = stage_spots(d, spots, n_spots);
    if (rc) return rc;
    const uint64_t end = n_histories > ~0ull - first_history ? ~0ull : first_history + n_histories;
    return enqueue_transport(d, d->d_raw_spots, n_spots, seed, first_history, end);
}

// Validates host spots and copies them (through the pinned staging buffer) to the
// device on the handle's stream.
static int stage_spots(sde_dose* d, const sde_spot* spots, int n_spots) {
    if (!d || !spots || n_spots < 1) return set_err(SDE_EINVAL, "bad run arguments");
    int rc = check_spots_host(d, spots, n_spots);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(d->device));
    rc = ensure_spot_capacity(d, n_spots);
    if (rc) return rc;
    // reuse the pinned staging buffer only after its previous copy finished
    CUDA_TRY(cudaEventSynchronize(d->stage_ev));
    if (n_spots > d->stage_cap) {
        if (d->h_stage) cudaFreeHost(d->h_stage);
        d->h_stage = nullptr;
        d->stage_cap = 0;
        CUDA_TRY(cudaMallocHost(&d->h_stage, (size_t)n_spots * sizeof(sde_spot)));
        d->stage_cap = n_spots;
    }
    memcpy(d->h_stage, spots, (size_t)n_spots * sizeof(sde_spot));
    CUDA_TRY(cudaMemcpyAsync(d->d_raw_spots, d->h_stage, (size_t)n_spots * sizeof(sde_spot),
                             cudaMemcpyHostToDevice, d->stream));
    CUDA_TRY(cudaEventRecord(d->stage_ev, d->stream));
    return SDE_OK;
}

extern "C" int sde_dose_run_device(sde_dose* d, const sde_spot* d_spots, int n_spots, uint64_t seed) {
    return sde_dose_run_device_range(d, d_spots, n_spots, seed, 0, ~0ull);
}

extern "C" int sde_dose_run_device_range(sde_dose* d, const sde_spot* d_spots, int n_spots, uint64_t seed,
                                         uint64_t first_history, uint64_t n_histories) {
    if (!d || !d_spots || n_spots < 1) return set_err(SDE_EINVAL, "bad run arguments");
    CUDA_TRY(cudaSetDevice(d->device));
    int rc = ensure_spot_capacity(d, n_spots);
    if (rc) return rc;
    const uint64_t end = n_histories > ~0ull - first_history ? ~0ull : first_history + n_histories;
    return enqueue_transport(d, d_spots, n_spots, seed, first_history, end);
}

// Autotuner: times the transport on a subsample of the plan under each
// candidate launch shape and keeps the fastest.  The tally does not depend on
// the launch shape, so only time is compared.
extern "C" int sde_dose_autotune(sde_dose* d, const sde_spot* spots, int n_spots, uint64_t seed,
                                 uint64_t max_histories, sde_tuning* best_out) {
    if (!d || !spots || n_spots < 1 || max_histories < 1) return set_err(SDE_EINVAL, "bad autotune arguments");
    int rc = check_spots_host(d, spots, n_spots);
    if (rc) return rc;
    CUDA_TRY(cudaSetDevice(d->device));
    uint64_t total = 0;
    for (int i = 0; i < n_spots; ++i) total += spots[i].n_hist;
    if (total == 0) return set_err(SDE_EINVAL, "autotune needs at least one history");
    double f = total > max_histories ? (double)max_histories / (double)total : 1.0;
    sde_spot* sub = (sde_spot*)malloc((size_t)n_spots * sizeof(sde_spot));
    if (!sub) return set_err(SDE_ENOMEM, "out of host memory");
    for (int i = 0; i < n_spots; ++i) {
        sub[i] = spots[i];
        if (spots[i].n_hist) sub[i].n_hist = (uint64_t)ceil((double)spots[i].n_hist * f);
    }
    static const sde_tuning cands[] = {
        {0, 8, 32, 32, 2, 1, 1}, {0, 8, 32, 16, 2, 1, 1}, {0, 4, 32, 32, 2, 1, 1}, {0, 8, 64, 32, 2, 1, 1},
        {0, 8, 32, 32, 1, 1, 1}, {0, 8, 32, 16, 1, 1, 1}, {0, 8, 32, 32, 2, 2, 1}, {0, 8, 32, 8, 2, 1, 1},
        {4, 8, 32, 32, 2, 1, 1}, {3, 8, 32, 32, 1, 1, 1}, {0, 8, 32, 32, 2, 1, 2},
    };
    const sde_tuning saved = d->tune;
    cudaEvent_t a = nullptr, b = nullptr;
    int out = SDE_OK;
    float best_ms = 1e30f;
    sde_tuning best = saved;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        out = set_err(SDE_ECUDA, "cudaEventCreate failed");
    } else {
        for (const sde_tuning& c : cands) {
            d->tune = c;
            if (c.blocks_per_sm == 0) d->tune.blocks_per_sm = 0;
            float t_best = 1e30f;
            for (int rep = 0; rep < 3 && out == SDE_OK; ++rep) {
                if (cudaEventRecord(a, d->stream) != cudaSuccess) out = set_err(SDE_ECUDA, "event record failed");
                if (out == SDE_OK) out = sde_dose_run(d, sub, n_spots, seed + rep);
                if (out == SDE_OK && cudaEventRecord(b, d->stream) != cudaSuccess)
                    out = set_err(SDE_ECUDA, "event record failed");
                float ms = 0.f;
                if (out == SDE_OK && (cudaEventSynchronize(b) != cudaSuccess ||
                                      cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
                    out = set_err(SDE_ECUDA, "event timing failed");
                if (out == SDE_OK && rep > 0) t_best = std::min(t_best, ms);  // first run warms up
            }
            if (out != SDE_OK) break;
            if (t_best < best_ms) {
                best_ms = t_best;
                best = c;
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    free(sub);
    d->tune = out == SDE_OK ? best : saved;
    int rc2 = sde_dose_reset(d);
    if (out == SDE_OK && rc2 != SDE_OK) out = rc2;
    if (out == SDE_OK) {
        // the tuning runs may have raised the device flag on a bad spot: clear it
        CUDA_TRY(cudaMemsetAsync(d->d_err, 0, sizeof(unsigned int), d->stream));
        CUDA_TRY(cudaStreamSynchronize(d->stream));
        if (best_out) *best_out = best;
    }
    return out;
}

static int read_counters(sde_dose* d, sde_balance* bal) {
    if (bal) {
        // the deposited energy of the balance is the sum of the tally
        CUDA_TRY(cudaMemsetAsync(d->d_counters + kCntDeposited, 0, sizeof(unsigned long long), d->stream));
        CUDA_TRY(launch_sum_u64(d->d_edep, d->nvox, d->d_counters + kCntDeposited, d->num_sms, d->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(d->h_counters, d->d_counters, kCntWords * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(cudaMemcpyAsync(d->h_counters + kCntWords, d->d_err, sizeof(unsigned int),
                             cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    unsigned int err = (unsigned int)(d->h_counters[kCntWords] & 0xffffffffu);
    if (bal) {
        const unsigned long long* c = d->h_counters;
        bal->incident = c[kCntIncident];
        bal->deposited = c[kCntDeposited];
        bal->escaped = c[kCntEscaped];
        bal->removed = c[kCntRemoved];
        bal->histories = c[kCntHistories];
        bal->steps = c[kCntSteps];
        bal->jumps_elastic = c[kCntJumpEl];
        bal->jumps_inelastic = c[kCntJumpInel];
    }
    if (err) {
        CUDA_TRY(cudaMemsetAsync(d->d_err, 0, sizeof(unsigned int), d->stream));
        CUDA_TRY(cudaStreamSynchronize(d->stream));
        return set_err(SDE_EDEVICE, "device error flag 0x%x:%s%s%s", err,
                       (err & kErrStepCap) ? " step cap reached (history stopped, energy counted as escaped);" : "",
                       (err & kErrBadSpot) ? " invalid device-resident spot (its histories were not run);" : "",
                       (err & kErrSecQueue) ? " secondary queue full (those secondaries' energy counted as removed);"
                                            : "");
    }
    return SDE_OK;
}

extern "C" int sde_dose_sync(sde_dose* d) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    CUDA_TRY(cudaSetDevice(d->device));
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    return read_counters(d, nullptr);
}

static int convert_into(sde_dose* d, double* dst) {
    double unit_J = ldexp(1.0, -d->p.fixed_point_shift) * kJoulePerMeV;
    double vol_kg_per_rho = d->h[0] * d->h[1] * d->h[2] * 1e-3 * 1e-3;  // mm^3 -> cm^3, g -> kg
    CUDA_TRY(launch_convert(d->d_edep, d->d_rho, d->nvox, unit_J, vol_kg_per_rho, dst, d->num_sms, d->stream));
    return SDE_OK;
}

extern "C" int sde_dose_fetch(sde_dose* d, double* dose_Gy, uint64_t* edep_fixed, sde_balance* bal) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    CUDA_TRY(cudaSetDevice(d->device));
    if (dose_Gy) {
        if (!d->d_dose) CUDA_TRY(cudaMalloc(&d->d_dose, d->nvox * sizeof(double)));
        int rc = convert_into(d, d->d_dose);
        if (rc) return rc;
        CUDA_TRY(cudaMemcpyAsync(dose_Gy, d->d_dose, d->nvox * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    }
    if (edep_fixed)
        CUDA_TRY(cudaMemcpyAsync(edep_fixed, d->d_edep, d->nvox * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                 d->stream));
    return read_counters(d, bal);
}

extern "C" int sde_dose_fetch_device(sde_dose* d, double* d_dose_Gy, uint64_t* d_edep_fixed, sde_balance* bal) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    CUDA_TRY(cudaSetDevice(d->device));
    if (d_dose_Gy) {
        int rc = convert_into(d, d_dose_Gy);
        if (rc) return rc;
    }
    if (d_edep_fixed)
        CUDA_TRY(cudaMemcpyAsync(d_edep_fixed, d->d_edep, d->nvox * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                 d->stream));
    if (bal) return read_counters(d, bal);
    return SDE_OK;
}

extern "C" int sde_dose_fetch_device_f32(sde_dose* d, float* d_dose_Gy) {
    if (!d || !d_dose_Gy) return set_err(SDE_EINVAL, "null argument");
    CUDA_TRY(cudaSetDevice(d->device));
    double unit_J = ldexp(1.0, -d->p.fixed_point_shift) * kJoulePerMeV;
    double vol_kg_per_rho = d->h[0] * d->h[1] * d->h[2] * 1e-3 * 1e-3;
    CUDA_TRY(launch_convert_f32(d->d_edep, d->d_rho, d->nvox, unit_J, vol_kg_per_rho, d_dose_Gy, d->num_sms,
                                d->stream));
    return SDE_OK;
}

extern "C" int sde_dose_reset(sde_dose* d) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    CUDA_TRY(cudaSetDevice(d->device));
    CUDA_TRY(cudaMemsetAsync(d->d_edep, 0, d->nvox * sizeof(unsigned long long), d->stream));
    CUDA_TRY(cudaMemsetAsync(d->d_counters, 0, kCntWords * sizeof(unsigned long long), d->stream));
    return SDE_OK;
}

extern "C" void sde_dose_destroy(sde_dose* d) {
    if (!d) return;
    cudaSetDevice(d->device);
    cudaStreamSynchronize(d->stream);
    free_all(d);
    delete d;
}

extern "C" int sde_dose_info(const sde_dose* d, uint64_t* n_vox, int* table_points, double* e_min,
                             double* e_max, int* n_mats) {
    if (!d) return set_err(SDE_EINVAL, "null handle");
    if (n_vox) *n_vox = d->nvox;
    if (table_points) *table_points = d->p.table_points;
    if (e_min) *e_min = d->p.e_min_MeV;
    if (e_max) *e_max = d->p.e_max_MeV;
    if (n_mats) *n_mats = d->n_mats;
    return SDE_OK;
}

extern "C" int sde_dose_tables(const sde_dose* d, int m, float* out, float* rates_out, double* csda_out) {
    if (!d || m < 0 || m >= d->n_mats) return set_err(SDE_EINVAL, "bad handle or material index");
    CUDA_TRY(cudaSetDevice(d->device));
    const size_t N = d->p.table_points;
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    if (out)
        CUDA_TRY(cudaMemcpy(out, d->d_raw + (size_t)m * N * kRawFields, N * kRawFields * sizeof(float),
                            cudaMemcpyDeviceToHost));
    if (rates_out) {
        // compact [N][2*MAX] -> [N][2*n_el]
        float* tmp = (float*)malloc(N * 2 * SDE_MAX_ELEMENTS * sizeof(float));
        if (!tmp) return set_err(SDE_ENOMEM, "out of host memory");
        cudaError_t e = cudaMemcpy(tmp, d->d_jrates + (size_t)m * N * 2 * SDE_MAX_ELEMENTS,
                                   N * 2 * SDE_MAX_ELEMENTS * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            free(tmp);
            return set_err(SDE_ECUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
        }
        int ne = d->mats[m].n_el;
        double lr = log(d->p.e_max_MeV / d->p.e_min_MeV);
        for (size_t k = 0; k < N; ++k) {
            double E = d->p.e_min_MeV * exp(lr * (double)k / (double)(N - 1));
            for (int c = 0; c < 2; ++c)
                for (int i = 0; i < ne; ++i) {
                    double v = tmp[k * 2 * SDE_MAX_ELEMENTS + c * SDE_MAX_ELEMENTS + i];
                    // the device keeps elastic rates multiplied by E^2
                    rates_out[k * 2 * ne + c * ne + i] = (float)(c == 0 ? v / (E * E) : v);
                }
        }
        free(tmp);
    }
    if (csda_out)
        CUDA_TRY(cudaMemcpy(csda_out, d->d_csda + (size_t)m * N, N * sizeof(double), cudaMemcpyDeviceToHost));
    return SDE_OK;
}

extern "C" int sde_dose_probe_steps(sde_dose* d, int m, double rho, double E, uint64_t seed, uint64_t h0, int n,
                                    float* E_out, float* cos_out, int* jump_out, float* ux_out, float* uy_out) {
    if (!d || m < 0 || m >= d->n_mats || n < 1 || !(rho >= 0.0) || !(E > d->p.e_min_MeV) ||
        !(E <= d->p.e_max_MeV))
        return set_err(SDE_EINVAL, "bad probe arguments");
    CUDA_TRY(cudaSetDevice(d->device));
    float* buf = nullptr;
    size_t per = (size_t)n;
    CUDA_TRY(cudaMalloc(&buf, per * 5 * sizeof(float)));
    KParams P = make_kparams(d, 0, seed);
    float* Eo = buf;
    float* co = buf + per;
    int* jo = (int*)(buf + 2 * per);
    float* uxo = buf + 3 * per;
    float* uyo = buf + 4 * per;
    cudaError_t e = launch_probe(P, m, (float)rho, (float)E, h0, n, Eo, co, jo, uxo, uyo, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e == cudaSuccess && E_out) e = cudaMemcpy(E_out, Eo, per * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cos_out) e = cudaMemcpy(cos_out, co, per * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && jump_out) e = cudaMemcpy(jump_out, jo, per * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ux_out) e = cudaMemcpy(ux_out, uxo, per * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && uy_out) e = cudaMemcpy(uy_out, uyo, per * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return set_err(SDE_ECUDA, "probe failed: %s", cudaGetErrorString(e));
    return SDE_OK;
}
