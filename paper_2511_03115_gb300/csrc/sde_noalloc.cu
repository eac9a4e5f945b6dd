// sde_noalloc.cu -- a transport entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework that
// owns every device allocation (a memory pool or arena it must account for), and
// real-time services that forbid allocation after start-up because an allocation
// can block and fail at an arbitrary point.  sde_transport_noalloc serves them:
// the caller passes the phantom, the spots and the tally buffer in device memory
// it already owns, and every other buffer the transport needs (physics tables,
// spot records in device form, the history prefix, the work-queue cursor and the
// balance counters) lives in one fixed array compiled into this library.
//
// The array is a file-scope __device__ object of kScratchBytes (1 MiB).  Every
// GPU on which the library is loaded holds its own copy until the process exits.
// Host code cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it.
//
// The caller's voxel words are checked on the device before the transport reads
// any table with them (material id < n_mats, density finite in [0, 1e3)): a bad
// word raises a device error bit and leaves the work queue empty, so no history
// runs and no table is indexed out of range.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "sde_internal.cuh"
#include "sde_tables.h"
#include "sde_transport.h"

namespace {

using namespace sde;

constexpr size_t kScratchBytes = size_t(1) << 20;
constexpr int kNoallocMaxMaterials = 4;
constexpr int kNoallocMaxTablePoints = 256;
constexpr int kNoallocMaxSpots = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device error bit of this entry point beside the transport's own (step cap 1, bad spot 2).
constexpr unsigned int kErrBadVoxel = 8u;

// Checks every caller-supplied voxel word before any kernel indexes a table with it:
// material id < n_mats and density finite in [0, 1e3) g/cm^3 (the checks sde_dose_create
// makes on the host).  A bad word raises kErrBadVoxel and moves the work-queue cursor
// (set by the spot preparation just before) past every history id, so the transport
// that follows claims no history.
__global__ void k_check_voxels(const uint32_t* __restrict__ vox, size_t nv, int n_mats, unsigned int* err,
                               unsigned long long* cursor) {
    bool bad = false;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
        const uint32_t w = vox[v];
        const float rho = __uint_as_float(w & ~15u);
        bad |= (int)(w & 15u) >= n_mats || !(rho >= 0.f && rho < 1e3f);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        atomicOr(err, kErrBadVoxel);
        atomicExch(cursor, 1ull << 62);  // above any plan's history count: the queue is drained
    }
}

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

int noalloc_fail(int code, const char* msg) {
    set_last_error(msg);
    return code;
}

// Device address of this device's scratch array (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int sde_transport_noalloc(int nx, int ny, int nz, const double voxel_mm[3], const double origin_mm[3],
                                     const uint32_t* d_vox, const sde_material* mats, int n_mats,
                                     const sde_params* params, const sde_spot* d_spots, int n_spots,
                                     uint64_t seed, unsigned long long* d_edep, sde_balance* bal,
                                     unsigned int* d_status, void* cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !voxel_mm || !origin_mm || !d_vox || !mats || !params || !d_spots ||
        !d_edep)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: null pointer or empty grid");
    if ((size_t)nx * ny * nz > (size_t)INT32_MAX)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: grid has more than 2^31-1 voxels");
    if (n_mats < 1 || n_mats > kNoallocMaxMaterials)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: n_mats must be 1..4 (scratch limit)");
    if (n_spots < 1 || n_spots > kNoallocMaxSpots)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: n_spots must be 1..4096 (scratch limit)");
    const sde_params& p = *params;
    if (p.theta_cut_sigmas != 0.0)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: the energy-dependent cut-off needs sde_dose_create");
    if (p.secondary_fraction != 0.0)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: the branching model (secondary_fraction) needs "
                                        "sde_dose_create");
    if (p.table_points < 64 || p.table_points > kNoallocMaxTablePoints)
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: table_points must be 64..256 (scratch limit)");
    if (!(p.step_cm > 0.0 && p.step_cm <= 1.0 && p.msc_z_cm > 0.0 && p.F > 0.0 && p.F < 1.0 &&
          p.theta_cut_rad > 0.0 && p.theta_cut_rad < 3.0 && p.backscatter_rad > 0.0 && p.backscatter_rad < 1.5 &&
          p.e_min_MeV > 0.0 && p.K > 0.0 && p.inel_u_lo >= 0.0 && p.inel_u_hi <= 1.0 &&
          p.inel_u_lo <= p.inel_u_hi && p.km_r >= 0.0 && p.km_r < 1.0 && p.e_max_MeV > 2.0 * p.e_min_MeV &&
          p.e_max_MeV <= 1000.0 && (p.tally_mode == 0 || p.tally_mode == 1) && p.fixed_point_shift >= 0 &&
          p.fixed_point_shift <= 30 && p.max_steps > 0 && p.physics_mask >= 0 && p.physics_mask <= SDE_PHYS_ALL))
        return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: invalid sde_params");
    for (int a = 0; a < 3; ++a)
        if (!(voxel_mm[a] > 0.0))
            return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: voxel size must be > 0");

    MatHost mh[kNoallocMaxMaterials];
    MatJump mj[kNoallocMaxMaterials];
    char msg[200];
    for (int i = 0; i < n_mats; ++i) {
        if (resolve_material(mats[i], &mh[i], msg, sizeof msg) != SDE_OK)
            return noalloc_fail(SDE_EINVAL, msg);
        memset(&mj[i], 0, sizeof mj[i]);
        mj[i].n_el = mh[i].n_el;
        for (int e = 0; e < mh[i].n_el; ++e) {
            mj[i].Z[e] = mh[i].Z[e];
            mj[i].A[e] = (float)mh[i].A[e];
            mj[i].m2[e] = (float)(mh[i].Z[e] == 1 ? kProtonMass : mh[i].A[e] * kAtomicMassUnit);
        }
    }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SDE_ECUDA, "sde_transport_noalloc: no usable current device");
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return noalloc_fail(SDE_ECUDA, "sde_transport_noalloc: cannot query the device");
    unsigned char* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess)
        return noalloc_fail(SDE_ECUDA, "sde_transport_noalloc: cudaGetSymbolAddress of the scratch array failed");

    // Scratch layout (each part 256-byte aligned).
    const int N = p.table_points;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char* q = base + off;
        off += align256(bytes);
        return q;
    };
    auto* counters = (unsigned long long*)carve(kCntWords * sizeof(unsigned long long));
    auto* err = (unsigned int*)carve(sizeof(unsigned int));
    auto* dep = (unsigned long long*)carve(2 * sizeof(unsigned long long));  // tally sum before / after
    auto* d_mh = (MatHost*)carve(n_mats * sizeof(MatHost));
    auto* d_mj = (MatJump*)carve(n_mats * sizeof(MatJump));
    const size_t table_bytes = (size_t)n_mats * N * kRowFloat4 * sizeof(float4);
    auto* table = (float4*)carve(table_bytes);
    auto* raw = (float*)carve((size_t)n_mats * N * kRawFields * sizeof(float));
    auto* jrates = (float*)carve((size_t)n_mats * N * 2 * SDE_MAX_ELEMENTS * sizeof(float));
    auto* pick = (float2*)carve((size_t)n_mats * N * 2 * SDE_MAX_ELEMENTS * sizeof(float2));
    auto* mott_g = (float4*)carve((size_t)N * sizeof(float4));
    auto* mott_r = (float2*)carve((size_t)N * kMottKnots * sizeof(float2));
    auto* csda = (double*)carve((size_t)n_mats * N * sizeof(double));
    auto* spots = (SpotDev*)carve((size_t)n_spots * sizeof(SpotDev));
    auto* prefix = (unsigned long long*)carve(((size_t)n_spots + 1) * sizeof(unsigned long long));
    if (off > kScratchBytes) return noalloc_fail(SDE_EINVAL, "sde_transport_noalloc: inputs exceed the scratch array");

#define NA_TRY(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            char m_[256];                                                                \
            snprintf(m_, sizeof m_, "%s failed: %s", #call, cudaGetErrorString(e_));     \
            set_last_error(m_);                                                          \
            return SDE_ECUDA;                                                            \
        }                                                                                \
    } while (0)

    // The scratch keeps the previous call's contents: clear the counters and flag.
    NA_TRY(cudaMemsetAsync(counters, 0, kCntWords * sizeof(unsigned long long), st));
    NA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    NA_TRY(cudaMemcpyAsync(d_mh, mh, n_mats * sizeof(MatHost), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_mj, mj, n_mats * sizeof(MatJump), cudaMemcpyHostToDevice, st));

    TableBuild tb;
    tb.N = N;
    tb.n_mats = n_mats;
    tb.e_min = p.e_min_MeV;
    tb.e_max = p.e_max_MeV;
    tb.K = p.K;
    tb.F = p.F;
    tb.z = p.msc_z_cm;
    tb.step = p.step_cm;
    tb.theta_cut = p.theta_cut_rad;
    tb.theta_back = p.backscatter_rad;
    tb.mask = p.physics_mask;
    tb.d_mats = d_mh;
    tb.d_raw = raw;
    tb.d_jrates = jrates;
    tb.d_csda = csda;
    tb.d_table = table;
    tb.d_pick = pick;
    tb.d_mott_g = mott_g;
    tb.d_mott_r = mott_r;
    NA_TRY(build_tables(tb, st));
    NA_TRY(launch_prep(d_spots, n_spots, spots, prefix, counters, err, origin_mm, voxel_mm, p.e_min_MeV,
                       p.e_max_MeV, st));
    const size_t nv = (size_t)nx * ny * nz;
    k_check_voxels<<<sms * 4, 256, 0, st>>>(d_vox, nv, n_mats, err, counters + kCntCursor);
    NA_TRY(cudaGetLastError());
    if (bal) {  // the tally may already hold earlier calls' deposits: the balance takes the difference
        NA_TRY(cudaMemsetAsync(dep, 0, 2 * sizeof(unsigned long long), st));
        NA_TRY(launch_sum_u64(d_edep, nv, dep, sms, st));
    }

    KParams P;
    memset(&P, 0, sizeof P);
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.n_mats = n_mats;
    P.inv_hx = (float)(1.0 / voxel_mm[0]);
    P.inv_hy = (float)(1.0 / voxel_mm[1]);
    P.inv_hz = (float)(1.0 / voxel_mm[2]);
    P.step_mm = (float)(p.step_cm * 10.0);
    P.half_step_mm = (float)(p.step_cm * 5.0);
    P.sv_xy = make_float2((float)(p.step_cm * 10.0 / voxel_mm[0]), (float)(p.step_cm * 10.0 / voxel_mm[1]));
    P.sv_z = (float)(p.step_cm * 10.0 / voxel_mm[2]);
    P.hv_xy = make_float2((float)(p.step_cm * 5.0 / voxel_mm[0]), (float)(p.step_cm * 5.0 / voxel_mm[1]));
    P.hv_z = (float)(p.step_cm * 5.0 / voxel_mm[2]);
    P.inv_delta_cm = (float)(1.0 / p.step_cm);
    P.e_min = (float)p.e_min_MeV;
    P.e_max = (float)p.e_max_MeV;
    P.qscale = (float)ldexp(1.0, p.fixed_point_shift);
    P.max_steps = p.max_steps;
    P.mask = p.physics_mask;
    P.tally_mode = p.tally_mode;
    P.N = N;
    P.lg2_emin = (float)log2(p.e_min_MeV);
    P.inv_dlg2 = (float)((N - 1) / (log2(p.e_max_MeV) - log2(p.e_min_MeV)));
    double s_cut = 2.0 * sin(0.5 * p.theta_cut_rad) * sin(0.5 * p.theta_cut_rad);
    P.s_cut = (float)s_cut;
    P.ruth_span = (float)(1.0 / s_cut - 0.5);
    P.s_back = (float)(2.0 * sin(0.5 * p.backscatter_rad) * sin(0.5 * p.backscatter_rad));
    P.inel_lo = (float)p.inel_u_lo;
    P.inel_span = (float)(p.inel_u_hi - p.inel_u_lo);
    P.km_r = (float)p.km_r;
    P.batch = 32;
    P.refill_min = 32;
    P.aggregate = 0;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.rk0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        P.rk1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.strag_on = (p.physics_mask & SDE_PHYS_STRAGGLING) ? 1.f : 0.f;
    P.mcs_on = (p.physics_mask & SDE_PHYS_MCS) ? 1.f : 0.f;
    P.vox = d_vox;
    P.edep = d_edep;
    P.table = table;
    P.jrates = jrates;
    P.pick = pick;
    P.mott_g = mott_g;
    P.mott_r = mott_r;
    P.mott_lg2_lo = (float)mott_knot_lo(p.theta_cut_rad);
    P.mott_inv_dj = (float)((kMottKnots - 1) / -mott_knot_lo(p.theta_cut_rad));
    P.mats = d_mj;
    P.spots = spots;
    P.prefix = prefix;
    P.h_end = ~0ull;
    P.n_spots = n_spots;
    P.counters = counters;
    P.err = err;

    const int block = 8 * 32;
    int per_sm = transport_max_blocks_per_sm(block, table_bytes, false, p.tally_mode, false);
    if (per_sm < 1) return noalloc_fail(SDE_ECUDA, "sde_transport_noalloc: transport kernel cannot be resident");
    NA_TRY(launch_transport(P, sms * per_sm, block, table_bytes, false, st));

    if (d_status) NA_TRY(cudaMemcpyAsync(d_status, err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
    if (bal) {
        NA_TRY(launch_sum_u64(d_edep, nv, dep + 1, sms, st));
        unsigned long long c[kCntWords], sums[2];
        unsigned int flag = 0;
        NA_TRY(cudaMemcpyAsync(c, counters, sizeof c, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaMemcpyAsync(sums, dep, sizeof sums, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaStreamSynchronize(st));
        bal->incident = c[kCntIncident];
        bal->deposited = sums[1] - sums[0];  // this call's deposit (unsigned difference, exact)
        bal->escaped = c[kCntEscaped];
        bal->removed = c[kCntRemoved];
        bal->histories = c[kCntHistories];
        bal->steps = c[kCntSteps];
        bal->jumps_elastic = c[kCntJumpEl];
        bal->jumps_inelastic = c[kCntJumpInel];
        if (flag)
            return noalloc_fail(SDE_EDEVICE,
                                (flag & kErrBadVoxel)
                                    ? "sde_transport_noalloc: a voxel word has a material id >= n_mats or a density "
                                      "outside [0, 1e3) g/cm3; no history was run"
                                    : (flag & kErrStepCap) ? "sde_transport_noalloc: step cap reached"
                                                           : "sde_transport_noalloc: invalid spot");
    }
#undef NA_TRY
    return SDE_OK;
}
