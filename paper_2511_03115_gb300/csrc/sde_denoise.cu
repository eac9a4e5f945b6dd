// sde_denoise.cu -- tensor-core (tcgen05) kernels of the learned dose denoiser.
//
// The denoiser is a 3D convolutional encoder-decoder applied to a low-history dose
// and the density map; its convolutions are implicit GEMMs on the 5th-generation
// tensor core with BF16 operands in shared memory and FP32 accumulators in tensor
// memory.  This file holds the GEMM building block and its C entry point.
#include <cuda_bf16.h>
#include <stdio.h>

#include <mutex>

#include "sde_dose.h"
#include "sde_tables.h"
#include "sde_denoise.h"
#include "sde_umma.cuh"

namespace sde {

namespace {

constexpr long long kWaitCycles = 1ll << 31;  // ~1 s at 2 GHz: a stuck wait sets the error flag

// D[M x N] (FP32, row-major) = A[M x K] x B[N x K]^T with A, B row-major BF16 (both
// K-major).  One CTA of 128 threads per 128-row tile of D; K is staged in chunks of
// 64 through shared memory in the core-matrix layout; one thread issues the MMAs.
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* __restrict__ A,
                                                   const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
                                                   int M, int N, int K, unsigned int* status) {
    constexpr int KC = 64;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + 128 * KC * 2;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 256 * KC * 2);
    uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const uint32_t ncols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
    if (warp == 0) {
        umma::tmem_alloc(slot, ncols);
        umma::tmem_relinquish();
    }
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *slot;
    const uint32_t idesc = umma::idesc_bf16_f32(128, N);
    bool ok = true;
    int it = 0;
    for (int k0 = 0; k0 < K; k0 += KC, ++it) {
        const int kc = min(KC, K - k0);
        const int q8 = kc >> 3;
        for (int c = tid; c < 128 * q8; c += 128) {
            int r = c / q8, q = c - r * q8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M) v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + k0 + q * 8);
            *reinterpret_cast<uint4*>(sA + umma::core_offset(r, q * 8, kc)) = v;
        }
        for (int c = tid; c < N * q8; c += 128) {
            int r = c / q8, q = c - r * q8;
            uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k0 + q * 8);
            *reinterpret_cast<uint4*>(sB + umma::core_offset(r, q * 8, kc)) = v;
        }
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            for (int ks = 0; ks < (kc >> 4); ++ks) {
                uint64_t ad = umma::smem_desc(umma::smem_addr(sA) + ks * 256, 128, 16 * kc);
                uint64_t bd = umma::smem_desc(umma::smem_addr(sB) + ks * 256, 128, 16 * kc);
                umma::mma_bf16(tbase, ad, bd, idesc, (k0 > 0 || ks > 0) ? 1u : 0u);
            }
            umma::mma_commit(mbar);
        }
        bool done = umma::mbar_wait(mbar, (uint32_t)(it & 1), kWaitCycles);
        umma::fence_after_sync();
        if (!__syncthreads_and(done ? 1 : 0)) {
            ok = false;
            break;
        }
    }
    if (ok) {
        for (int c = 0; c < N; c += 8) {
            float v[8];
            umma::tmem_ld8(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            int row = m0 + 32 * warp + lane;
            if (row < M)
                for (int j = 0; j < 8; ++j) D[(size_t)row * N + c + j] = v[j];
        }
    } else if (tid == 0) {
        atomicOr(status, 1u);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tbase, ncols);
}

std::mutex g_status_mutex;
unsigned int* g_status[64] = {};

// A device status word per device (allocated on first use).
cudaError_t status_word(unsigned int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_status_mutex);
    if (!g_status[dev]) {
        e = cudaMalloc(&g_status[dev], sizeof(unsigned int));
        if (e != cudaSuccess) return e;
        e = cudaMemset(g_status[dev], 0, sizeof(unsigned int));
        if (e != cudaSuccess) return e;
    }
    *out = g_status[dev];
    return cudaSuccess;
}

int report(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SDE_OK;
    char m[256];
    snprintf(m, sizeof m, "%s: %s", what, cudaGetErrorString(e));
    set_last_error(m);
    return e == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA;
}

}  // namespace

cudaError_t denoise_status_word(unsigned int** out) { return status_word(out); }

// Reads and clears the device status word; SDE_EDEVICE when a tensor-core wait timed out.
int denoise_check_status(cudaStream_t st) {
    unsigned int* d_status = nullptr;
    int rc = report(status_word(&d_status), "status word");
    if (rc) return rc;
    unsigned int h = 0;
    rc = report(cudaMemcpyAsync(&h, d_status, sizeof h, cudaMemcpyDeviceToHost, st), "status copy");
    if (rc) return rc;
    rc = report(cudaStreamSynchronize(st), "status sync");
    if (rc) return rc;
    if (h) {
        cudaMemsetAsync(d_status, 0, sizeof h, st);
        cudaStreamSynchronize(st);
        set_last_error("a tensor-core completion wait timed out (result not written)");
        return SDE_EDEVICE;
    }
    return SDE_OK;
}

}  // namespace sde

using namespace sde;

extern "C" int sde_gemm_bf16(const void* d_A, const void* d_B, float* d_D, int M, int N, int K, void* stream) {
    if (!d_A || !d_B || !d_D || M < 1 || N < 16 || N > 256 || (N % 16) || K < 16 || (K % 16)) {
        set_last_error("sde_gemm_bf16: need M >= 1, N a multiple of 16 in [16, 256], K a multiple of 16");
        return SDE_EINVAL;
    }
    if (((uintptr_t)d_A | (uintptr_t)d_B) & 15) {
        set_last_error("sde_gemm_bf16: A and B must be 16-byte aligned");
        return SDE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* d_status = nullptr;
    int rc = report(status_word(&d_status), "status word");
    if (rc) return rc;
    const size_t smem = 128 * 64 * 2 + 256 * 64 * 2 + 64;
    rc = report(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                "cudaFuncSetAttribute");
    if (rc) return rc;
    k_gemm_bf16<<<(M + 127) / 128, 128, smem, st>>>(static_cast<const __nv_bfloat16*>(d_A),
                                                       static_cast<const __nv_bfloat16*>(d_B), d_D, M, N, K,
                                                       d_status);
    rc = report(cudaGetLastError(), "k_gemm_bf16 launch");
    if (rc) return rc;
    return denoise_check_status(st);
}

// ============================================================================
// 3D convolution (3x3x3, stride 1, zero padding 1) as implicit GEMMs on the tensor
// core.  Activations are channels-last BF16: x[n][z][y][x][c].  Weights w[co][tap][ci]
// (tap = 9 kz + 3 ky + kx).
// ============================================================================
namespace sde {
namespace {

// ----------------------------------------------------------------------------
// Brick convolution.  A work item computes Ty full output rows (all x) of one z plane
// for Cp output channels.  Per 16-channel chunk of Cin the zero-padded input "brick" --
// planes z-1..z+1, rows y0-1..y0+Ty, columns -1..W -- is staged in shared memory once,
// as two 8-channel planes in which brick position f = (zb Yb + yb) P + xp (P = W + 2,
// Yb = Ty + 2) holds 16 bytes.  In that layout 8 consecutive positions form a K-major
// core matrix, so the A operand of tap (dz, dy, dx) for an M tile starting at brick
// position f0 is the same buffer read from f0 + (dz Yb + dy) P + dx: the 27 taps are 27
// descriptor offsets, not 27 copies.  The input is padded channel-group-major, so each
// (channel group, plane) part of the brick is one contiguous run of Yb P x 16 bytes in
// global memory and a chunk arrives in six bulk copies.  When W is a multiple of 128 an M
// tile is 128 consecutive x of one output row and no padding column is computed;
// otherwise M tiles of 128 consecutive positions cover the Ty rows including their
// padding columns and the epilogue drops the rows that are not output voxels.
//
// Persistent and warp-specialised: the producer warp streams (brick, weight) chunks into
// a ring of shared-memory stages, one bulk copy per lane (each stage's "full" barrier
// completes when the bytes of its copies have landed); one thread in each of two MMA
// warps issues tcgen05.mma for the M tiles of its parity into one of two tensor-memory
// accumulators, and both release stages and accumulators through tcgen05.commit; the
// kConvWorkers epilogue warps turn a finished accumulator into output (bias, leaky ReLU,
// BF16 or FP32 store) while the tensor core works on the next item.  Every wait is bounded; a timeout sets a shared abort flag that
// ends all roles' loops, and the producer waits for its copies in flight before the CTA
// exits.
// ----------------------------------------------------------------------------
constexpr int kPipeStages = 2;
constexpr int kPipeHeader = 1024;  // barriers, tensor-memory slot, abort flag

__device__ __forceinline__ bool pipe_wait(uint64_t* m, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!umma::mbar_try_wait(m, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Epilogue warps of the brick convolution; two share each tensor-memory lane quarter
// (warp & 3).  The two MMA warps and the producer warp follow them.
constexpr int kConvWorkers = 8;
constexpr int kConvWorkerThreads = 32 * kConvWorkers;
constexpr int kConvThreads = kConvWorkerThreads + 96;

// AND of a predicate over the NT worker threads of a kernel (its warps 0 .. NT/32 - 1),
// named barrier 1.
template <int NT>
__device__ __forceinline__ bool workers_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}

// Brick position of output row 0's first M-tile row, shifted to tile m (tap offsets are
// added to it): row tiles are 128 x of one output row, flat tiles 128 consecutive positions
// starting at output (y0, x = -1).
__device__ __forceinline__ int tile_base(int m, bool rowtile, int P, int Yb, int tpr) {
    return rowtile ? (Yb + 1) * P + 1 + (m / tpr) * P + (m % tpr) * 128 : (Yb + 1) * P + 128 * m;
}

// The 27 x TILES MMAs of one channel chunk, fully unrolled so that the issuing thread spends
// one integer add per instruction: A's start field is the stage's plus (tile base + tap
// offset), B's steps by one tap tile (Cp x 16 BF16 = 2 Cp units of 16 bytes).  The start
// fields stay within 14 bits (shared addresses below 256 KB, lowest start one position
// into the stage), so adding to the low word never carries or borrows into the others.
template <int TILES, int PAR>
__device__ __forceinline__ void conv_chunk_mma(uint32_t dacc, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo,
                                               uint32_t b_hi, uint32_t idesc, int Cp, const int (&toff)[27],
                                               bool rowtile, int P, int Yb, int tpr, uint32_t first_accum) {
    int tb[TILES];
#pragma unroll
    for (int m = PAR; m < TILES; m += 2) tb[m] = tile_base(m, rowtile, P, Yb, tpr);
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const uint32_t bl = b_lo + (uint32_t)(2 * Cp * t);
#pragma unroll
        for (int m = PAR; m < TILES; m += 2)
            umma::mma_bf16_lohi(dacc + (uint32_t)(m * Cp), a_lo + (uint32_t)(tb[m] + toff[t]), a_hi, bl, b_hi, idesc,
                                t > 0 ? 1u : first_accum);
    }
}

// Folded variant (one 128-voxel row per tile): per (z, y) tap pair q one MMA of N = 3 Cp whose
// B is the three consecutive x-tap tiles of the pair and whose A is the pair's dx = 0
// window; accumulator column block j then holds the window's product with the dx = j - 1
// weights, and the epilogue adds the blocks shifted by one position.
template <int TILES, int PAR>
__device__ __forceinline__ void conv_chunk_mma_fold(uint32_t dacc, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo,
                                                    uint32_t b_hi, uint32_t idesc, int Cp, const int (&toff)[27],
                                                    int P, int Yb, uint32_t first_accum) {
    int tb[TILES];
#pragma unroll
    for (int m = PAR; m < TILES; m += 2) tb[m] = tile_base(m, true, P, Yb, 1);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const uint32_t bl = b_lo + (uint32_t)(6 * Cp * q);  // taps 3q .. 3q+2
#pragma unroll
        for (int m = PAR; m < TILES; m += 2)
            umma::mma_bf16_lohi(dacc + (uint32_t)(3 * m * Cp), a_lo + (uint32_t)(tb[m] + toff[3 * q + 1]), a_hi, bl,
                                b_hi, idesc, q > 0 ? 1u : first_accum);
    }
}

// Named barrier over the 128 threads of one group of four epilogue warps.
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Work item of the brick convolution: (sample, Cout part, row block, z plane).
struct BrickItem {
    int n, part, y0, z;
};
__device__ __forceinline__ BrickItem brick_item(const BrickPlan& b, int D, int item) {
    BrickItem t;
    t.z = item % D;
    item /= D;
    t.y0 = (item % b.nyb) * b.Ty;
    item /= b.nyb;
    t.part = item % b.nsplit;
    t.n = item / b.nsplit;
    return t;
}

__global__ void __launch_bounds__(kConvThreads, 1) k_conv3d_brick(ConvArgs a, BrickPlan b) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Cin = a.Cin, Cp = b.Cp, W = a.W, H = a.H, D = a.D;
    const int P = b.P, Yb = b.Yb;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [kPipeStages]
    uint64_t* empty = full + kPipeStages;                 // [kPipeStages]
    uint64_t* tfull = empty + kPipeStages;                // [2]
    uint64_t* tempty = tfull + 2;                         // [2]
    uint64_t* wfull = tempty + 2;                         // resident weights landed
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 128);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 132);
    const uint32_t s_stage0 = umma::smem_addr(smem) + kPipeHeader;
    if (warp == 0) {
        umma::tmem_alloc(slot, (uint32_t)b.tcols);
        umma::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kPipeStages; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 2);  // one commit per MMA thread
        }
        for (int s = 0; s < 2; ++s) {
            umma::mbar_init(&tfull[s], 2);
            umma::mbar_init(&tempty[s], kConvWorkerThreads);
        }
        umma::mbar_init(wfull, 1);
        *abort_flag = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *slot;
    const int nchunk = Cin >> 4;
    const int acc_cols = b.tiles * Cp * (b.fold ? 3 : 1);
    const int tpr = W >> 7;                          // row tiles: M tiles per output row
    const uint32_t w_chunk = (uint32_t)(27 * Cp * 32);  // bytes of one chunk's weights
    const uint32_t s_wres = s_stage0 + (uint32_t)(kPipeStages * b.stage);
    const Pcg pg{D, H, W};

    if (warp == kConvWorkers + 2) {
        // producer warp: lane 0 waits for a free stage and posts the bytes it will receive, then
        // lanes 0-5 issue the six brick runs and lane 6 the weight chunk (one thread can issue
        // a bulk copy only every ~100 cycles, which made the copies the bottleneck of the
        // 96-channel layer)
        const int Gin = Cin >> 3;
        int k = 0;
        if (b.wres && lane == 0) {
            umma::mbar_arrive_expect_tx(wfull, (uint32_t)nchunk * w_chunk);
            umma::bulk_g2s(s_wres, a.wpk, (uint32_t)nchunk * w_chunk, wfull);
        }
        bool ok = true;
        for (int item = blockIdx.x; ok && item < b.items; item += gridDim.x) {
            const BrickItem t = brick_item(b, D, item);
            const __nv_bfloat16* wpart = a.wpk + (size_t)t.part * nchunk * 27 * Cp * 16;
            // one (channel group, plane) part of the brick: padded rows y0 .. y0+Yb-1, fewer in a
            // last row block that passes H (the rows it leaves stale feed only outputs y >= H,
            // which the epilogue drops)
            const int rows = Yb < H + 2 - t.y0 ? Yb : H + 2 - t.y0;
            const uint32_t run = (uint32_t)(rows * P * 16);
            const uint32_t slot = (uint32_t)(Yb * P * 16);
            for (int c = 0; c < nchunk; ++c, ++k) {
                const int s = k % kPipeStages, u = k / kPipeStages;
                bool got = true;
                if (lane == 0 && u >= 1) got = pipe_wait(&empty[s], (uint32_t)(u - 1) & 1u, abort_flag);
                if (!__shfl_sync(0xffffffffu, got, 0)) {
                    ok = false;
                    break;
                }
                const uint32_t st = s_stage0 + (uint32_t)(s * b.stage);
                if (lane == 0) umma::mbar_arrive_expect_tx(&full[s], 6u * run + (b.wres ? 0u : w_chunk));
                __syncwarp();
                if (lane < 6) {  // rows y0-1 .. y0+Ty of plane z+zb-1, columns -1 .. W
                    const int gg = lane / 3, zb = lane - 3 * gg;
                    umma::bulk_g2s(st + 128u + (uint32_t)(gg * b.plane) + (uint32_t)zb * slot,
                                   a.x + 8 * pg.unit(t.n, Gin, 2 * c + gg, t.z + zb - 1, t.y0 - 1, -1), run, &full[s]);
                } else if (lane == 6 && !b.wres) {
                    umma::bulk_g2s(st + (uint32_t)b.w_off, wpart + (size_t)c * 27 * Cp * 16, w_chunk, &full[s]);
                }
            }
        }
        if (lane == 0) {
            // no copy may still be writing shared memory when the CTA exits: wait for the
            // last kPipeStages chunks (earlier ones were consumed before their stage was reused)
            for (int kk = k > kPipeStages ? k - kPipeStages : 0; kk < k; ++kk)
                umma::mbar_wait(&full[kk % kPipeStages], (uint32_t)(kk / kPipeStages) & 1u, kWaitCycles);
            if (b.wres) umma::mbar_wait(wfull, 0u, kWaitCycles);
        }
        __syncwarp();
    } else if (warp >= kConvWorkers) {
        // two MMA threads (one thread can issue a tcgen05.mma only every ~65 cycles, two are
        // bound by the operand reads from shared memory): issuer iss takes the M tiles of its
        // parity, so each accumulator column range has one issuer
        const int iss = warp - kConvWorkers;
        if (lane == 0) {
            const uint32_t idesc = umma::idesc_bf16_f32(128, b.fold ? 3 * Cp : Cp);
            int toff[27];  // tap (dz, dy, dx) -> brick position offset (dz Yb + dy) P + dx
#pragma unroll
            for (int t = 0; t < 27; ++t) toff[t] = ((t / 9 - 1) * Yb + ((t / 3) % 3 - 1)) * P + (t % 3 - 1);
            int k = 0;
            bool ok = !b.wres || pipe_wait(wfull, 0u, abort_flag);
            for (int item = blockIdx.x, j = 0; ok && item < b.items; item += gridDim.x, ++j) {
                const int acc = j % b.nacc, v = j / b.nacc;
                if (v >= 1 && !pipe_wait(&tempty[acc], (uint32_t)(v - 1) & 1u, abort_flag)) break;
                umma::fence_after_sync();
                const uint32_t dacc = tbase + (uint32_t)(acc * acc_cols);
                for (int c = 0; c < nchunk; ++c, ++k) {
                    const int s = k % kPipeStages, u = k / kPipeStages;
                    if (!pipe_wait(&full[s], (uint32_t)u & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    umma::fence_after_sync();
                    const uint32_t st = s_stage0 + (uint32_t)(s * b.stage);
                    const uint64_t a0 = umma::smem_desc(st + 128u, (uint32_t)b.plane, 128);
                    const uint64_t b0 = umma::smem_desc(
                        b.wres ? s_wres + (uint32_t)c * w_chunk : st + (uint32_t)b.w_off, 128, 256);
                    const uint32_t a_lo = (uint32_t)a0, a_hi = (uint32_t)(a0 >> 32);
                    const uint32_t b_lo = (uint32_t)b0, b_hi = (uint32_t)(b0 >> 32);
                    const uint32_t first = c > 0 ? 1u : 0u;
                    const bool rt = b.rowtile != 0;
                    if (b.fold) {
                        switch (b.tiles) {
#define SDE_CONV_FOLD(T)                                                                             \
    case T:                                                                                          \
        if (iss) conv_chunk_mma_fold<T, 1>(dacc, a_lo, a_hi, b_lo, b_hi, idesc, Cp, toff, P, Yb, first); \
        else conv_chunk_mma_fold<T, 0>(dacc, a_lo, a_hi, b_lo, b_hi, idesc, Cp, toff, P, Yb, first); \
        break;
                            SDE_CONV_FOLD(1)
                            SDE_CONV_FOLD(2)
                            SDE_CONV_FOLD(3)
                            SDE_CONV_FOLD(4)
#undef SDE_CONV_FOLD
                            default:  // the plan keeps folded items to <= 4 tiles
                                *abort_flag = 1;
                        }
                    } else {
                        switch (b.tiles) {
#define SDE_CONV_TILES(T)                                                                          \
    case T:                                                                                        \
        if (iss) conv_chunk_mma<T, 1>(dacc, a_lo, a_hi, b_lo, b_hi, idesc, Cp, toff, rt, P, Yb, tpr, first); \
        else conv_chunk_mma<T, 0>(dacc, a_lo, a_hi, b_lo, b_hi, idesc, Cp, toff, rt, P, Yb, tpr, first); \
        break;
                            SDE_CONV_TILES(1)
                            SDE_CONV_TILES(2)
                            SDE_CONV_TILES(3)
                            SDE_CONV_TILES(4)
                            SDE_CONV_TILES(5)
                            SDE_CONV_TILES(6)
                            SDE_CONV_TILES(7)
                            SDE_CONV_TILES(8)
#undef SDE_CONV_TILES
                            default:  // the plan keeps items to <= 8 tiles
                                *abort_flag = 1;
                        }
                    }
                    umma::mma_commit(&empty[s]);
                }
                if (ok) umma::mma_commit(&tfull[acc]);
            }
        }
        __syncwarp();
    } else {
        // epilogue: thread 0 polls each barrier and the outcome is shared through a
        // named-barrier vote, so control flow stays uniform and a timeout ends all warps
        bool ok = true;
        auto worker_wait = [&](uint64_t* m, uint32_t parity) {
            bool done = true;
            if (tid == 0) done = pipe_wait(m, parity, abort_flag);
            return workers_all<kConvWorkerThreads>(done);
        };
        const int quarter = warp & 3;  // tensor-memory lanes 32 quarter .. + 31
        const int grp = warp >> 2;     // warps 0-3 take the even tiles of an item, 4-7 the odd ones
        const int Gy = a.y_cstride >> 3;
        // fold: per group two buffers (alternate tiles) of [lane quarter][Cp] column values at
        // the quarter's edges: D[x = 32 quarter + 31][co] and D[x = 32 quarter][2 Cp + co]
        float* xbuf = reinterpret_cast<float*>(smem + b.xch);
        int par = 0;
        for (int item = blockIdx.x, j = 0; ok && item < b.items; item += gridDim.x, ++j) {
            const int acc = j % b.nacc, v = j / b.nacc;
            if (!worker_wait(&tfull[acc], (uint32_t)v & 1u)) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const BrickItem t = brick_item(b, D, item);
            const int cbase = t.part * Cp;
            const uint32_t trow = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(acc * acc_cols);
            for (int m = warp >> 2; m < b.tiles; m += kConvWorkers / 4) {
                int yy, xx;
                bool valid = true;
                if (b.rowtile) {
                    yy = t.y0 + m / tpr;
                    xx = 128 * (m % tpr) + 32 * quarter + lane;
                    valid = yy < H;
                } else {
                    const int q = P + 128 * m + 32 * quarter + lane;  // position in brick plane zb = 1
                    const int yb = q / P, xp = q - yb * P;
                    yy = t.y0 + yb - 1;
                    xx = xp - 1;
                    valid = yb >= 1 && yb <= b.Ty && xp >= 1 && xp <= W && yy < H;
                }
                // fold: out[x] = D[x-1][co] + D[x][Cp + co] + D[x+1][2 Cp + co]; x - 1 and x + 1 of the
                // quarter's edge lanes belong to the neighbouring quarter (another warp of the group),
                // x = -1 and x = 128 are padding (their D is zero).  Columns move 16 at a time, all
                // loads of a chunk in flight before one wait.
                const uint32_t tcol = trow + (uint32_t)(m * Cp * (b.fold ? 3 : 1));
                float* xlo = xbuf + (size_t)((grp * 2 + par) * 2) * 4 * Cp;
                float* xhi = xlo + 4 * Cp;
                for (int c = 0; c < Cp; c += 16) {
                    uint32_t v[16];
                    __syncwarp();
                    if (b.fold) {
                        uint32_t lo[16], hi[16];
                        umma::tmem_ld16_nowait(tcol + (uint32_t)c, lo);
                        umma::tmem_ld16_nowait(tcol + (uint32_t)(Cp + c), v);
                        umma::tmem_ld16_nowait(tcol + (uint32_t)(2 * Cp + c), hi);
                        umma::tmem_wait_ld16(lo);
                        umma::tmem_touch16(v);
                        umma::tmem_touch16(hi);
                        // edge lanes publish their 16 values with four 16-byte stores
                        if (lane == 31 || lane == 0) {
                            uint4* dst = reinterpret_cast<uint4*>((lane == 31 ? xlo : xhi) + quarter * Cp + c);
                            const uint32_t* src = lane == 31 ? lo : hi;
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4)
                                dst[q4] = make_uint4(src[4 * q4], src[4 * q4 + 1], src[4 * q4 + 2], src[4 * q4 + 3]);
                        }
                        uint32_t l[16], r[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            l[e] = __shfl_up_sync(0xffffffffu, lo[e], 1);
                            r[e] = __shfl_down_sync(0xffffffffu, hi[e], 1);
                        }
                        group_sync(2 + grp);
                        if (lane == 0 || lane == 31) {
                            const bool left = lane == 0;
                            const bool edge = left ? quarter == 0 : quarter == 3;  // padding column
                            const int nq = left ? (quarter > 0 ? quarter - 1 : 0) : (quarter < 3 ? quarter + 1 : 3);
                            const uint4* src = reinterpret_cast<const uint4*>((left ? xlo : xhi) + nq * Cp + c);
                            uint32_t* dst = left ? l : r;
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const uint4 w = edge ? make_uint4(0u, 0u, 0u, 0u) : src[q4];
                                dst[4 * q4] = w.x;
                                dst[4 * q4 + 1] = w.y;
                                dst[4 * q4 + 2] = w.z;
                                dst[4 * q4 + 3] = w.w;
                            }
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            v[e] = __float_as_uint(__uint_as_float(v[e]) + (__uint_as_float(l[e]) + __uint_as_float(r[e])));
                    } else {
                        umma::tmem_ld16_nowait(tcol + (uint32_t)c, v);
                        umma::tmem_wait_ld16(v);
                    }
                    if (valid) {
                        float rr[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) rr[e] = __uint_as_float(v[e]);
                        if (a.bias) {
                            const float4* bq = reinterpret_cast<const float4*>(a.bias + cbase + c);
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const float4 bb = __ldg(bq + q4);
                                rr[4 * q4] += bb.x;
                                rr[4 * q4 + 1] += bb.y;
                                rr[4 * q4 + 2] += bb.z;
                                rr[4 * q4 + 3] += bb.w;
                            }
                        }
                        if (a.relu)
#pragma unroll
                            for (int e = 0; e < 16; ++e) rr[e] = rr[e] > 0.f ? rr[e] : a.slope * rr[e];
                        if (a.y_fp32) {
                            const size_t vox = (size_t)t.n * a.nvox + ((size_t)t.z * H + yy) * W + xx;
                            if (a.y_keep) {  // leading channels only (the first chunk of part 0)
                                if (cbase + c == 0)
#pragma unroll
                                    for (int e = 0; e < 16; ++e)  // constant indices keep rr in registers
                                        if (e < a.y_keep) static_cast<float*>(a.y)[vox * a.y_keep + e] = rr[e];
                            } else {
                                float4* yo = reinterpret_cast<float4*>(static_cast<float*>(a.y) + vox * a.y_cstride +
                                                                       a.y_coffset + cbase + c);
                                for (int q4 = 0; q4 < 4; ++q4)
                                    yo[q4] = make_float4(rr[4 * q4], rr[4 * q4 + 1], rr[4 * q4 + 2], rr[4 * q4 + 3]);
                            }
                        } else {
                            for (int h = 0; h < 2; ++h) {
                                __nv_bfloat162 pk[4];
                                for (int e = 0; e < 4; ++e)
                                    pk[e] = __floats2bfloat162_rn(rr[8 * h + 2 * e], rr[8 * h + 2 * e + 1]);
                                const int gy = (a.y_coffset + cbase + c + 8 * h) >> 3;
                                __nv_bfloat16* yo =
                                    static_cast<__nv_bfloat16*>(a.y) + 8 * pg.unit(t.n, Gy, gy, t.z, yy, xx);
                                const uint4 val = *reinterpret_cast<uint4*>(pk);
                                *reinterpret_cast<uint4*>(yo) = val;
                                if (a.y_up) {  // the eight children on the doubled grid
                                    const Pcg pf{2 * D, 2 * H, 2 * W};
                                    const int gu = (a.y_up_coffset + cbase + c + 8 * h) >> 3;
                                    __nv_bfloat16* yu = static_cast<__nv_bfloat16*>(a.y_up);
#pragma unroll
                                    for (int d = 0; d < 8; ++d)
                                        *reinterpret_cast<uint4*>(
                                            yu + 8 * pf.unit(t.n, a.y_up_cstride >> 3, gu, 2 * t.z + (d >> 2),
                                                             2 * yy + ((d >> 1) & 1), 2 * xx + (d & 1))) = val;
                                }
                            }
                        }
                    }
                }
                par ^= 1;
            }
            umma::fence_before_sync();
            umma::mbar_arrive(&tempty[acc]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (tid == 0 && *abort_flag) atomicOr(a.status, 1u);
    if (warp == 0) umma::tmem_dealloc(tbase, (uint32_t)b.tcols);
}

// ----------------------------------------------------------------------------
// Brick weight gradient: dW[co][tap][ci] = sum over output positions v of
// dy[v][co] x[v + off(tap)][ci].  Per work item (Ty output rows of one z plane) the
// output-gradient rows and the zero-padded input brick are staged once, both as 8-channel
// planes with 16 bytes per position, i.e. M/N-major core matrices (8 positions x 8
// channels); both tensors are padded channel-group-major, so each 8-channel plane of the
// rows, and each (8-channel plane, z plane) part of the brick, is one bulk copy.  The MMA's A operand is dy (M = co, padded to 128: rows past Cout read
// whatever follows and are never stored), K = 16 positions; B is the brick read from the
// tap's offset (N = Nc input channels).  All taps of the pass use the same A, so the
// tensor core fetches it once per K step.  dW accumulates in tensor memory over all the
// CTA's items and is added to global memory once, at the end.  Padding positions of dy
// are zero, so brick positions under them contribute nothing -- provided they hold no
// NaN or Inf: the few positions B reads just outside the staged data (before the first
// plane, between planes, after the last) are zeroed once at start and never written.
// ----------------------------------------------------------------------------
// The weight-gradient MMAs of one K step for taps T0 .. T1-1 (fully unrolled) of a pass
// whose first tap is P0: the accumulator of tap t starts at column (t - P0) Nc, B's start
// field is the K step's plus the tap's brick offset.
template <int P0, int T0, int T1>
__device__ __forceinline__ void wgrad_taps(uint32_t tbase, int Nc, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo,
                                           uint32_t b_hi, uint32_t idesc, uint32_t accum, const int (&toff)[27]) {
#pragma unroll
    for (int t = T0; t < T1; ++t)
        umma::mma_bf16_lohi(tbase + (uint32_t)((t - P0) * Nc), a_lo, a_hi, b_lo + (uint32_t)toff[t], b_hi, idesc,
                            accum);
}

__global__ void __launch_bounds__(192, 1) k_wgrad_brick(WgradArgs a, WgradPlan b) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Cin = a.Cin, Cout = a.Cout, W = a.W, H = a.H, D = a.D, Nc = b.Nc;
    const int P = b.P, Yb = b.Yb;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [kPipeStages]
    uint64_t* empty = full + kPipeStages;                 // [kPipeStages]
    uint64_t* dfull = empty + kPipeStages;                // all MMAs of the CTA done
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 128);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 132);
    const uint32_t s_stage0 = umma::smem_addr(smem) + kPipeHeader;
    const int pass = blockIdx.y;
    const int c = pass / b.ngroups;  // input-channel chunk
    const int t0 = (pass % b.ngroups) * b.ntap;
    const int t1 = t0 + b.ntap < 27 ? t0 + b.ntap : 27;
    const int my_items =
        b.items > (int)blockIdx.x ? (b.items - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    {  // zero both stages: gaps around the staged data must read as 0, not leftover bits
        uint4* z = reinterpret_cast<uint4*>(smem + kPipeHeader);
        const int n16 = kPipeStages * b.stage / 16;
        for (int i = tid; i < n16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        umma::fence_async_smem();  // generic-proxy stores -> tensor-core reads
    }
    if (warp == 0) {
        umma::tmem_alloc(slot, 512u);
        umma::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kPipeStages; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 2);  // one commit per MMA thread
        }
        umma::mbar_init(dfull, 2);
        *abort_flag = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *slot;
    const int fB = (Yb + 1) * P;  // brick position under output position 0 of the item

    if (warp >= 4) {
        // two MMA threads split each pass's taps (each tap has its own accumulator columns)
        const int iss = warp - 4;
        if (lane == 0) {
            const uint32_t idesc = umma::idesc_bf16_f32(128, Nc, 1, 1);
            int toff[27];  // tap (dz, dy, dx) -> brick position offset (dz Yb + dy) P + dx
#pragma unroll
            for (int t = 0; t < 27; ++t) toff[t] = ((t / 9 - 1) * Yb + ((t / 3) % 3 - 1)) * P + (t % 3 - 1);
            bool ok = true;
            for (int j = 0; j < my_items && ok; ++j) {
                const int s = j % kPipeStages, u = j / kPipeStages;
                if (!pipe_wait(&full[s], (uint32_t)u & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t st = s_stage0 + (uint32_t)(s * b.stage);
                // M/N-major: leading byte offset = next 8 positions (K), stride = next 8 channels
                const uint64_t a0 = umma::smem_desc(st, 128, (uint32_t)b.plane_dy);
                const uint64_t b0 = umma::smem_desc(st + (uint32_t)b.x_off, 128, (uint32_t)b.plane_x);
                const uint32_t a_hi = (uint32_t)(a0 >> 32), b_hi = (uint32_t)(b0 >> 32);
                for (int ks = 0; ks < b.kst; ++ks) {
                    const uint32_t a_lo = (uint32_t)a0 + (uint32_t)(16 * ks);  // 16 positions of 16 bytes
                    const uint32_t b_lo = (uint32_t)b0 + (uint32_t)(fB + 16 * ks);
                    // each tap's accumulator starts at its first MMA: item 0, K step 0
                    const uint32_t accum = (j > 0 || ks > 0) ? 1u : 0u;
                        // unrolled over this pass's taps: one add per instruction; fB + offset >= -1,
                    // one position before the brick at most (dy is zero there), so the start
                    // field never borrows
                    if (t0 == 0 && t1 == 27) {
                        if (iss) wgrad_taps<0, 14, 27>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                        else wgrad_taps<0, 0, 14>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                    } else if (t0 == 0 && t1 == 14) {
                        if (iss) wgrad_taps<0, 7, 14>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                        else wgrad_taps<0, 0, 7>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                    } else if (t0 == 14 && t1 == 27) {
                        if (iss) wgrad_taps<14, 21, 27>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                        else wgrad_taps<14, 14, 21>(tbase, Nc, a_lo, a_hi, b_lo, b_hi, idesc, accum, toff);
                    } else
                        for (int t = t0 + iss; t < t1; t += 2)
                            umma::mma_bf16_lohi(tbase + (uint32_t)((t - t0) * Nc), a_lo, a_hi,
                                                b_lo + (uint32_t)(((t / 9 - 1) * Yb + ((t / 3) % 3 - 1)) * P +
                                                                  (t % 3 - 1)),
                                                b_hi, idesc, accum);
                }
                umma::mma_commit(&empty[s]);
            }
            if (ok) umma::mma_commit(dfull);
        }
        __syncwarp();
    } else {
        bool ok = true;
        auto worker_wait = [&](uint64_t* m, uint32_t parity) {
            bool done = true;
            if (tid == 0) done = pipe_wait(m, parity, abort_flag);
            return workers_all<128>(done);
        };
        if (tid == 0) {  // producer: per item Cout/8 runs of dy rows and Nc/8 x 3 runs of the input brick
            const Pcg pg{D, H, W};
            const uint32_t run_dy = (uint32_t)(b.Ty * P * 16), run_x = (uint32_t)(Yb * P * 16);
            const int gdy = Cout >> 3, gx = Nc >> 3;
            int j = 0;
            for (; j < my_items; ++j) {
                const int s = j % kPipeStages, u = j / kPipeStages;
                if (u >= 1 && !pipe_wait(&empty[s], (uint32_t)(u - 1) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                int r = (int)blockIdx.x + j * (int)gridDim.x;
                const int z = r % D;
                r /= D;
                const int y0 = (r % b.nyb) * b.Ty;
                const int n = r / b.nyb;
                const uint32_t st = s_stage0 + (uint32_t)(s * b.stage);
                umma::mbar_arrive_expect_tx(&full[s], (uint32_t)gdy * run_dy + (uint32_t)(3 * gx) * run_x);
                // output-gradient rows y0 .. y0+Ty-1 with their zero padding columns; the
                // positions up to kst*16 past them stay zero from the start
                for (int q = 0; q < gdy; ++q)
                    umma::bulk_g2s(st + (uint32_t)(q * b.plane_dy), a.dy + 8 * pg.unit(n, gdy, q, z, y0, -1), run_dy,
                                   &full[s]);
                for (int g = 0; g < gx; ++g)
                    for (int zb = 0; zb < 3; ++zb)
                        umma::bulk_g2s(st + (uint32_t)(b.x_off + g * b.plane_x) + (uint32_t)zb * run_x,
                                       a.x + 8 * pg.unit(n, Cin >> 3, c * gx + g, z + zb - 1, y0 - 1, -1), run_x,
                                       &full[s]);
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int jj = j > kPipeStages ? j - kPipeStages : 0; jj < j; ++jj)
                umma::mbar_wait(&full[jj % kPipeStages], (uint32_t)(jj / kPipeStages) & 1u, kWaitCycles);
        }
        ok = workers_all<128>(ok);
        if (ok && my_items > 0 && worker_wait(dfull, 0u)) {
            umma::fence_after_sync();
            const int co = 32 * warp + lane;
            if (32 * warp < Cout) {  // warp-uniform: lanes past Cout load but do not store
                for (int t = t0; t < t1; ++t)
                    for (int cc = 0; cc < Nc; cc += 8) {
                        float v[8];
                        __syncwarp();
                        umma::tmem_ld8(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)((t - t0) * Nc + cc), v);
                        if (co < Cout)
                            for (int e = 0; e < 8; ++e)
                                atomicAdd(&a.dw[((size_t)co * 27 + t) * Cin + c * Nc + cc + e], v[e]);
                    }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (tid == 0 && *abort_flag) atomicOr(a.status, 1u);
    if (warp == 0) umma::tmem_dealloc(tbase, 512u);
}

// wd[ci][26 - tap][co] = w[co][tap][ci]: the data gradient of a 3x3x3 convolution is
// the convolution of dy with these weights.
__global__ void k_flip_weights(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout) {
    const int n = Cout * 27 * Cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, tap = (i / Cin) % 27, co = i / (27 * Cin);
        wd[((size_t)ci * 27 + (26 - tap)) * Cout + co] = w[i];
    }
}

}  // namespace

cudaError_t flip_weights_launch(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout, cudaStream_t st) {
    k_flip_weights<<<256, 256, 0, st>>>(w, wd, Cin, Cout);
    return cudaGetLastError();
}

// Work decomposition of the pipelined brick kernel for one layer shape: output channels
// split into parts of Cp, weights resident or streamed, rows per item Ty (the last row block
// may pass H),
// and for 128-voxel rows the x-tap fold, chosen by a cost model calibrated on GB300 with
// per-role cycle counters in this kernel: a tcgen05.mma (M = 128, K = 16) takes ~64 cycles
// of one issuing thread at N = 32, ~85 at N = 64, ~90 at N = 96 and about N / 2 from
// N = 192, less with two issuers (mma_pair_factor); bulk copies of brick runs move ~64 bytes per cycle per SM; the epilogue takes
// ~700 cycles per tile and 8 columns (~850 folded) on each of its two warp groups and
// overlaps the MMAs only with two accumulators; copies and MMAs overlap, but not perfectly
// (a quarter of the shorter one shows).
static double mma_cycles(int N) {
    return N <= 32 ? 64.0 : (N <= 64 ? 85.0 : (N <= 96 ? 90.0 : (N <= 192 ? 96.0 + (N - 128) / 2.0 : N / 2.0)));
}
// Time per MMA with two issuers relative to one (microbenchmark: 65 cycles from one thread,
// (4 KB of A + N x 32 bytes of B) / 128 bytes per cycle from two, at least the dense peak).
static double mma_pair_factor(int N) {
    const double two = (4096.0 + 32.0 * N) / 128.0, peak = 2.0 * 128 * N * 16 / 8192.0;
    return (two > peak ? two : peak) / 65.0 < 1.0 ? (two > peak ? two : peak) / 65.0 : 1.0;
}

static bool brick_plan(int D, int H, int W, int Cin, int Cout, int batch, BrickPlan* out, size_t* smem_out) {
    const int P = W + 2;
    const size_t smem_cap = 227 * 1024;
    const bool rowtile = W % 128 == 0;
    double best = 1e300;
    bool found = false;
    const int nchunk = Cin / 16;
    for (int nsplit = 1; nsplit <= Cout / 16; ++nsplit) {
        if (Cout % nsplit || (Cout / nsplit) % 16) continue;
        const int Cp = Cout / nsplit;
        if (Cp > 256) continue;
        const size_t w_bytes = (size_t)27 * Cp * 32;
        for (int fold = 0; fold <= (W == 128 && 3 * Cp <= 256 ? 1 : 0); ++fold)
            for (int wres = nsplit == 1 ? 1 : 0; wres >= 0; --wres)  // ties keep the weights resident
                for (int Ty = 1; Ty <= H; ++Ty) {
                    const int nyb = (H + Ty - 1) / Ty;
                    const int tiles = rowtile ? Ty * (W / 128) : (Ty * P + 127) / 128;
                    const int cols = tiles * Cp * (fold ? 3 : 1);  // accumulator columns per item
                    if (cols > 512 || tiles > (fold ? 4 : 8)) break;  // the MMA loops are unrolled up to these
                    const int nacc = 2 * cols <= 512 ? 2 : 1;
                    const size_t run = (size_t)(Ty + 2) * P * 16;
                    const size_t plane = (3 * run + 127) / 128 * 128;
                    // flat tiles read up to 128 positions past the end of the second plane
                    const size_t w_off = (128 + 2 * plane + (rowtile ? 0 : 2048) + 127) / 128 * 128;
                    const size_t stage = wres ? w_off : (w_off + w_bytes + 127) / 128 * 128;
                    const size_t xch = kPipeHeader + kPipeStages * stage + (wres ? nchunk * w_bytes : 0);
                    const size_t smem = xch + (fold ? (size_t)128 * Cp : 0);
                    if (smem > smem_cap || plane >= (1u << 18)) break;
                    // two issuers share the tiles: pairs of tiles at the two-issuer rate, an odd
                    // last tile at one issuer's
                    const int Nmma = fold ? 3 * Cp : Cp;
                    const double per_tile = (fold ? 9 : 27) * mma_cycles(Nmma);
                    const double mma = (double)nchunk * per_tile * ((tiles / 2) * 2 * mma_pair_factor(Nmma) + tiles % 2);
                    const double load = (double)nchunk * (6 * run + (wres ? 0 : w_bytes)) / 64.0;
                    const double epi = ((tiles + 1) / 2) * (Cp / 8.0) * (fold ? 850.0 : 700.0);
                    double item = (mma > load ? mma : load) + 0.25 * (mma > load ? load : mma);
                    item = nacc == 2 ? (item > epi ? item : epi) : item + epi;
                    const double cost = item * nyb / ((double)H * W) * nsplit;  // per output voxel, all parts
                    if (cost < best) {
                        best = cost;
                        found = true;
                        int tcols = 32;
                        while (tcols < nacc * cols) tcols <<= 1;
                        BrickPlan bp{};
                        bp.Ty = Ty;
                        bp.tiles = tiles;
                        bp.rowtile = rowtile ? 1 : 0;
                        bp.fold = fold;
                        bp.nyb = nyb;
                        bp.P = P;
                        bp.Yb = Ty + 2;
                        bp.Cp = Cp;
                        bp.nsplit = nsplit;
                        bp.plane = (int)plane;
                        bp.w_off = (int)w_off;
                        bp.wres = wres;
                        bp.stage = (int)stage;
                        bp.nacc = nacc;
                        bp.xch = (int)xch;
                        bp.tcols = tcols;
                        bp.items = batch * nsplit * nyb * D;
                        *out = bp;
                        *smem_out = smem;
                    }
                }
    }
    return found;
}

// wpk[part][chunk][tap][core-matrix image of the Cp x 16 tile] = w[part Cp + r][tap][16 chunk + k]
static __global__ void k_pack_weights(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wpk, int Cin,
                               int Cout, int Cp) {
    const int n = Cout * 27 * Cin, nchunk = Cin >> 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, tap = (i / Cin) % 27, co = i / (27 * Cin);
        const int part = co / Cp, r = co - part * Cp, c = ci >> 4, k = ci & 15;
        const size_t tile = (((size_t)part * nchunk + c) * 27 + tap) * Cp * 16;
        wpk[tile + umma::core_offset(r, k, 16) / 2] = w[i];
    }
}

int conv_plan_cp(int D, int H, int W, int Cin, int Cout) {
    BrickPlan bp{};
    size_t smem = 0;
    return brick_plan(D, H, W, Cin, Cout, 1, &bp, &smem) ? bp.Cp : 0;
}

cudaError_t conv_pack_weights(const __nv_bfloat16* w, __nv_bfloat16* wpk, int Cin, int Cout, int Cp,
                              cudaStream_t st) {
    if (Cp <= 0 || Cout % Cp || Cin % 16) return cudaErrorInvalidValue;
    k_pack_weights<<<256, 256, 0, st>>>(w, wpk, Cin, Cout, Cp);
    return cudaGetLastError();
}

cudaError_t conv3d_launch(const ConvArgs& a, int batch, cudaStream_t st) {
    BrickPlan bp{};
    size_t bsmem = 0;
    if (!brick_plan(a.D, a.H, a.W, a.Cin, a.Cout, batch, &bp, &bsmem) || bp.Cp != a.wpk_cp)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int ctas = bp.items < sms ? bp.items : sms;
    k_conv3d_brick<<<ctas, kConvThreads, bsmem, st>>>(a, bp);
    return cudaGetLastError();
}

// Plan of the brick weight gradient: Nc in {16, 32} input channels per pass, as many
// taps per pass as 512 tensor-memory columns hold, and Ty a divisor of H whose two stages
// fit; the cost model (~56 cycles per MMA; bulk copies ~64 bytes per cycle per SM) picks
// among them.  Measured alternative, slower on the denoiser's
// layers: one input plane per pass with the nine taps of one dz (more rows per item).
static bool wgrad_plan(const WgradArgs& a, int sms, WgradPlan* out, size_t* smem_out) {
    const int P = a.W + 2;
    double best = 1e300;
    bool found = false;
    for (int Nc = 16; Nc <= 32; Nc += 16) {
        if (a.Cin % Nc) continue;
        const int ntap = Nc == 16 ? 27 : 14;
        const int ngroups = (27 + ntap - 1) / ntap;
        for (int Ty = 1; Ty <= a.H; ++Ty) {
            if (a.H % Ty) continue;
            const int kst = (Ty * P + 15) / 16;
            const size_t plane_dy = (size_t)kst * 256;
            const size_t dy_bytes = (size_t)(a.Cout / 8) * plane_dy;
            const size_t plane_x = ((size_t)3 * (Ty + 2) * P * 16 + 127) / 128 * 128;
            const size_t x_off = (dy_bytes + 16 + 127) / 128 * 128;  // >= 16 bytes before the brick
            size_t stage = (x_off + (size_t)(Nc / 8) * plane_x + 512 + 127) / 128 * 128;
            if (stage < 16 * plane_dy) stage = (16 * plane_dy + 127) / 128 * 128;  // A rows past Cout stay inside
            const size_t smem = kPipeHeader + kPipeStages * stage;
            if (smem > 227 * 1024 || plane_x >= (1u << 18) || plane_dy >= (1u << 18)) break;
            const double pos = (double)Ty * a.W;  // output voxels per item
            const double mma = (double)kst * 27 * 56.0 * (a.Cin / Nc);
            const double bytes = (double)(a.Cout / 8) * Ty * P * 16 + (double)(Nc / 8) * 3 * (Ty + 2) * P * 16;
            const double load = bytes / 64.0 * (a.Cin / Nc) * ngroups;
            const double cost = (mma > load ? mma : load) / pos;
            if (cost < best) {
                best = cost;
                found = true;
                const int nyb = a.H / Ty;
                const int items = a.batch * nyb * a.D;
                const int passes = (a.Cin / Nc) * ngroups;
                // CTAs per pass: all passes in one wave on the SMs (a CTA past it would run its
                // whole share again after the others)
                int G = sms / passes > 1 ? sms / passes : 1;
                if (G > items) G = items;
                *out = WgradPlan{Ty, nyb, P, Ty + 2, Nc, ntap, ngroups, kst, (int)plane_dy, (int)plane_x,
                                 (int)x_off, (int)stage, items, G};
                *smem_out = smem;
            }
        }
    }
    return found;
}

cudaError_t wgrad_launch(const WgradArgs& a, cudaStream_t st) {
    WgradPlan wp{};
    size_t wsmem = 0;
    int dev = 0, sms = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    if (!wgrad_plan(a, sms, &wp, &wsmem)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)wp.G, (unsigned)((a.Cin / wp.Nc) * wp.ngroups));
    k_wgrad_brick<<<grid, 192, wsmem, st>>>(a, wp);
    return cudaGetLastError();
}

}  // namespace sde

static bool conv_shape_ok(int D, int H, int W, int Cin, int Cout, int batch) {
    const long long vp = (long long)(D + 2) * (H + 2) * (W + 2);
    return batch >= 1 && D >= 1 && H >= 1 && W >= 1 && W <= 256 && vp * batch * 256 < (1ll << 40) && Cin >= 16 &&
           Cin <= 192 && Cin % 16 == 0 && Cout >= 16 && Cout <= 256 && Cout % 16 == 0;
}

extern "C" int sde_conv3d_forward(const void* d_x, int batch, int D, int H, int W, int Cin, const void* d_w,
                                  const float* d_bias, int Cout, void* d_y, int y_cstride, int y_coffset,
                                  int y_fp32, int relu, void* stream) {
    if (!d_x || !d_w || !d_y || !conv_shape_ok(D, H, W, Cin, Cout, batch) || y_cstride < Cout + y_coffset ||
        y_coffset < 0 || (y_coffset % 8) || (y_cstride % 8) ||
        (((uintptr_t)d_x | (uintptr_t)d_y | (uintptr_t)d_bias) & 15)) {
        set_last_error("sde_conv3d_forward: need W <= 256, Cin in 16..192 and Cout in 16..256 (multiples of 16), "
                       "y_cstride >= Cout + y_coffset, both multiples of 8, 16-byte aligned x, y and bias");
        return SDE_EINVAL;
    }
    unsigned int* d_status = nullptr;
    int rc = report(status_word(&d_status), "status word");
    if (rc) return rc;
    const int Cp = conv_plan_cp(D, H, W, Cin, Cout);
    if (!Cp) {
        set_last_error("sde_conv3d_forward: no tile plan fits shared memory for this shape");
        return SDE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    __nv_bfloat16* wpk = nullptr;  // weights in the tensor core's layout, stream-ordered scratch
    rc = report(cudaMallocAsync(reinterpret_cast<void**>(&wpk), (size_t)Cout * 27 * Cin * 2, st), "cudaMallocAsync");
    if (rc) return rc;
    rc = report(conv_pack_weights(static_cast<const __nv_bfloat16*>(d_w), wpk, Cin, Cout, Cp, st), "pack weights");
    ConvArgs a;
    a.x = static_cast<const __nv_bfloat16*>(d_x);
    a.wpk = wpk;
    a.wpk_cp = Cp;
    a.bias = d_bias;
    a.y = d_y;
    a.D = D;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.nvox = D * H * W;
    a.y_cstride = y_cstride;
    a.y_coffset = y_coffset;
    a.y_fp32 = y_fp32;
    a.y_keep = 0;
    a.y_up = nullptr;
    a.y_up_cstride = a.y_up_coffset = 0;
    a.relu = relu;
    a.slope = 0.f;
    a.status = d_status;
    if (!rc) rc = report(conv3d_launch(a, batch, st), "conv3d launch");
    const int rf = report(cudaFreeAsync(wpk, st), "cudaFreeAsync");
    return rc ? rc : rf;
}

extern "C" int sde_conv3d_wgrad(const void* d_x, const void* d_dy, float* d_dw, int batch, int D, int H, int W,
                                int Cin, int Cout, void* stream) {
    if (!d_x || !d_dy || !d_dw || !conv_shape_ok(D, H, W, Cin, Cout, batch) || Cout > 128 ||
        (((uintptr_t)d_x | (uintptr_t)d_dy) & 15)) {
        set_last_error("sde_conv3d_wgrad: need W <= 256, Cin in 16..192, Cout in 16..128 (multiples of 16), "
                       "16-byte aligned x and dy");
        return SDE_EINVAL;
    }
    unsigned int* d_status = nullptr;
    int rc = report(status_word(&d_status), "status word");
    if (rc) return rc;
    WgradArgs a;
    a.x = static_cast<const __nv_bfloat16*>(d_x);
    a.dy = static_cast<const __nv_bfloat16*>(d_dy);
    a.dw = d_dw;
    a.D = D;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.nvox = D * H * W;
    a.batch = batch;
    a.status = d_status;
    return report(wgrad_launch(a, (cudaStream_t)stream), "wgrad launch");
}

extern "C" int sde_conv3d_flip_weights(const void* d_w, void* d_wd, int Cin, int Cout, void* stream) {
    if (!d_w || !d_wd || Cin < 1 || Cout < 1) {
        set_last_error("sde_conv3d_flip_weights: bad arguments");
        return SDE_EINVAL;
    }
    k_flip_weights<<<256, 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16*>(d_w),
                                                            static_cast<__nv_bfloat16*>(d_wd), Cin, Cout);
    return report(cudaGetLastError(), "k_flip_weights launch");
}

extern "C" int sde_denoise_status(void* stream) { return denoise_check_status((cudaStream_t)stream); }

// Host-only views of the two plans (no CUDA call).
extern "C" int sde_conv3d_plan(int batch, int D, int H, int W, int Cin, int Cout, int32_t* fields, int n_fields,
                               uint64_t* smem_bytes) {
    BrickPlan bp{};
    size_t smem = 0;
    if (!conv_shape_ok(D, H, W, Cin, Cout, batch) || n_fields < 0 || (n_fields > 0 && !fields) ||
        !brick_plan(D, H, W, Cin, Cout, batch, &bp, &smem)) {
        set_last_error("sde_conv3d_plan: shape rejected by the convolution or without a plan");
        return SDE_EINVAL;
    }
    const int32_t v[17] = {bp.Ty,    bp.tiles, bp.rowtile, bp.fold,  bp.nyb, bp.P,    bp.Yb,  bp.Cp,   bp.nsplit,
                           bp.plane, bp.w_off, bp.wres,    bp.stage, bp.nacc, bp.xch, bp.tcols, bp.items};
    for (int i = 0; i < n_fields && i < 17; ++i) fields[i] = v[i];
    if (smem_bytes) *smem_bytes = smem;
    return SDE_OK;
}

extern "C" int sde_conv3d_wgrad_plan(int batch, int D, int H, int W, int Cin, int Cout, int sms, int32_t* fields,
                                     int n_fields, uint64_t* smem_bytes) {
    WgradArgs a{};
    a.D = D;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.nvox = D * H * W;
    a.batch = batch;
    WgradPlan wp{};
    size_t smem = 0;
    if (!conv_shape_ok(D, H, W, Cin, Cout, batch) || Cout > 128 || sms < 1 || n_fields < 0 ||
        (n_fields > 0 && !fields) || !wgrad_plan(a, sms, &wp, &smem)) {
        set_last_error("sde_conv3d_wgrad_plan: shape rejected by the weight gradient or without a plan");
        return SDE_EINVAL;
    }
    const int32_t v[14] = {wp.Ty,       wp.nyb,     wp.P,     wp.Yb,    wp.Nc,    wp.ntap,  wp.ngroups,
                           wp.kst,      wp.plane_dy, wp.plane_x, wp.x_off, wp.stage, wp.items, wp.G};
    for (int i = 0; i < n_fields && i < 14; ++i) fields[i] = v[i];
    if (smem_bytes) *smem_bytes = smem;
    return SDE_OK;
}
