// sde_denoiser.cu -- native runtime of the learned dose denoiser: a 3-level 3D
// convolutional encoder-decoder (32/64/128 channels, 3x3x3 kernels, BF16
// activations and weights, FP32 accumulation) that maps a low-history SDE dose
// and the density map to the high-history dose, with its forward pass, hand-derived
// backward pass and Adam optimiser, plus a GPU 3D gamma index for its evaluation.
//
// Network (per sample, channels-last):
//   in0  = [dose_low * s, density / 2, 0...]            16 ch   (s = 1 / max dose_low)
//   (relu = leaky ReLU, slope 0.1)
//   e1a  = relu(conv(in0))  32;  e1 = relu(conv(e1a)) 32    -> cat1[..., 64:96]
//   p1   = avgpool2(e1)     32
//   e2a  = relu(conv(p1))   64;  e2 = relu(conv(e2a)) 64    -> cat2[..., 128:192]
//   p2   = avgpool2(e2)     64
//   b1   = relu(conv(p2))  128;  b2 = relu(conv(b1)) 128
//   cat2[..., 0:128] = up2(b2);  d2a = relu(conv(cat2)) 64;  d2 = relu(conv(d2a)) 64
//   cat1[..., 0:64]  = up2(d2);  d1a = relu(conv(cat1)) 32;  d1 = relu(conv(d1a)) 32
//   out  = conv(d1) (FP32, channel 0 used);  prediction = dose_low * s + out[0]
// Loss: squared error of the prediction against dose_high * s, weighted by
// 1/(dose_high * s + 0.05) (relative error, as the local-normalisation gamma sees it).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "sde_denoise.h"
#include "sde_dose.h"
#include "sde_tables.h"

namespace sde {
namespace {

using bf16 = __nv_bfloat16;

constexpr float kLossKappa = 0.05f;  // relative-error weighting floor (fraction of the max dose)
constexpr float kLeak = 0.1f;        // leaky ReLU slope (plain ReLU units died in training)

// -------------------------------------------------------------- small kernels
__global__ void k_absmax(const float* __restrict__ x, size_t n_per, int batch, unsigned int* out_bits) {
    for (int b = 0; b < batch; ++b) {
        float m = 0.f;
        const float* xb = x + (size_t)b * n_per;
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_per; i += (size_t)gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf(xb[i]));
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
        if ((threadIdx.x & 31) == 0) atomicMax(&out_bits[b], __float_as_uint(m));
    }
}

__device__ __forceinline__ float scale_of(const unsigned int* maxbits, int b) {
    float m = __uint_as_float(maxbits[b]);
    return m > 0.f ? 1.f / m : 1.f;
}

// Input channels (padded channel-group-major, two groups): group 0 of voxel v of sample b
// holds (dose * s_b, density / 2, 0, ...); group 1 stays zero.
__global__ void k_prepare_input(const float* __restrict__ dose, const float* __restrict__ rho, Pcg g, int batch,
                                const unsigned int* maxbits, bf16* __restrict__ in0) {
    const size_t V = (size_t)g.D * g.H * g.W, n = V * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / V);
        const int v = (int)(i - (size_t)b * V);
        const int x = v % g.W, y = (v / g.W) % g.H, z = v / (g.W * g.H);
        __nv_bfloat162 p[4];
        p[0] = __floats2bfloat162_rn(dose[i] * scale_of(maxbits, b), 0.5f * rho[v]);
        for (int j = 1; j < 4; ++j) p[j] = __floats2bfloat162_rn(0.f, 0.f);
        *reinterpret_cast<uint4*>(in0 + 8 * g.unit(b, 2, 0, z, y, x)) = *reinterpret_cast<uint4*>(p);
    }
}

__device__ __forceinline__ void ld8(const bf16* p, float (&f)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ void st8(bf16* p, const float (&f)[8]) {
    __nv_bfloat162 h[4];
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(h);
}

// Two resolutions: the fine grid F (D, H, W even) and the coarse grid C = F / 2.  The
// resampling kernels run one thread per (coarse voxel, 8-channel group) on the launch grid
// (ceil(Wc G / 256), Hc, Dc batch) with 256 threads, x fastest across threads, and move 16
// bytes per access: a warp reads 32 consecutive coarse voxels of one group (512 contiguous
// bytes) and writes or reads their fine children as 32-byte pairs along x (1 KB contiguous
// per (dz, dy)).  Channel counts, strides and offsets are multiples of 8 (offsets and
// strides below are in channels).
struct Grid2 {
    Pcg F, C;
};
__host__ __device__ inline Grid2 grid2(int D, int H, int W) { return Grid2{Pcg{D, H, W}, Pcg{D / 2, H / 2, W / 2}}; }

struct CoarseIdx {
    int q, xc, yc, zc, b;
};
__device__ __forceinline__ bool coarse_idx(const Grid2& g, int G, CoarseIdx& c) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.C.W * G) return false;
    c.q = t / g.C.W;
    c.xc = t - c.q * g.C.W;
    c.yc = blockIdx.y;
    c.zc = blockIdx.z % g.C.D;
    c.b = blockIdx.z / g.C.D;
    return true;
}
// 16-byte unit of fine child d = (dz, dy, dx) bits (4, 2, 1) of coarse voxel c, group gq of Gt
__device__ __forceinline__ size_t fine_unit(const Grid2& g, const CoarseIdx& c, int Gt, int gq, int d) {
    return g.F.unit(c.b, Gt, gq, 2 * c.zc + (d >> 2), 2 * c.yc + ((d >> 1) & 1), 2 * c.xc + (d & 1));
}
__device__ __forceinline__ size_t coarse_unit(const Grid2& g, const CoarseIdx& c, int Gt, int gq) {
    return g.C.unit(c.b, Gt, gq, c.zc, c.yc, c.xc);
}

// out (C channels, coarse) = mean of the 8 children in in (channels ico .. ico+C of ics)
__global__ void k_avgpool2(const bf16* __restrict__ in, int ics, int ico, int C, Grid2 g, bf16* __restrict__ out) {
    CoarseIdx c;
    if (!coarse_idx(g, C >> 3, c)) return;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < 8; ++d) {
        float f[8];
        ld8(in + 8 * fine_unit(g, c, ics >> 3, (ico >> 3) + c.q, d), f);
        for (int e = 0; e < 8; ++e) acc[e] += f[e];
    }
    for (int e = 0; e < 8; ++e) acc[e] *= 0.125f;
    st8(out + 8 * coarse_unit(g, c, C >> 3, c.q), acc);
}

// din (C channels, fine) = dout[parent] / 8 + add (channels aco .. aco+C of acs; may be NULL)
__global__ void k_avgpool2_bwd(const bf16* __restrict__ dout, const bf16* __restrict__ add, int acs, int aco, int C,
                               Grid2 g, bf16* __restrict__ din) {
    CoarseIdx c;
    if (!coarse_idx(g, C >> 3, c)) return;
    float f[8];
    ld8(dout + 8 * coarse_unit(g, c, C >> 3, c.q), f);
    for (int e = 0; e < 8; ++e) f[e] *= 0.125f;
    for (int d = 0; d < 8; ++d) {
        float o[8];
        for (int e = 0; e < 8; ++e) o[e] = f[e];
        if (add) {
            float a[8];
            ld8(add + 8 * fine_unit(g, c, acs >> 3, (aco >> 3) + c.q, d), a);
            for (int e = 0; e < 8; ++e) o[e] += a[e];
        }
        st8(din + 8 * fine_unit(g, c, C >> 3, c.q, d), o);
    }
}

// dout (C channels, coarse) = sum over the 8 children of din (channels ico .. ico+C of ics):
// the adjoint of the nearest-neighbour upsampling that the convolution epilogue does
__global__ void k_upsample2_bwd(const bf16* __restrict__ din, int ics, int ico, int C, Grid2 g,
                                bf16* __restrict__ dout) {
    CoarseIdx c;
    if (!coarse_idx(g, C >> 3, c)) return;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < 8; ++d) {
        float f[8];
        ld8(din + 8 * fine_unit(g, c, ics >> 3, (ico >> 3) + c.q, d), f);
        for (int e = 0; e < 8; ++e) acc[e] += f[e];
    }
    st8(dout + 8 * coarse_unit(g, c, C >> 3, c.q), acc);
}

// Launch geometry of the coarse-voxel kernels.
static bool coarse_grid(const Grid2& g, int C, int batch, dim3& grid) {
    const int G = C >> 3;
    if (C % 8 || G <= 0 || (g.F.D | g.F.H | g.F.W) & 1) return false;
    const long long z = (long long)g.C.D * batch;
    if (z > 65535 || g.C.H > 65535) return false;
    grid = dim3((unsigned)((g.C.W * G + 255) / 256), (unsigned)g.C.H, (unsigned)z);
    return true;
}

// Leaky ReLU backward over the whole padded tensors (the border is zero in both and stays
// zero): dy[u] *= (y > 0 ? 1 : slope), y the matching group of channels yco .. of ycs
// (y has the sign of the pre-activation).  units = batch x C/8 x padded voxels.
__global__ void k_relu_bwd(bf16* __restrict__ dy, const bf16* __restrict__ y, int ycs, int yco, int C, int units,
                           int vp, float slope) {
    const int G = C >> 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < units; i += gridDim.x * blockDim.x) {
        const int r = i / vp, v = i - r * vp, q = r % G, b = r / G;
        float f[8], t[8];
        ld8(dy + (size_t)8 * i, f);
        ld8(y + 8 * (((size_t)b * (ycs >> 3) + (yco >> 3) + q) * vp + v), t);
        for (int e = 0; e < 8; ++e)
            if (!(t[e] > 0.f)) f[e] *= slope;
        st8(dy + (size_t)8 * i, f);
    }
}

// db[8q + e] += sum over voxels of channel 8q + e of dy (padded channel-group-major, G = C/8
// groups; the border is zero and adds nothing).  Launch grid (nx, G), 256 threads: block
// column q sums group q in registers, reduces by warp shuffles and shared memory, and adds
// one value per channel.
__global__ void k_bias_grad(const bf16* __restrict__ dy, int batch, int vp, int G, float* __restrict__ db) {
    __shared__ float red[8][8];  // [warp][channel of the group]
    const int q = blockIdx.y;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b = 0; b < batch; ++b) {
        const bf16* base = dy + 8 * (((size_t)b * G + q) * vp);
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < vp; v += gridDim.x * blockDim.x) {
            float f[8];
            ld8(base + (size_t)8 * v, f);
            for (int e = 0; e < 8; ++e) acc[e] += f[e];
        }
    }
    for (int e = 0; e < 8; ++e)
        for (int off = 16; off > 0; off >>= 1) acc[e] += __shfl_down_sync(0xffffffffu, acc[e], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int e = 0; e < 8; ++e) red[warp][e] = acc[e];
    __syncthreads();
    if (threadIdx.x < 8) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        atomicAdd(&db[8 * q + threadIdx.x], t);
    }
}

// Loss and its gradient: pred = dose_low s + out[0]; diff = pred - t with t = target c s
// (c the target scale, e.g. the ratio of history counts of the two runs).  The squared
// error is weighted by 1/(t + kappa): the gamma index compares doses with local
// normalisation, so relative errors in low-dose voxels matter as much as absolute
// errors at the peak.  loss_acc += w diff^2; channel 0 of dout at (b, v) = 2 w diff.  The gradient
// is that of the summed loss (the reported loss is its mean): averaging over millions
// of voxels would push the gradients far below Adam's epsilon.
__global__ void k_loss(const float* __restrict__ dose_low, const float* __restrict__ out, const float* __restrict__ target,
                       float target_scale, const unsigned int* maxbits, Pcg g, int batch, bf16* __restrict__ dout,
                       float* loss_acc) {
    const size_t V = (size_t)g.D * g.H * g.W, n = V * batch;
    const float gscale = 2.f;
    float local = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / V);
        const int v = (int)(i - (size_t)b * V);
        const float s = scale_of(maxbits, b);
        const float t = target[i] * target_scale * s;
        const float diff = dose_low[i] * s + out[i] - t;
        const float w = 1.f / (fabsf(t) + kLossKappa);
        local += w * diff * diff;
        __nv_bfloat162 p[4];
        p[0] = __floats2bfloat162_rn(gscale * w * diff, 0.f);
        for (int j = 1; j < 4; ++j) p[j] = __floats2bfloat162_rn(0.f, 0.f);
        const int x = v % g.W, y = (v / g.W) % g.H, z = v / (g.W * g.H);
        *reinterpret_cast<uint4*>(dout + 8 * g.unit(b, 2, 0, z, y, x)) = *reinterpret_cast<uint4*>(p);
    }
    for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, local);
}

// dose_out = dose_low + out[0] / s  (back to Gy)
__global__ void k_output(const float* __restrict__ dose_low, const float* __restrict__ out, const unsigned int* maxbits,
                         size_t V, int batch, float* __restrict__ dose_out) {
    const size_t n = V * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float s = scale_of(maxbits, (int)(i / V));
        dose_out[i] = dose_low[i] + out[i] / s;
    }
}

// Adam (Kingma & Ba 2015) on FP32 master parameters, writing the BF16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ p16, size_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        const float pi = p[i] - upd;
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16(pi);
    }
}

__global__ void k_scale(float* __restrict__ x, size_t n, float c) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] *= c;
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// ------------------------------------------------------------------- gamma
__device__ __forceinline__ float trilinear(const float* __restrict__ f, int nx, int ny, int nz, float px, float py,
                                           float pz) {
    px = fminf(fmaxf(px, 0.f), (float)(nx - 1));
    py = fminf(fmaxf(py, 0.f), (float)(ny - 1));
    pz = fminf(fmaxf(pz, 0.f), (float)(nz - 1));
    const int x0 = min((int)px, max(nx - 2, 0)), y0 = min((int)py, max(ny - 2, 0)), z0 = min((int)pz, max(nz - 2, 0));
    const int x1 = min(x0 + 1, nx - 1), y1 = min(y0 + 1, ny - 1), z1 = min(z0 + 1, nz - 1);
    const float fx = px - x0, fy = py - y0, fz = pz - z0;
    auto at = [&](int x, int y, int z) { return f[((size_t)z * ny + y) * nx + x]; };
    const float c00 = at(x0, y0, z0) * (1 - fx) + at(x1, y0, z0) * fx;
    const float c10 = at(x0, y1, z0) * (1 - fx) + at(x1, y1, z0) * fx;
    const float c01 = at(x0, y0, z1) * (1 - fx) + at(x1, y0, z1) * fx;
    const float c11 = at(x0, y1, z1) * (1 - fx) + at(x1, y1, z1) * fx;
    return (c00 * (1 - fy) + c10 * fy) * (1 - fz) + (c01 * (1 - fy) + c11 * fy) * fz;
}

// Local-normalisation gamma: a reference voxel with dose >= thr passes when some
// evaluated position within the DTA ball (grid step dta/steps, trilinear) has
// |dr|^2/dta^2 + (De - Dr)^2/(dd Dr)^2 <= 1.  counts[0] += evaluated, counts[1] += passed.
__global__ void k_gamma(const float* __restrict__ ref, const float* __restrict__ ev, int nx, int ny, int nz, float hx,
                        float hy, float hz, float dd, float dta, float thr, int steps, unsigned long long* counts) {
    const size_t n = (size_t)nx * ny * nz;
    unsigned int evals = 0, passes = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float r = ref[i];
        if (!(r >= thr) || !(r > 0.f)) continue;
        evals += 1;
        const float tol = dd * r;
        bool pass = fabsf(ev[i] - r) <= tol;
        if (!pass) {
            const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((size_t)nx * ny));
            const float st = dta / steps, inv_dta2 = 1.f / (dta * dta), inv_tol2 = 1.f / (tol * tol);
            for (int a = -steps; a <= steps && !pass; ++a)
                for (int b = -steps; b <= steps && !pass; ++b)
                    for (int c = -steps; c <= steps; ++c) {
                        const float oz = a * st, oy = b * st, ox = c * st;
                        const float d2 = (ox * ox + oy * oy + oz * oz) * inv_dta2;
                        if (d2 > 1.f) continue;
                        const float e = trilinear(ev, nx, ny, nz, ix + ox / hx, iy + oy / hy, iz + oz / hz);
                        if (d2 + (e - r) * (e - r) * inv_tol2 <= 1.f) {
                            pass = true;
                            break;
                        }
                    }
        }
        passes += pass ? 1u : 0u;
    }
    for (int off = 16; off > 0; off >>= 1) {
        evals += __shfl_down_sync(0xffffffffu, evals, off);
        passes += __shfl_down_sync(0xffffffffu, passes, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], (unsigned long long)evals);
        atomicAdd(&counts[1], (unsigned long long)passes);
    }
}

__global__ void k_max(const float* __restrict__ x, size_t n, unsigned int* out_bits) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, x[i]);
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

int fail(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SDE_OK;
    char m[256];
    snprintf(m, sizeof m, "%s: %s", what, cudaGetErrorString(e));
    set_last_error(m);
    return e == cudaErrorMemoryAllocation ? SDE_ENOMEM : SDE_ECUDA;
}

}  // namespace
}  // namespace sde

using namespace sde;

namespace {

struct Layer {
    int Cin, Cout;
    bool relu;
    int lvl;  // resolution level: grid / 2^lvl
    size_t nw;
    float *w32, *b32, *gw, *gb, *mw, *vw, *mb, *vb;
    bf16 *w16, *wflip;
    bf16 *wpk, *wpkf;  // w16 and wflip packed for the tensor core (conv_pack_weights)
    int cp, cpf;       // their output channels per part
};

// Each grid-stride kernel uses this many blocks.
constexpr int kBlocks = 152 * 8;

}  // namespace

struct sde_denoiser {
    int D = 0, H = 0, W = 0, batch_max = 0;
    size_t V1 = 0, V2 = 0, V3 = 0;
    cudaStream_t st = nullptr;
    Layer L[11];
    long long adam_t = 0;
    std::vector<void*> allocs;
    // activations
    bf16 *in0, *e1a, *cat1, *p1, *e2a, *cat2, *p2, *b1, *b2, *d2a, *d2, *d1a, *d1;
    float* out;
    // gradients
    bf16 *g_out, *g_d1, *g_d1a, *g_cat1, *g_d2, *g_d2a, *g_cat2, *g_b2, *g_b1, *g_p2, *g_e2, *g_e2a, *g_p1, *g_e1,
        *g_e1a;
    unsigned int* maxbits;
    float* loss_acc;
    unsigned long long* gcounts;
    unsigned int* gmax;
};

namespace {

template <typename T>
int dalloc(sde_denoiser* d, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) return fail(e, "cudaMalloc");
    d->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SDE_OK;
}

void free_denoiser(sde_denoiser* d) {
    for (void* p : d->allocs) cudaFree(p);
    d->allocs.clear();
}

// Deterministic normal draws for the weight initialisation (SplitMix64 + Box-Muller).
struct HostRng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return sqrt(-2.0 * log(uniform())) * cos(6.283185307179586 * uniform()); }
};

// One convolution of layer l at grid D x H x W: the forward one, or with flip the data
// gradient (dy convolved with the flipped weights, Cin and Cout exchanged).
int conv(sde_denoiser* d, const bf16* x, int batch, int D, int H, int W, const Layer& l, bool flip, int Cout,
         void* y, int cstride, int coffset, bool fp32, bool relu, const float* bias, int keep = 0,
         bf16* up = nullptr, int up_cstride = 0, int up_coffset = 0) {
    unsigned int* status = nullptr;
    int rc = fail(denoise_status_word(&status), "status word");
    if (rc) return rc;
    ConvArgs a;
    a.x = x;
    a.wpk = flip ? l.wpkf : l.wpk;
    a.wpk_cp = flip ? l.cpf : l.cp;
    a.bias = bias;
    a.y = y;
    a.D = D;
    a.H = H;
    a.W = W;
    a.Cin = flip ? l.Cout : l.Cin;
    a.Cout = Cout;
    a.nvox = D * H * W;
    a.y_cstride = cstride;
    a.y_coffset = coffset;
    a.y_fp32 = fp32 ? 1 : 0;
    a.y_keep = keep;
    a.y_up = up;
    a.y_up_cstride = up_cstride;
    a.y_up_coffset = up_coffset;
    a.relu = relu ? 1 : 0;
    a.slope = kLeak;
    a.status = status;
    return fail(conv3d_launch(a, batch, d->st), "conv3d launch");
}

int wgrad(sde_denoiser* d, const bf16* x, const bf16* dy, const Layer& l, int batch, int D, int H, int W) {
    unsigned int* status = nullptr;
    int rc = fail(denoise_status_word(&status), "status word");
    if (rc) return rc;
    WgradArgs a;
    a.x = x;
    a.dy = dy;
    a.dw = l.gw;
    a.D = D;
    a.H = H;
    a.W = W;
    a.Cin = l.Cin;
    a.Cout = l.Cout;
    a.nvox = D * H * W;
    a.batch = batch;
    a.status = status;
    rc = fail(wgrad_launch(a, d->st), "wgrad launch");
    if (rc) return rc;
    const int vp = (int)Pcg{D, H, W}.vp();
    const int G = l.Cout >> 3;
    const dim3 grid((unsigned)(kBlocks / G > 1 ? kBlocks / G : 1), (unsigned)G);
    k_bias_grad<<<grid, 256, 0, d->st>>>(dy, batch, vp, G, l.gb);
    return fail(cudaGetLastError(), "bias grad launch");
}

int relu_bwd(sde_denoiser* d, bf16* dy, const bf16* y, int ycs, int yco, int C, int batch, const Pcg& g) {
    const int vp = (int)g.vp();
    k_relu_bwd<<<kBlocks, 256, 0, d->st>>>(dy, y, ycs, yco, C, batch * (C >> 3) * vp, vp, kLeak);
    return fail(cudaGetLastError(), "relu bwd launch");
}

#define DN_TRY(x)              \
    do {                       \
        int rc_ = (x);         \
        if (rc_) return rc_;   \
    } while (0)

int forward(sde_denoiser* d, const float* dose_low, const float* rho, int batch) {
    const int D = d->D, H = d->H, W = d->W;
    const int D2 = D / 2, H2 = H / 2, W2 = W / 2, D3 = D / 4, H3 = H / 4, W3 = W / 4;
    const Grid2 g1 = grid2(D, H, W), g2 = grid2(D2, H2, W2);
    DN_TRY(fail(cudaMemsetAsync(d->maxbits, 0, sizeof(unsigned int) * d->batch_max, d->st), "memset"));
    k_absmax<<<kBlocks, 256, 0, d->st>>>(dose_low, d->V1, batch, d->maxbits);
    k_prepare_input<<<kBlocks, 256, 0, d->st>>>(dose_low, rho, g1.F, batch, d->maxbits, d->in0);
    DN_TRY(fail(cudaGetLastError(), "input launch"));
    Layer* L = d->L;
    DN_TRY(conv(d, d->in0, batch, D, H, W, L[0], false, 32, d->e1a, 32, 0, false, true, L[0].b32));
    DN_TRY(conv(d, d->e1a, batch, D, H, W, L[1], false, 32, d->cat1, 96, 64, false, true, L[1].b32));
    dim3 grid;
    if (!coarse_grid(g1, 64, batch, grid) || !coarse_grid(g2, 128, batch, grid))
        return fail(cudaErrorInvalidValue, "pooling grid");
    coarse_grid(g1, 32, batch, grid);
    k_avgpool2<<<grid, 256, 0, d->st>>>(d->cat1, 96, 64, 32, g1, d->p1);
    DN_TRY(conv(d, d->p1, batch, D2, H2, W2, L[2], false, 64, d->e2a, 64, 0, false, true, L[2].b32));
    DN_TRY(conv(d, d->e2a, batch, D2, H2, W2, L[3], false, 64, d->cat2, 192, 128, false, true, L[3].b32));
    coarse_grid(g2, 64, batch, grid);
    k_avgpool2<<<grid, 256, 0, d->st>>>(d->cat2, 192, 128, 64, g2, d->p2);
    DN_TRY(conv(d, d->p2, batch, D3, H3, W3, L[4], false, 128, d->b1, 128, 0, false, true, L[4].b32));
    // b2, and its nearest-neighbour upsampling into channels 0..127 of cat2, from one epilogue
    DN_TRY(conv(d, d->b1, batch, D3, H3, W3, L[5], false, 128, d->b2, 128, 0, false, true, L[5].b32, 0, d->cat2,
                192, 0));
    DN_TRY(conv(d, d->cat2, batch, D2, H2, W2, L[6], false, 64, d->d2a, 64, 0, false, true, L[6].b32));
    DN_TRY(conv(d, d->d2a, batch, D2, H2, W2, L[7], false, 64, d->d2, 64, 0, false, true, L[7].b32, 0, d->cat1,
                96, 0));
    DN_TRY(conv(d, d->cat1, batch, D, H, W, L[8], false, 32, d->d1a, 32, 0, false, true, L[8].b32));
    DN_TRY(conv(d, d->d1a, batch, D, H, W, L[9], false, 32, d->d1, 32, 0, false, true, L[9].b32));
    // only output channel 0 is the network's output (the other 15 of the padded layer are unused)
    DN_TRY(conv(d, d->d1, batch, D, H, W, L[10], false, 16, d->out, 16, 0, true, false, L[10].b32, 1));
    return fail(cudaGetLastError(), "forward launch");
}

int backward(sde_denoiser* d, int batch) {
    const int D = d->D, H = d->H, W = d->W;
    const int D2 = D / 2, H2 = H / 2, W2 = W / 2, D3 = D / 4, H3 = H / 4, W3 = W / 4;
    const Grid2 g1 = grid2(D, H, W), g2 = grid2(D2, H2, W2);
    const Pcg& P1 = g1.F;
    const Pcg& P2 = g2.F;
    const Pcg& P3 = g2.C;
    Layer* L = d->L;
    dim3 grid;
    // out layer
    DN_TRY(wgrad(d, d->d1, d->g_out, L[10], batch, D, H, W));
    DN_TRY(conv(d, d->g_out, batch, D, H, W, L[10], true, 32, d->g_d1, 32, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_d1, d->d1, 32, 0, 32, batch, P1));
    DN_TRY(wgrad(d, d->d1a, d->g_d1, L[9], batch, D, H, W));
    DN_TRY(conv(d, d->g_d1, batch, D, H, W, L[9], true, 32, d->g_d1a, 32, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_d1a, d->d1a, 32, 0, 32, batch, P1));
    DN_TRY(wgrad(d, d->cat1, d->g_d1a, L[8], batch, D, H, W));
    DN_TRY(conv(d, d->g_d1a, batch, D, H, W, L[8], true, 96, d->g_cat1, 96, 0, false, false, nullptr));
    coarse_grid(g1, 64, batch, grid);
    k_upsample2_bwd<<<grid, 256, 0, d->st>>>(d->g_cat1, 96, 0, 64, g1, d->g_d2);
    DN_TRY(relu_bwd(d, d->g_d2, d->d2, 64, 0, 64, batch, P2));
    DN_TRY(wgrad(d, d->d2a, d->g_d2, L[7], batch, D2, H2, W2));
    DN_TRY(conv(d, d->g_d2, batch, D2, H2, W2, L[7], true, 64, d->g_d2a, 64, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_d2a, d->d2a, 64, 0, 64, batch, P2));
    DN_TRY(wgrad(d, d->cat2, d->g_d2a, L[6], batch, D2, H2, W2));
    DN_TRY(conv(d, d->g_d2a, batch, D2, H2, W2, L[6], true, 192, d->g_cat2, 192, 0, false, false, nullptr));
    coarse_grid(g2, 128, batch, grid);
    k_upsample2_bwd<<<grid, 256, 0, d->st>>>(d->g_cat2, 192, 0, 128, g2, d->g_b2);
    DN_TRY(relu_bwd(d, d->g_b2, d->b2, 128, 0, 128, batch, P3));
    DN_TRY(wgrad(d, d->b1, d->g_b2, L[5], batch, D3, H3, W3));
    DN_TRY(conv(d, d->g_b2, batch, D3, H3, W3, L[5], true, 128, d->g_b1, 128, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_b1, d->b1, 128, 0, 128, batch, P3));
    DN_TRY(wgrad(d, d->p2, d->g_b1, L[4], batch, D3, H3, W3));
    DN_TRY(conv(d, d->g_b1, batch, D3, H3, W3, L[4], true, 64, d->g_p2, 64, 0, false, false, nullptr));
    coarse_grid(g2, 64, batch, grid);
    k_avgpool2_bwd<<<grid, 256, 0, d->st>>>(d->g_p2, d->g_cat2, 192, 128, 64, g2, d->g_e2);
    DN_TRY(relu_bwd(d, d->g_e2, d->cat2, 192, 128, 64, batch, P2));
    DN_TRY(wgrad(d, d->e2a, d->g_e2, L[3], batch, D2, H2, W2));
    DN_TRY(conv(d, d->g_e2, batch, D2, H2, W2, L[3], true, 64, d->g_e2a, 64, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_e2a, d->e2a, 64, 0, 64, batch, P2));
    DN_TRY(wgrad(d, d->p1, d->g_e2a, L[2], batch, D2, H2, W2));
    DN_TRY(conv(d, d->g_e2a, batch, D2, H2, W2, L[2], true, 32, d->g_p1, 32, 0, false, false, nullptr));
    coarse_grid(g1, 32, batch, grid);
    k_avgpool2_bwd<<<grid, 256, 0, d->st>>>(d->g_p1, d->g_cat1, 96, 64, 32, g1, d->g_e1);
    DN_TRY(relu_bwd(d, d->g_e1, d->cat1, 96, 64, 32, batch, P1));
    DN_TRY(wgrad(d, d->e1a, d->g_e1, L[1], batch, D, H, W));
    DN_TRY(conv(d, d->g_e1, batch, D, H, W, L[1], true, 32, d->g_e1a, 32, 0, false, false, nullptr));
    DN_TRY(relu_bwd(d, d->g_e1a, d->e1a, 32, 0, 32, batch, P1));
    DN_TRY(wgrad(d, d->in0, d->g_e1a, L[0], batch, D, H, W));
    return fail(cudaGetLastError(), "backward launch");
}

// After every change of the BF16 weights: the flipped copies and both packed images.
int refresh_weights(sde_denoiser* d) {
    for (int i = 0; i < 11; ++i) {
        Layer& l = d->L[i];
        DN_TRY(fail(conv_pack_weights(l.w16, l.wpk, l.Cin, l.Cout, l.cp, d->st), "pack"));
        if (i == 0) continue;  // the input layer needs no data gradient
        DN_TRY(fail(flip_weights_launch(l.w16, l.wflip, l.Cin, l.Cout, d->st), "flip"));
        DN_TRY(fail(conv_pack_weights(l.wflip, l.wpkf, l.Cout, l.Cin, l.cpf, d->st), "pack"));
    }
    return SDE_OK;
}


}  // namespace

extern "C" int sde_denoiser_create(sde_denoiser** out, int D, int H, int W, int batch_max, uint64_t seed) {
    if (!out || D < 4 || H < 4 || W < 4 || (D % 4) || (H % 4) || (W % 4) || W > 256 || batch_max < 1 ||
        (long long)(D + 2) * (H + 2) * (W + 2) * batch_max * 24 >= (1ll << 31)) {
        set_last_error("sde_denoiser_create: D, H, W must be multiples of 4, W <= 256, and (D+2)(H+2)(W+2) batch_max "
                       "below 2^31 / 24");
        return SDE_EINVAL;
    }
    sde_denoiser* d = new (std::nothrow) sde_denoiser();
    if (!d) {
        set_last_error("out of host memory");
        return SDE_ENOMEM;
    }
    d->D = D;
    d->H = H;
    d->W = W;
    d->batch_max = batch_max;
    d->V1 = (size_t)D * H * W;
    d->V2 = d->V1 / 8;
    d->V3 = d->V2 / 8;
    const int cin[11] = {16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 32};
    const int cout[11] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16};
    const int lvl[11] = {0, 0, 1, 1, 2, 2, 1, 1, 0, 0, 0};
    HostRng rng{seed ^ 0xD1B54A32D192ED03ull};
    int rc = SDE_OK;
    for (int i = 0; i < 11 && rc == SDE_OK; ++i) {
        Layer& l = d->L[i];
        l.Cin = cin[i];
        l.Cout = cout[i];
        l.relu = i < 10;
        l.lvl = lvl[i];
        l.nw = (size_t)l.Cout * 27 * l.Cin;
        const int Dl = D >> l.lvl, Hl = H >> l.lvl, Wl = W >> l.lvl;
        l.cp = conv_plan_cp(Dl, Hl, Wl, l.Cin, l.Cout);
        l.cpf = conv_plan_cp(Dl, Hl, Wl, l.Cout, l.Cin);
        if (!l.cp || !l.cpf) {
            set_last_error("sde_denoiser_create: no convolution tile plan for this grid");
            rc = SDE_EINVAL;
            break;
        }
        rc = dalloc(d, &l.w32, l.nw);
        if (!rc) rc = dalloc(d, &l.gw, l.nw);
        if (!rc) rc = dalloc(d, &l.mw, l.nw);
        if (!rc) rc = dalloc(d, &l.vw, l.nw);
        if (!rc) rc = dalloc(d, &l.b32, (size_t)l.Cout);
        if (!rc) rc = dalloc(d, &l.gb, (size_t)l.Cout);
        if (!rc) rc = dalloc(d, &l.mb, (size_t)l.Cout);
        if (!rc) rc = dalloc(d, &l.vb, (size_t)l.Cout);
        if (!rc) rc = dalloc(d, &l.w16, l.nw);
        if (!rc) rc = dalloc(d, &l.wflip, l.nw);
        if (!rc) rc = dalloc(d, &l.wpk, l.nw);
        if (!rc) rc = dalloc(d, &l.wpkf, l.nw);
        if (rc) break;
        // He initialisation; the input layer sees two live channels; the output layer
        // starts at zero, so that the untrained network is the identity on the dose
        // (its output is a correction added to the input dose).
        const int fan_in = 27 * (i == 0 ? 2 : l.Cin);
        const double sd = (i == 10 ? 0.0 : 1.0) * sqrt(2.0 / fan_in);
        std::vector<float> w(l.nw);
        for (size_t k = 0; k < l.nw; ++k) w[k] = (float)(sd * rng.normal());
        rc = fail(cudaMemcpy(l.w32, w.data(), l.nw * sizeof(float), cudaMemcpyHostToDevice), "weights upload");
        if (!rc) rc = fail(cudaMemset(l.b32, 0, l.Cout * sizeof(float)), "memset");
        if (!rc) rc = fail(cudaMemset(l.mw, 0, l.nw * sizeof(float)), "memset");
        if (!rc) rc = fail(cudaMemset(l.vw, 0, l.nw * sizeof(float)), "memset");
        if (!rc) rc = fail(cudaMemset(l.mb, 0, l.Cout * sizeof(float)), "memset");
        if (!rc) rc = fail(cudaMemset(l.vb, 0, l.Cout * sizeof(float)), "memset");
        if (!rc) {
            k_to_bf16<<<kBlocks, 256>>>(l.w32, l.w16, l.nw);
            rc = fail(cudaGetLastError(), "to bf16");
        }
    }
    // activations and their gradients: padded channel-group-major, borders zero for good
    const size_t B = (size_t)batch_max;
    const size_t V1 = Pcg{D, H, W}.vp() * B, V2 = Pcg{D / 2, H / 2, W / 2}.vp() * B,
                 V3 = Pcg{D / 4, H / 4, W / 4}.vp() * B;
    struct {
        bf16** p;
        size_t n;
    } acts[] = {{&d->in0, V1 * 16}, {&d->e1a, V1 * 32}, {&d->cat1, V1 * 96}, {&d->p1, V2 * 32},
                {&d->e2a, V2 * 64}, {&d->cat2, V2 * 192}, {&d->p2, V3 * 64}, {&d->b1, V3 * 128},
                {&d->b2, V3 * 128}, {&d->d2a, V2 * 64}, {&d->d2, V2 * 64}, {&d->d1a, V1 * 32},
                {&d->d1, V1 * 32}, {&d->g_out, V1 * 16}, {&d->g_d1, V1 * 32}, {&d->g_d1a, V1 * 32},
                {&d->g_cat1, V1 * 96}, {&d->g_d2, V2 * 64}, {&d->g_d2a, V2 * 64}, {&d->g_cat2, V2 * 192},
                {&d->g_b2, V3 * 128}, {&d->g_b1, V3 * 128}, {&d->g_p2, V3 * 64}, {&d->g_e2, V2 * 64},
                {&d->g_e2a, V2 * 64}, {&d->g_p1, V2 * 32}, {&d->g_e1, V1 * 32}, {&d->g_e1a, V1 * 32}};
    for (auto& a : acts) {
        if (!rc) rc = dalloc(d, a.p, a.n);
        if (!rc) rc = fail(cudaMemset(*a.p, 0, a.n * sizeof(bf16)), "memset");
    }
    if (!rc) rc = dalloc(d, &d->out, d->V1 * B);  // FP32 output channel 0, plain [n][voxel]
    if (!rc) rc = dalloc(d, &d->maxbits, B);
    if (!rc) rc = dalloc(d, &d->loss_acc, (size_t)1);
    if (!rc) rc = dalloc(d, &d->gcounts, (size_t)2);
    if (!rc) rc = dalloc(d, &d->gmax, (size_t)1);
    if (!rc) rc = refresh_weights(d);
    if (!rc) rc = fail(cudaDeviceSynchronize(), "create sync");
    if (rc) {
        free_denoiser(d);
        delete d;
        return rc;
    }
    *out = d;
    return SDE_OK;
}

extern "C" void sde_denoiser_destroy(sde_denoiser* d) {
    if (!d) return;
    cudaStreamSynchronize(d->st);
    free_denoiser(d);
    delete d;
}

extern "C" int sde_denoiser_set_stream(sde_denoiser* d, void* stream) {
    if (!d) {
        set_last_error("null denoiser");
        return SDE_EINVAL;
    }
    d->st = (cudaStream_t)stream;
    return SDE_OK;
}

extern "C" int sde_denoiser_num_params(const sde_denoiser* d, uint64_t* n) {
    if (!d || !n) {
        set_last_error("null argument");
        return SDE_EINVAL;
    }
    uint64_t t = 0;
    for (const Layer& l : d->L) t += l.nw + l.Cout;
    *n = t;
    return SDE_OK;
}

extern "C" int sde_denoiser_infer(sde_denoiser* d, const float* d_dose_low, const float* d_density, int batch,
                                  float* d_dose_out) {
    if (!d || !d_dose_low || !d_density || !d_dose_out || batch < 1 || batch > d->batch_max) {
        set_last_error("sde_denoiser_infer: bad arguments");
        return SDE_EINVAL;
    }
    DN_TRY(forward(d, d_dose_low, d_density, batch));
    k_output<<<kBlocks, 256, 0, d->st>>>(d_dose_low, d->out, d->maxbits, d->V1, batch, d_dose_out);
    return fail(cudaGetLastError(), "output launch");
}

extern "C" int sde_denoiser_train_step(sde_denoiser* d, const float* d_dose_low, const float* d_density,
                                       const float* d_dose_high, float target_scale, int batch, float lr,
                                       float* loss_out) {
    if (!d || !d_dose_low || !d_density || !d_dose_high || batch < 1 || batch > d->batch_max || !(lr > 0.f)) {
        set_last_error("sde_denoiser_train_step: bad arguments");
        return SDE_EINVAL;
    }
    DN_TRY(forward(d, d_dose_low, d_density, batch));
    DN_TRY(fail(cudaMemsetAsync(d->loss_acc, 0, sizeof(float), d->st), "memset"));
    k_loss<<<kBlocks, 256, 0, d->st>>>(d_dose_low, d->out, d_dose_high, target_scale, d->maxbits,
                                       Pcg{d->D, d->H, d->W}, batch, d->g_out, d->loss_acc);
    DN_TRY(fail(cudaGetLastError(), "loss launch"));
    for (Layer& l : d->L) {
        DN_TRY(fail(cudaMemsetAsync(l.gw, 0, l.nw * sizeof(float), d->st), "memset"));
        DN_TRY(fail(cudaMemsetAsync(l.gb, 0, l.Cout * sizeof(float), d->st), "memset"));
    }
    DN_TRY(backward(d, batch));
    d->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)d->adam_t), bc2 = 1.f - powf(b2, (float)d->adam_t);
    for (Layer& l : d->L) {
        k_adam<<<kBlocks, 256, 0, d->st>>>(l.w32, l.gw, l.mw, l.vw, l.w16, l.nw, lr, b1, b2, 1e-8f, bc1, bc2);
        k_adam<<<8, 256, 0, d->st>>>(l.b32, l.gb, l.mb, l.vb, nullptr, (size_t)l.Cout, lr, b1, b2, 1e-8f, bc1, bc2);
    }
    DN_TRY(fail(cudaGetLastError(), "adam launch"));
    DN_TRY(refresh_weights(d));
    if (loss_out) {
        float h = 0.f;
        DN_TRY(fail(cudaMemcpyAsync(&h, d->loss_acc, sizeof h, cudaMemcpyDeviceToHost, d->st), "loss copy"));
        DN_TRY(denoise_check_status(d->st));
        *loss_out = h / (float)(d->V1 * batch);
    }
    return SDE_OK;
}

// Parameters as one FP32 vector (per layer: weights [Cout][27][Cin], then biases).
extern "C" int sde_denoiser_get_params(const sde_denoiser* d, float* host, uint64_t n) {
    uint64_t need = 0;
    if (!d || !host || sde_denoiser_num_params(d, &need) || n < need) {
        set_last_error("sde_denoiser_get_params: bad arguments");
        return SDE_EINVAL;
    }
    cudaStreamSynchronize(d->st);
    size_t o = 0;
    for (const Layer& l : d->L) {
        DN_TRY(fail(cudaMemcpy(host + o, l.w32, l.nw * sizeof(float), cudaMemcpyDeviceToHost), "params copy"));
        o += l.nw;
        DN_TRY(fail(cudaMemcpy(host + o, l.b32, l.Cout * sizeof(float), cudaMemcpyDeviceToHost), "params copy"));
        o += l.Cout;
    }
    return SDE_OK;
}

extern "C" int sde_denoiser_set_params(sde_denoiser* d, const float* host, uint64_t n) {
    uint64_t need = 0;
    if (!d || !host || sde_denoiser_num_params(d, &need) || n < need) {
        set_last_error("sde_denoiser_set_params: bad arguments");
        return SDE_EINVAL;
    }
    cudaStreamSynchronize(d->st);
    size_t o = 0;
    for (Layer& l : d->L) {
        DN_TRY(fail(cudaMemcpy(l.w32, host + o, l.nw * sizeof(float), cudaMemcpyHostToDevice), "params copy"));
        o += l.nw;
        DN_TRY(fail(cudaMemcpy(l.b32, host + o, l.Cout * sizeof(float), cudaMemcpyHostToDevice), "params copy"));
        o += l.Cout;
        k_to_bf16<<<kBlocks, 256, 0, d->st>>>(l.w32, l.w16, l.nw);
    }
    DN_TRY(refresh_weights(d));
    return fail(cudaDeviceSynchronize(), "set params sync");
}

// Gradient of the loss with respect to all parameters for one batch, without an
// update (for checking the backward pass).  host: FP32 vector in the order of
// sde_denoiser_get_params.
extern "C" int sde_denoiser_gradients(sde_denoiser* d, const float* d_dose_low, const float* d_density,
                                      const float* d_dose_high, float target_scale, int batch, float* host_grad,
                                      uint64_t n, float* loss_out) {
    uint64_t need = 0;
    if (!d || !host_grad || sde_denoiser_num_params(d, &need) || n < need || batch < 1 || batch > d->batch_max) {
        set_last_error("sde_denoiser_gradients: bad arguments");
        return SDE_EINVAL;
    }
    DN_TRY(forward(d, d_dose_low, d_density, batch));
    DN_TRY(fail(cudaMemsetAsync(d->loss_acc, 0, sizeof(float), d->st), "memset"));
    k_loss<<<kBlocks, 256, 0, d->st>>>(d_dose_low, d->out, d_dose_high, target_scale, d->maxbits,
                                       Pcg{d->D, d->H, d->W}, batch, d->g_out, d->loss_acc);
    for (Layer& l : d->L) {
        DN_TRY(fail(cudaMemsetAsync(l.gw, 0, l.nw * sizeof(float), d->st), "memset"));
        DN_TRY(fail(cudaMemsetAsync(l.gb, 0, l.Cout * sizeof(float), d->st), "memset"));
    }
    DN_TRY(backward(d, batch));
    DN_TRY(denoise_check_status(d->st));
    size_t o = 0;
    for (const Layer& l : d->L) {
        DN_TRY(fail(cudaMemcpy(host_grad + o, l.gw, l.nw * sizeof(float), cudaMemcpyDeviceToHost), "grad copy"));
        o += l.nw;
        DN_TRY(fail(cudaMemcpy(host_grad + o, l.gb, l.Cout * sizeof(float), cudaMemcpyDeviceToHost), "grad copy"));
        o += l.Cout;
    }
    if (loss_out) {
        float h = 0.f;
        DN_TRY(fail(cudaMemcpy(&h, d->loss_acc, sizeof h, cudaMemcpyDeviceToHost), "loss copy"));
        *loss_out = h / (float)(d->V1 * batch);
    }
    return SDE_OK;
}

extern "C" int sde_scale_f32(float* d_x, uint64_t n, float factor, void* stream) {
    if (!d_x) {
        set_last_error("sde_scale_f32: null pointer");
        return SDE_EINVAL;
    }
    k_scale<<<kBlocks, 256, 0, (cudaStream_t)stream>>>(d_x, (size_t)n, factor);
    return fail(cudaGetLastError(), "scale launch");
}

extern "C" int sde_gamma3d(const float* d_ref, const float* d_eval, int nx, int ny, int nz, const double voxel_mm[3],
                           double dd, double dta_mm, double threshold, int steps, uint64_t* n_eval,
                           uint64_t* n_pass, void* stream) {
    if (!d_ref || !d_eval || nx < 1 || ny < 1 || nz < 1 || !voxel_mm || !(dd > 0) || !(dta_mm > 0) || steps < 1 ||
        steps > 50 || !n_eval || !n_pass) {
        set_last_error("sde_gamma3d: bad arguments");
        return SDE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* counts = nullptr;
    unsigned int* mx = nullptr;
    DN_TRY(fail(cudaMallocAsync(&counts, 2 * sizeof(unsigned long long) + sizeof(unsigned int), st), "alloc"));
    mx = reinterpret_cast<unsigned int*>(counts + 2);
    int rc = fail(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long) + sizeof(unsigned int), st), "memset");
    const size_t n = (size_t)nx * ny * nz;
    unsigned int h_mx = 0;
    unsigned long long h[2] = {0, 0};
    if (!rc) {
        k_max<<<kBlocks, 256, 0, st>>>(d_ref, n, mx);
        rc = fail(cudaMemcpyAsync(&h_mx, mx, sizeof h_mx, cudaMemcpyDeviceToHost, st), "copy");
    }
    if (!rc) rc = fail(cudaStreamSynchronize(st), "sync");
    if (!rc) {
        float dmax;
        memcpy(&dmax, &h_mx, sizeof dmax);
        k_gamma<<<kBlocks, 256, 0, st>>>(d_ref, d_eval, nx, ny, nz, (float)voxel_mm[0], (float)voxel_mm[1],
                                         (float)voxel_mm[2], (float)dd, (float)dta_mm, (float)(threshold * dmax),
                                         steps, counts);
        rc = fail(cudaGetLastError(), "gamma launch");
    }
    if (!rc) rc = fail(cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st), "copy");
    if (!rc) rc = fail(cudaStreamSynchronize(st), "sync");
    cudaFreeAsync(counts, st);
    if (rc) return rc;
    *n_eval = h[0];
    *n_pass = h[1];
    return SDE_OK;
}
