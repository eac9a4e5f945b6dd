// sde_denoise.h -- internal interface of the denoiser's tensor-core kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sde {

// 3x3x3 convolution as an implicit GEMM (see sde_denoise.cu).
struct ConvArgs {
    const __nv_bfloat16* x;
    const __nv_bfloat16* w;
    const float* bias;
    void* y;
    int D, H, W, Cin, Cout;
    int nvox;  // D*H*W (a multiple of 128)
    int y_cstride, y_coffset, y_fp32, relu;
    float slope;  // with relu: y = x > 0 ? x : slope * x (0: ReLU, > 0: leaky ReLU)
    unsigned int* status;
};

// Work decomposition and shared-memory layout of the pipelined brick convolution
// (host-chosen per layer shape).  A work item is (sample, Cout part, row block, z plane).
struct BrickPlan {
    int Ty;      // output rows (y) per work item, all x of one z plane
    int tiles;   // M tiles of 128 brick positions per work item
    int nyb;     // ceil(H / Ty)
    int P;       // W + 2: brick row pitch in positions
    int Yb;      // Ty + 2: brick rows per plane
    int Cp;      // output channels per work item
    int nsplit;  // Cout / Cp
    int plane;   // bytes between the two 8-channel planes of a 16-channel chunk
    int w_off;   // offset of the chunk's weights (27 taps x Cp x 16) within a stage (wres = 0)
    int wres;    // 1: all chunks' weights stay resident after the stages (loaded once per CTA)
    int stage;   // bytes per pipeline stage (brick chunk + weight chunk)
    int nacc;    // tensor-memory accumulators (2: epilogue overlaps the next item)
    int tcols;   // tensor-memory columns allocated (power of two >= nacc x tiles x Cp)
    int items;   // batch x nsplit x nyb x D
};

// Weight gradient: dw[co][tap][ci] += sum_v dy[v][co] x[v + off(tap)][ci] (brick kernel,
// see sde_denoise.cu).
struct WgradArgs {
    const __nv_bfloat16* x;   // [n][V][Cin]
    const __nv_bfloat16* dy;  // [n][V][Cout]
    float* dw;                // [Cout][27][Cin], accumulated
    int D, H, W, Cin, Cout, nvox, batch;
    unsigned int* status;
};

// Work decomposition of the brick weight-gradient kernel (host-chosen).  A pass is one
// chunk of Nc input channels and one group of taps (its accumulators fill tensor memory);
// a work item is Ty output rows of one z plane.
struct WgradPlan {
    int Ty, nyb, P, Yb;  // as BrickPlan
    int Nc;              // input channels per pass (MMA N)
    int ntap, ngroups;   // taps per pass, tap groups
    int kst;             // K steps (16 positions) per item
    int plane_dy;        // bytes between 8-channel planes of the output-gradient rows
    int plane_x;         // bytes between 8-channel planes of the input brick
    int x_off;           // offset of the input brick within a stage
    int stage;           // bytes per stage
    int items;           // batch x nyb x D
    int G;               // CTAs per pass
};

cudaError_t conv3d_launch(const ConvArgs& a, int batch, cudaStream_t st);
cudaError_t wgrad_launch(const WgradArgs& a, cudaStream_t st);
cudaError_t flip_weights_launch(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout, cudaStream_t st);
cudaError_t denoise_status_word(unsigned int** out);
int denoise_check_status(cudaStream_t st);

}  // namespace sde
