// sde_denoise.h -- internal interface of the denoiser's tensor-core kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sde {

// Activation layout of the denoiser ("padded channel-group-major"): a BF16 tensor of C
// channels on a D x H x W grid is stored as [n][C/8][D+2][H+2][W+2][8], i.e. per group of
// eight channels a zero-padded volume whose voxels hold 16 bytes.  The one-voxel border is
// the convolutions' zero padding: it is zeroed when the buffer is created and no kernel
// writes it.  In this layout the rows y0-1 .. y0+Ty of one padded plane of one channel
// group are a single contiguous run of (Ty+2)(W+2) x 16 bytes, which one bulk copy moves
// into exactly the shared-memory image the tensor core reads.
struct Pcg {
    int D, H, W;
    __host__ __device__ size_t vp() const { return (size_t)(D + 2) * (H + 2) * (W + 2); }
    // 16-byte unit of voxel (z, y, x) (interior coordinates, -1 .. D etc. reach the border)
    // of channel group g of sample n, in a tensor of G groups
    __host__ __device__ size_t unit(int n, int G, int g, int z, int y, int x) const {
        return ((((size_t)n * G + g) * (D + 2) + (z + 1)) * (H + 2) + (y + 1)) * (W + 2) + (x + 1);
    }
};

// 3x3x3 convolution as an implicit GEMM (see sde_denoise.cu).  x is padded
// channel-group-major with Cin channels; the BF16 output is padded channel-group-major
// with y_cstride channels (written from channel y_coffset on), the FP32 output plain
// channels-last [n][D H W][y_cstride].  wpk holds the weights packed for the tensor core
// with wpk_cp output channels per part (conv_pack_weights; the plan's Cp must match).
struct ConvArgs {
    const __nv_bfloat16* x;
    const __nv_bfloat16* wpk;
    int wpk_cp;
    const float* bias;
    void* y;
    int D, H, W, Cin, Cout;
    int nvox;  // D*H*W
    int y_cstride, y_coffset, y_fp32, relu;
    int y_keep;   // FP32 output only: > 0 stores just output channels 0 .. y_keep-1 (<= 16), dense [n][D H W][y_keep]
    // BF16 output only, optional: also store every output voxel to its eight children in a padded
    // channel-group-major tensor on the grid 2D x 2H x 2W (nearest-neighbour upsampling), at
    // channel y_up_coffset of y_up_cstride
    void* y_up;
    int y_up_cstride, y_up_coffset;
    float slope;  // with relu: y = x > 0 ? x : slope * x (0: ReLU, > 0: leaky ReLU)
    unsigned int* status;
};

// Work decomposition and shared-memory layout of the pipelined brick convolution
// (host-chosen per layer shape).  A work item is (sample, Cout part, row block, z plane).
struct BrickPlan {
    int Ty;       // output rows (y) per work item, all x of one z plane (the last block may pass H)
    int tiles;    // M tiles of 128 positions per work item
    int rowtile;  // 1: W is a multiple of 128 and each tile is 128 x of one output row
    int fold;     // 1 (row tiles only): the three x taps of a (z, y) tap pair in one MMA of N = 3 Cp
    int nyb;      // ceil(H / Ty)
    int P;        // W + 2: brick row pitch in positions
    int Yb;       // Ty + 2: brick rows per plane
    int Cp;       // output channels per work item
    int nsplit;   // Cout / Cp
    int plane;    // bytes between the two 8-channel planes of a 16-channel chunk
    int w_off;    // offset of the chunk's weights (27 taps x Cp x 16) within a stage (wres = 0)
    int wres;     // 1: all chunks' weights stay resident after the stages (loaded once per CTA)
    int stage;    // bytes per pipeline stage (brick chunk + weight chunk)
    int nacc;     // tensor-memory accumulators (2: epilogue overlaps the next item)
    int xch;      // fold: offset of the epilogue's boundary-exchange buffer in shared memory
    int tcols;    // tensor-memory columns allocated (power of two >= nacc x tiles x Cp x (fold ? 3 : 1))
    int items;    // batch x nsplit x nyb x D
};

// Weight gradient of the convolution; x and dy padded channel-group-major.
struct WgradArgs {
    const __nv_bfloat16* x;   // Cin channels
    const __nv_bfloat16* dy;  // Cout channels
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

// Output channels per part that conv3d_launch will use for this layer shape (the packing
// of its weights), or 0 if the shape has no plan.
int conv_plan_cp(int D, int H, int W, int Cin, int Cout);
// wpk = w [Cout][27][Cin] in the tensor core's shared-memory image:
// [Cout/Cp][Cin/16][27][Cp x 16 K-major core matrices].
cudaError_t conv_pack_weights(const __nv_bfloat16* w, __nv_bfloat16* wpk, int Cin, int Cout, int Cp, cudaStream_t st);
cudaError_t conv3d_launch(const ConvArgs& a, int batch, cudaStream_t st);
cudaError_t wgrad_launch(const WgradArgs& a, cudaStream_t st);
cudaError_t flip_weights_launch(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout, cudaStream_t st);
cudaError_t denoise_status_word(unsigned int** out);
int denoise_check_status(cudaStream_t st);

}  // namespace sde
