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

// Weight gradient: dw[co][tap][ci] += sum_v dy[v][co] x[v + off(tap)][ci].  One CTA per
// (tap, voxel chunk); the GEMM has rows = co (padded to 128), columns = ci, K = voxels,
// with both operands M/N-major (channels contiguous, as stored).
struct WgradArgs {
    const __nv_bfloat16* x;   // [n][V][Cin]
    const __nv_bfloat16* dy;  // [n][V][Cout]
    float* dw;                // [Cout][27][Cin], accumulated
    int D, H, W, Cin, Cout, nvox, batch, chunk;
    unsigned int* status;
};

cudaError_t conv3d_launch(const ConvArgs& a, int batch, cudaStream_t st);
cudaError_t wgrad_launch(const WgradArgs& a, cudaStream_t st);
cudaError_t flip_weights_launch(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout, cudaStream_t st);
cudaError_t denoise_status_word(unsigned int** out);
int denoise_check_status(cudaStream_t st);

}  // namespace sde
