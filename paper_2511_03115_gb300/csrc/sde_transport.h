// sde_transport.h -- host launchers of the transport kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sde_internal.cuh"

namespace sde {

constexpr int kMaxWarpsPerBlock = 8;  // the transport kernel is compiled for <= 256 threads

cudaError_t launch_transport(const KParams& P, int grid, int block, size_t smem_table, bool use_smem,
                             cudaStream_t st);
int transport_max_blocks_per_sm(int block, size_t smem, bool use_smem, int tally_mode, bool aggregate,
                                bool cut = false, int branch = 0);
cudaError_t launch_branch_chunk(unsigned long long* counters, unsigned long long* sec_ctl,
                                unsigned long long h_begin, cudaStream_t st);
// Spot records -> device form (positions in voxel units of voxel size h) and the history
// prefix; sets the work-queue cursor to h_begin.
cudaError_t launch_prep(const sde_spot* raw, int n, SpotDev* out, unsigned long long* prefix,
                        unsigned long long* counters, unsigned int* err, const double o[3], const double h[3],
                        double e_min, double e_lim, cudaStream_t st, unsigned long long h_begin = 0);
cudaError_t launch_probe(const KParams& P, int m, float rho, float E0, uint64_t h0, int n, float* Eo,
                         float* co, int* jo, float* uxo, float* uyo, cudaStream_t st);
cudaError_t launch_sum_u64(const unsigned long long* v, size_t n, unsigned long long* out, int num_sms,
                           cudaStream_t st);
cudaError_t launch_convert(const unsigned long long* edep, const float* rho, size_t nv, double unit_J,
                           double vol_kg_per_rho, double* dose, int num_sms, cudaStream_t st);
cudaError_t launch_convert_f32(const unsigned long long* edep, const float* rho, size_t nv, double unit_J,
                               double vol_kg_per_rho, float* dose, int num_sms, cudaStream_t st);

}  // namespace sde
