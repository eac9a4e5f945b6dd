// sde_tables.h -- host interface of the physics-table builder.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sde_dose.h"

namespace sde {

// A material resolved against the element table (host and device copy).
struct MatHost {
    int n_el;
    int Z[SDE_MAX_ELEMENTS];
    double A[SDE_MAX_ELEMENTS];
    double w[SDE_MAX_ELEMENTS];  // renormalised mass fractions
    double I_eV_el[SDE_MAX_ELEMENTS];
    double I_eV;  // of the medium (given or Bragg-additive)
};

bool element_row(int Z, double* A, double* I_eV);
int resolve_material(const sde_material& m, MatHost* out, char* err, size_t errlen);

struct TableBuild {
    int N, n_mats;
    double e_min, e_max, K, F, z, step, theta_cut, theta_back;
    int mask;
    const MatHost* d_mats;
    float* d_raw;
    float* d_jrates;
    double* d_csda;
    float4* d_table;
    float4* d_cut = nullptr;  // optional [n_mats][N][2]: Coulomb coefficients (variable cut-off)
    float2* d_pick = nullptr;  // optional [n_mats][N][2*SDE_MAX_ELEMENTS]: cumulative rates for the event pick
    float4* d_mott_g = nullptr;  // optional [N]: hydrogen primitive at the cut-off and backscatter limits
    float2* d_mott_r = nullptr;  // optional [N][kMottKnots]: hydrogen inversion ratios (fixed cut-off)
};

cudaError_t build_tables(const TableBuild& tb, cudaStream_t st);
// log2 of the first knot of the hydrogen inversion table: log2(1 - cos theta_cut).
double mott_knot_lo(double theta_cut);

// Message for sde_last_error() (defined with the C ABI).
void set_last_error(const char* msg);

}  // namespace sde
