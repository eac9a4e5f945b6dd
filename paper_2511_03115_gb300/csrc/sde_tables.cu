// sde_tables.cu -- physics-table builder of the jump-SDE proton engine.
//
// For every material and every point E_k of a ln-uniform energy grid the
// functionals of arXiv 2511.03115 are evaluated in FP64 on the device and
// stored as FP32:
//   varsigma_1   Bethe stopping with Bragg additivity, Eq. BraggAditivty
//   varsigma_2^2 relativistic Bohr straggling, Eq. energystraggling
//   chi_c^2, chi_alpha^2 -> Lynch-Dahl width sigma(E) and m = sigma/sqrt(z)
//                (Sec. 2.1.4, compound rules as stated there)
//   sigma_e      large-angle elastic rate per element: CM Rutherford (Z>1),
//                Mott identical-particle term (H), Eqs. large_elastic_cm(_hydrogen)
//   sigma_ne     non-elastic rate per element (Sec. 2.1.5)
// plus the CSDA range R(E) = int dE / varsigma_1 by Gauss-Legendre quadrature.
// Rates and stopping are stored per unit density so that one table serves
// every voxel density of a material.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "sde_internal.cuh"
#include "sde_tables.h"

namespace sde {

// Standard atomic weights (IUPAC) and mean excitation energies (eV): ICRU
// Report 37 values for H, C, N, O, F, Cl bound in condensed compounds, the
// elemental ICRU 37 values otherwise (used for Bragg-additive ln I).
struct ElementRow {
    int Z;
    double A, I;
};
static const ElementRow kElements[] = {
    {1, 1.008, 19.2},        {2, 4.002602, 41.8},     {6, 12.011, 81.0},       {7, 14.007, 82.0},
    {8, 15.999, 106.0},      {9, 18.998403, 112.0},   {11, 22.989769, 149.0},  {12, 24.305, 156.0},
    {13, 26.981538, 166.0},  {14, 28.085, 173.0},     {15, 30.973762, 173.0},  {16, 32.06, 180.0},
    {17, 35.45, 180.0},      {18, 39.948, 188.0},     {19, 39.0983, 190.0},    {20, 40.078, 191.0},
    {22, 47.867, 233.0},     {26, 55.845, 286.0},     {29, 63.546, 322.0},     {30, 65.38, 330.0},
};

bool element_row(int Z, double* A, double* I_eV) {
    for (const ElementRow& e : kElements)
        if (e.Z == Z) {
            *A = e.A;
            *I_eV = e.I;
            return true;
        }
    return false;
}

int resolve_material(const sde_material& m, MatHost* out, char* err, size_t errlen) {
    if (!m.el || m.n_el < 1 || m.n_el > SDE_MAX_ELEMENTS) {
        snprintf(err, errlen, "material needs 1..%d elements", SDE_MAX_ELEMENTS);
        return SDE_EINVAL;
    }
    memset(out, 0, sizeof *out);
    double total = 0.0;
    for (int i = 0; i < m.n_el; ++i) {
        double A, I;
        if (!element_row(m.el[i].Z, &A, &I)) {
            snprintf(err, errlen, "element Z=%d is not supported", m.el[i].Z);
            return SDE_EINVAL;
        }
        if (!(m.el[i].mass_fraction > 0.0) || !isfinite(m.el[i].mass_fraction)) {
            snprintf(err, errlen, "mass fraction of Z=%d must be > 0", m.el[i].Z);
            return SDE_EINVAL;
        }
        out->Z[i] = m.el[i].Z;
        out->A[i] = A;
        out->I_eV_el[i] = I;
        out->w[i] = m.el[i].mass_fraction;
        total += m.el[i].mass_fraction;
    }
    out->n_el = m.n_el;
    double zsum = 0.0, lsum = 0.0;
    for (int i = 0; i < out->n_el; ++i) {
        out->w[i] /= total;
        double ne = out->w[i] * out->Z[i] / out->A[i];  // electrons per gram / N_A
        zsum += ne;
        lsum += ne * log(out->I_eV_el[i]);
    }
    out->I_eV = m.I_eV > 0.0 ? m.I_eV : exp(lsum / zsum);
    return SDE_OK;
}

// ------------------------------------------------------------ device physics
struct Kin {
    double beta2, gamma2, p2, pbeta;
};

__device__ __forceinline__ Kin kin_of(double E) {
    Kin k;
    double tot = E + kProtonMass;
    k.p2 = E * (E + 2.0 * kProtonMass);
    k.beta2 = k.p2 / (tot * tot);
    k.gamma2 = tot * tot / (kProtonMass * kProtonMass);
    k.pbeta = k.p2 / tot;
    return k;
}

// Letaw-Silberberg-Tsao (1983) non-elastic cross section in mb with a
// classical Coulomb-barrier factor; zero for hydrogen (no p-p non-elastic
// channel at these energies).  Stand-in for the unavailable ENDF tables.
__device__ double nonelastic_mb(int Z, double A, double E) {
    if (Z == 1) return 0.0;
    double high = 45.0 * pow(A, 0.7) * (1.0 + 0.016 * sin(5.3 - 2.63 * log(A)));
    double shape = 1.0 - 0.62 * exp(-E / 200.0) * sin(10.9 * pow(E, -0.28));
    double m2 = A * kAtomicMassUnit;
    double e_cm = E * m2 / (kProtonMass + m2);
    double barrier = Z * kFineStructure * kHbarcMeVfm / (1.3 * (cbrt(A) + 1.0));
    return e_cm > barrier ? high * shape * (1.0 - barrier / e_cm) : 0.0;
}

// Identical-particle Coulomb antiderivative in units of (eta/k)^2:
// int 2(1+x^2)/(1-x^2)^2 - cos(eta ln((1+x)/(1-x)))/(1-x^2) dx.
__device__ double mott_primitive(double x, double eta) {
    double L = log1p(x) - log1p(-x);
    return 2.0 * x / ((1.0 - x) * (1.0 + x)) - sin(eta * L) / (2.0 * eta);
}

struct TableArgs {
    int N, n_mats;
    double lnEmin, dlnE;
    double K, F, z, step;
    double cos_cut, cos_back;
    int mask;
    const MatHost* mats;
    float* raw;     // [n_mats][N][kRawFields]
    float* jrates;  // [n_mats][N][2*SDE_MAX_ELEMENTS]: sigma_e E^2 / rho, then sigma_ne / rho
    double* csda;   // [n_mats][N]
    float4* table;  // [n_mats][N][kRowFloat4]
    float4* cut;    // [n_mats][N][2] or null
    float2* pick;   // [n_mats][N][2*SDE_MAX_ELEMENTS] cumulative rates {value, slope} or null
    float4* mott_g; // [N] or null
    float2* mott_r; // [N][kMottKnots] or null
    double mott_lg2_lo, mott_dj;
};

__device__ double stopping_per_rho(const MatHost& m, double K, double E) {
    Kin k = kin_of(E);
    double zA = 0.0;
    for (int i = 0; i < m.n_el; ++i) zA += m.w[i] * m.Z[i] / m.A[i];
    double I = m.I_eV * 1e-6;
    // beta^2 / (1 - beta^2) = beta^2 gamma^2
    return K * zA / k.beta2 * (log(2.0 * kElectronMass * k.beta2 * k.gamma2 / I) - k.beta2);
}

// All functionals of one material at one energy, per unit density, FP64.
struct Point {
    double s1;       // varsigma_1 / rho
    double s2;       // varsigma_2^2 / rho
    double chic;     // chi_c^2 / rho over the path z
    double chia;     // chi_alpha^2
    double cc;       // chi_c^2 (p beta)^2 / rho: a material constant
    double se[SDE_MAX_ELEMENTS], sne[SDE_MAX_ELEMENTS];
    double se_tot, sne_tot;
};

__device__ void physics_point(const TableArgs& a, const MatHost& m, double E, Point& o) {
    Kin k = kin_of(E);
    double zA = 0.0, zz = 0.0, lsum = 0.0;
    for (int i = 0; i < m.n_el; ++i) {
        double Z = m.Z[i];
        zA += m.w[i] * Z / m.A[i];
        double wz = m.w[i] * Z * (Z + 1.0) / m.A[i];
        zz += wz;
        double za = Z * kFineStructure;
        lsum += wz * log(2.007e-5 * pow(Z, 2.0 / 3.0) * (1.0 + 3.34 * za * za / k.beta2) / k.p2);
    }
    o.s1 = stopping_per_rho(m, a.K, E);
    double ahc = kFineStructure * kHbarcMeVfm * 1e-13;  // e^2 in MeV cm
    o.s2 = 4.0 * kPi * kAvogadro * ahc * ahc * zA * k.gamma2 * (1.0 - 0.5 * k.beta2);
    o.cc = 0.157 * zz * a.z;
    o.chic = o.cc / (k.pbeta * k.pbeta);
    o.chia = exp(lsum / zz);
    double vnr = sqrt(2.0 * E / kProtonMass);  // non-relativistic v/c (ENDF Coulomb terms)
    double s_cut = 1.0 - a.cos_cut;
    o.se_tot = 0.0;
    o.sne_tot = 0.0;
    for (int i = 0; i < SDE_MAX_ELEMENTS; ++i) {
        double el = 0.0, ne = 0.0;
        if (i < m.n_el) {
            double Z = m.Z[i];
            double m2 = m.Z[i] == 1 ? kProtonMass : m.A[i] * kAtomicMassUnit;
            double mu_red = kProtonMass * m2 / (kProtonMass + m2);
            double eta = Z * kFineStructure / vnr;
            double kwave = mu_red * vnr / kHbarcMeVfm;         // fm^-1
            double r2 = (eta / kwave) * (eta / kwave) * 1e-26;  // cm^2
            double atoms = kAvogadro * m.w[i] / m.A[i];         // per gram
            double ang;
            if (m.Z[i] == 1)
                ang = mott_primitive(a.cos_cut, eta) - mott_primitive(-a.cos_back, eta);
            else
                ang = 1.0 / s_cut - 0.5;
            if (a.mask & SDE_PHYS_ELASTIC) el = atoms * 2.0 * kPi * r2 * ang;
            if (a.mask & SDE_PHYS_INELASTIC) ne = atoms * nonelastic_mb(m.Z[i], m.A[i], E) * 1e-27;
        }
        o.se[i] = el;
        o.sne[i] = ne;
        o.se_tot += el;
        o.sne_tot += ne;
    }
}

__global__ void k_build_raw(TableArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * a.n_mats) return;
    int mi = idx / a.N, kk = idx % a.N;
    double E = exp(a.lnEmin + kk * a.dlnE);
    Point o;
    physics_point(a, a.mats[mi], E, o);
    float* jr = a.jrates + ((size_t)mi * a.N + kk) * (2 * SDE_MAX_ELEMENTS);
    for (int i = 0; i < SDE_MAX_ELEMENTS; ++i) {
        jr[i] = (float)(o.se[i] * E * E);  // ~flat in E: the Coulomb rates fall as 1/E^2
        jr[SDE_MAX_ELEMENTS + i] = (float)o.sne[i];
    }
    float* raw = a.raw + ((size_t)mi * a.N + kk) * kRawFields;
    raw[0] = (float)o.s1;
    raw[1] = (float)o.s2;
    raw[2] = (float)o.chic;
    raw[3] = (float)(1.0 / (2.0 * o.chia * (1.0 - a.F)));
    raw[4] = (float)(o.se_tot + o.sne_tot);
}

// Hot-row fields, chosen so that they are nearly linear in ln E; the kernel
// multiplies back the kinematic factors it computes from E:
//   f1 = varsigma_1 beta^2 Delta / rho        (x 1/beta^2)
//   f2 = sqrt(varsigma_2^2 Delta / rho)        (x sqrt(rho))
//   bt = 1 / (2 chi_alpha^2 (1-F) p^2)         (w = rho cw bt / beta^2)
//   fe = sigma_e E^2 Delta / rho               (x 1/E^2)
//   fn = sigma_ne Delta / rho
//   cw = chi_c^2 (p beta)^2 / rho, ct = cw Delta / (z (1+F^2))   (material constants)
__device__ void hot_values(const TableArgs& a, int mi, int kk, double v[7]) {
    double E = exp(a.lnEmin + kk * a.dlnE);
    Kin k = kin_of(E);
    Point o;
    physics_point(a, a.mats[mi], E, o);
    v[0] = o.s1 * k.beta2 * a.step;
    v[1] = sqrt(o.s2 * a.step);
    v[2] = 1.0 / (2.0 * o.chia * (1.0 - a.F) * k.p2);
    v[3] = o.se_tot * E * E * a.step;
    v[4] = o.sne_tot * a.step;
    v[5] = o.cc;
    v[6] = o.cc * a.step / (a.z * (1.0 + a.F * a.F));
}

__global__ void k_build_hot(TableArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * a.n_mats) return;
    int mi = idx / a.N, kk = idx % a.N;
    double v0[7], v1[7];
    hot_values(a, mi, kk, v0);
    if (kk + 1 < a.N)
        hot_values(a, mi, kk + 1, v1);
    else
        for (int i = 0; i < 7; ++i) v1[i] = v0[i];
    float4* row = a.table + ((size_t)mi * a.N + kk) * kRowFloat4;
    row[0] = make_float4((float)v0[0], (float)(v1[0] - v0[0]), (float)v0[1], (float)(v1[1] - v0[1]));
    row[1] = make_float4((float)v0[2], (float)(v1[2] - v0[2]), (float)v0[3], (float)(v1[3] - v0[3]));
    row[2] = make_float4((float)v0[4], (float)(v1[4] - v0[4]), (float)v0[5], (float)v0[6]);
}

// Rows for picking the channel and element of a large-angle event (fixed cut-off): at each
// grid point the cumulative elastic rates sum_{j<=i} sigma_e,j E^2 Delta / rho over the
// elements in order, then the cumulative non-elastic rates sum_{j<=i} sigma_ne,j Delta / rho,
// each as {value at E_k, difference to E_k+1} for linear interpolation in ln E.  Interpolated
// cumulative sums are the cumulative sums of interpolated rates, so the pick follows the
// same rule as summing the rates one by one: the first channel whose cumulative rate
// exceeds the uniform target.
__global__ void k_build_pick(TableArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * a.n_mats) return;
    int mi = idx / a.N, kk = idx % a.N;
    double c0[2 * SDE_MAX_ELEMENTS], c1[2 * SDE_MAX_ELEMENTS];
    for (int side = 0; side < 2; ++side) {
        const int kq = kk + side < a.N ? kk + side : kk;
        const double E = exp(a.lnEmin + kq * a.dlnE);
        Point o;
        physics_point(a, a.mats[mi], E, o);
        double* c = side ? c1 : c0;
        double ae = 0.0, an = 0.0;
        for (int i = 0; i < SDE_MAX_ELEMENTS; ++i) {
            ae += o.se[i] * E * E * a.step;
            an += o.sne[i] * a.step;
            c[i] = ae;
            c[SDE_MAX_ELEMENTS + i] = an;
        }
    }
    float2* row = a.pick + ((size_t)mi * a.N + kk) * (2 * SDE_MAX_ELEMENTS);
    for (int i = 0; i < 2 * SDE_MAX_ELEMENTS; ++i) row[i] = make_float2((float)c0[i], (float)(c1[i] - c0[i]));
}

// Hydrogen (identical-particle Coulomb) inversion for the fixed cut-off.  In the forward
// variable s = 1 - |mu| the primitive is G(s) = 2(1-s)/(s(2-s)) - sin(eta ln((2-s)/s))/(2 eta),
// decreasing from +inf to 0 on (0, 1]; without the sine term it is G0(s), whose inverse
// s0(y) is closed-form.  For each energy point and each knot s0_j (uniform in log2 from
// 1 - cos theta_cut to 1) the table holds rho = s / s0_j with G(s) = G0(s0_j), found by
// bisection in FP64; the kernel interpolates rho bilinearly and takes one Newton step.
// mott_g holds the primitive at the two ends of the sampled range per energy point.
__device__ double mott_G(double s, double eta) {
    return 2.0 * (1.0 - s) / (s * (2.0 - s)) - sin(eta * log((2.0 - s) / s)) / (2.0 * eta);
}

__device__ double mott_eta(double E) { return kFineStructure / sqrt(2.0 * E / kProtonMass); }

__global__ void k_build_mott(TableArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * kMottKnots) return;
    const int kk = idx / kMottKnots, j = idx % kMottKnots;
    const double eta = mott_eta(exp(a.lnEmin + kk * a.dlnE));
    double rho[2];
    for (int q = 0; q < 2; ++q) {
        const int jj = j + q < kMottKnots ? j + q : j;
        const double s0 = exp2(a.mott_lg2_lo + jj * a.mott_dj);
        const double y = 2.0 * (1.0 - s0) / (s0 * (2.0 - s0));
        double lo = log(1e-12), hi = 0.0;  // bisection in ln s
        for (int it = 0; it < 80; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mott_G(exp(mid), eta) > y)
                lo = mid;
            else
                hi = mid;
        }
        rho[q] = exp(0.5 * (lo + hi)) / s0;
    }
    a.mott_r[(size_t)kk * kMottKnots + j] = make_float2((float)rho[0], (float)rho[1]);
    if (j == 0) {
        double g[2][2];
        for (int q = 0; q < 2; ++q) {
            const double e2 = mott_eta(exp(a.lnEmin + (kk + q < a.N ? kk + q : kk) * a.dlnE));
            g[q][0] = mott_G(1.0 - a.cos_cut, e2);
            g[q][1] = -mott_G(1.0 - a.cos_back, e2);
        }
        a.mott_g[kk] = make_float4((float)g[0][0], (float)(g[1][0] - g[0][0]), (float)g[0][1],
                                   (float)(g[1][1] - g[0][1]));
    }
}

// Coefficients of the large-angle elastic rate with a variable cut-off, per unit density,
// times E^2 Delta (flat in E like fe): the Rutherford sum over elements other than
// hydrogen, R = sum n_i 2 pi (eta_i/k_i)^2, multiplies 1/(1 - mu_c) - 1/2; hydrogen's
// Hc = n_H 2 pi (eta/k)^2 multiplies the Mott primitive at mu_c, minus Hlo = Hc G(mu_lo)
// at the backscatter limit.  Row 0 {R, dR, Hc, dHc}, row 1 {Hlo, dHlo, 0, 0}.
__device__ void cut_values(const TableArgs& a, int mi, int kk, double v[3]) {
    const MatHost& m = a.mats[mi];
    double E = exp(a.lnEmin + kk * a.dlnE);
    double vnr = sqrt(2.0 * E / kProtonMass);
    v[0] = v[1] = v[2] = 0.0;
    if (!(a.mask & SDE_PHYS_ELASTIC)) return;
    for (int i = 0; i < m.n_el; ++i) {
        double m2 = m.Z[i] == 1 ? kProtonMass : m.A[i] * kAtomicMassUnit;
        double mu_red = kProtonMass * m2 / (kProtonMass + m2);
        double eta = m.Z[i] * kFineStructure / vnr;
        double kwave = mu_red * vnr / kHbarcMeVfm;
        double coef = kAvogadro * m.w[i] / m.A[i] * 2.0 * kPi * (eta / kwave) * (eta / kwave) * 1e-26 * E * E * a.step;
        if (m.Z[i] == 1) {
            v[1] += coef;
            v[2] += coef * mott_primitive(-a.cos_back, eta);
        } else {
            v[0] += coef;
        }
    }
}

__global__ void k_build_cut(TableArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * a.n_mats) return;
    int mi = idx / a.N, kk = idx % a.N;
    double v0[3], v1[3];
    cut_values(a, mi, kk, v0);
    if (kk + 1 < a.N)
        cut_values(a, mi, kk + 1, v1);
    else
        for (int i = 0; i < 3; ++i) v1[i] = v0[i];
    float4* row = a.cut + ((size_t)mi * a.N + kk) * 2;
    row[0] = make_float4((float)v0[0], (float)(v1[0] - v0[0]), (float)v0[1], (float)(v1[1] - v0[1]));
    row[1] = make_float4((float)v0[2], (float)(v1[2] - v0[2]), 0.f, 0.f);
}

// CSDA range at unit density: one block per material; thread j integrates
// [E_j, E_j+1] by 8-point Gauss-Legendre in ln E, then a serial prefix sum.
__global__ void k_csda(TableArgs a) {
    int mi = blockIdx.x;
    const MatHost& m = a.mats[mi];
    // Gauss-Legendre nodes and weights on [-1, 1], n = 8 (Abramowitz & Stegun 25.4)
    const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                         0.9602898564975363};
    const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                         0.1012285362903763};
    double* out = a.csda + (size_t)mi * a.N;
    for (int j = threadIdx.x; j < a.N - 1; j += blockDim.x) {
        double lo = a.lnEmin + j * a.dlnE, half = 0.5 * a.dlnE, mid = lo + half;
        double acc = 0.0;
        for (int q = 0; q < 4; ++q)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double E = exp(mid + sgn * half * x[q]);
                acc += w[q] * E / stopping_per_rho(m, a.K, E);
            }
        out[j + 1] = acc * half;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = 0.0;
        for (int j = 1; j < a.N; ++j) out[j] += out[j - 1];
    }
}

double mott_knot_lo(double theta_cut) { return log2(1.0 - cos(theta_cut)); }

cudaError_t build_tables(const TableBuild& tb, cudaStream_t st) {
    TableArgs a;
    a.N = tb.N;
    a.n_mats = tb.n_mats;
    a.lnEmin = log(tb.e_min);
    a.dlnE = (log(tb.e_max) - log(tb.e_min)) / (tb.N - 1);
    a.K = tb.K;
    a.F = tb.F;
    a.z = tb.z;
    a.step = tb.step;
    a.cos_cut = cos(tb.theta_cut);
    a.cos_back = cos(tb.theta_back);
    a.mask = tb.mask;
    a.mats = tb.d_mats;
    a.raw = tb.d_raw;
    a.jrates = tb.d_jrates;
    a.csda = tb.d_csda;
    a.table = tb.d_table;
    a.cut = tb.d_cut;
    a.pick = tb.d_pick;
    a.mott_g = tb.d_mott_g;
    a.mott_r = tb.d_mott_r;
    a.mott_lg2_lo = mott_knot_lo(tb.theta_cut);
    a.mott_dj = -a.mott_lg2_lo / (kMottKnots - 1);
    int total = tb.N * tb.n_mats;
    int threads = 128, blocks = (total + threads - 1) / threads;
    k_build_raw<<<blocks, threads, 0, st>>>(a);
    k_build_hot<<<blocks, threads, 0, st>>>(a);
    k_csda<<<tb.n_mats, 256, 0, st>>>(a);
    if (a.cut) k_build_cut<<<blocks, threads, 0, st>>>(a);
    if (a.pick) k_build_pick<<<blocks, threads, 0, st>>>(a);
    if (a.mott_g && a.mott_r) k_build_mott<<<(tb.N * kMottKnots + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sde
