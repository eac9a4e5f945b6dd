/*
 * sde_oracle.h -- plain FP64 CPU oracle of the jump-SDE proton transport
 * (Dean, Perez-Lara, Horton, Southerby, Koskela, Kyprianou, "SDE-based Monte
 * Carlo dose calculation for proton therapy validated against Geant4",
 * arXiv 2511.03115).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it
 * is slow on purpose (formulas evaluated directly every step, no tables).
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header or constant with the CUDA library.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or garbled the reading taken is stated beside the code.
 *
 * Parity status of each part (what pins it) is listed in the file header of
 * sde_oracle.c.
 */
#ifndef SDE_ORACLE_H
#define SDE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORACLE_OK = 0,
    ORACLE_EINVAL = -1,
    ORACLE_ENOMEM = -2,
    ORACLE_ESTEPCAP = -5
};

/* physics_mask bits: a set bit turns the term ON. */
enum {
    ORACLE_PHYS_STRAGGLING = 1, /* clamped Gaussian term of Eq. VSDE (energy line) */
    ORACLE_PHYS_MCS = 2,        /* spherical Brownian increment Xi_n           */
    ORACLE_PHYS_ELASTIC = 4,    /* large-angle elastic jumps (sigma_e, pi_e)    */
    ORACLE_PHYS_INELASTIC = 8,  /* non-elastic jumps (sigma_ne, pi_ne)          */
    ORACLE_PHYS_ALL = 15
};

typedef struct {
    int Z;
    double mass_fraction;
} oracle_element_frac;

typedef struct {
    const oracle_element_frac* el;
    int n_el;
    double I_eV; /* <= 0: Bragg-additive ln I from the element table */
} oracle_material;

typedef struct {
    double E_MeV, sigma_E_MeV;
    double x_mm, y_mm, z_mm;
    double ux, uy, uz;
    double sigma_xy_mm, sigma_angle_rad;
    uint64_t n_hist;
} oracle_spot;

typedef struct {
    double step_cm;          /* Delta, Euler-Maruyama increment (Sec. 3.1.3: 0.5 mm) */
    double msc_z_cm;         /* z of the Lynch-Dahl width and m = sigma/sqrt(z) (0.05 cm) */
    double F;                /* Lynch-Dahl central fraction (0.98) */
    double theta_cut_rad;    /* large-angle elastic cut-off, CM (0.02 rad) */
    double backscatter_rad;  /* hydrogen backscatter limit (0.04 rad) */
    double e_min_MeV;        /* absorption energy (0.05 MeV) */
    double K;                /* Bethe prefactor, Eq. bethbloch (0.3072) */
    double inel_u_lo;        /* surrogate pi_ne: u ~ U(inel_u_lo, inel_u_hi) */
    double inel_u_hi;
    double km_r;             /* surrogate Kalbach-Mann pre-equilibrium fraction r */
    int tally_mode;          /* 0: deposit at the step midpoint; 1: split along the chord */
    int fixed_point_shift;   /* S: one tally unit is 2^-S MeV (24) */
    int jump_clock;          /* 0: one Bernoulli draw per step (paper); 1: exponential clock */
    int max_steps;           /* step cap per history */
    int physics_mask;        /* ORACLE_PHYS_* */
    double theta_cut_sigmas; /* 0: fixed theta_cut_rad; k > 0: energy-dependent cut-off
                                theta_c = k sigma(E) (Sec. 2.1.3, k = 2.5), clamped to
                                [1e-4, 1] rad */
    double secondary_fraction; /* 0: the paper's single-proton model.  kappa in (0, 1]:
                                  branching SDE (Sec. 2.1.1, the extension the paper leaves
                                  to future work): each non-elastic event of a primary also
                                  emits a secondary proton carrying kappa u E' of the energy
                                  deficit u E', transported by the same SDE */
} oracle_params;

typedef struct {
    uint64_t incident, deposited, escaped, removed;
    uint64_t histories, steps, jumps_elastic, jumps_inelastic;
} oracle_balance;

/* Per-material physics at one energy and density (Secs. 2.1.3-2.1.5). */
#define ORACLE_MAX_EL 16
typedef struct {
    double beta2, gamma, p_MeV;
    double I_eV;
    double s1;            /* varsigma_1, MeV/cm                       */
    double s2sq;          /* varsigma_2^2, MeV^2/cm                   */
    double chi_c2;        /* compound chi_c^2 over path z             */
    double chi_a2;        /* compound chi_alpha^2                     */
    double w;             /* Lynch-Dahl w                             */
    double sigma_msc;     /* sigma(E), rad                            */
    double t_sbm;         /* m^2 Delta = sigma^2 Delta / z            */
    double sig_e;         /* total large-angle elastic rate, 1/cm     */
    double sig_ne;        /* total non-elastic rate, 1/cm             */
    double theta_cut;     /* large-angle cut-off used, CM, rad        */
    int n_el;
    double sig_e_el[ORACLE_MAX_EL];
    double sig_ne_el[ORACLE_MAX_EL];
} oracle_physics_out;

typedef struct oracle_dose oracle_dose;

void oracle_default_params(oracle_params* p);
const char* oracle_last_error(void);
int oracle_set_threads(int n);

int oracle_create(oracle_dose** out, int nx, int ny, int nz, const double voxel_mm[3],
                  const double origin_mm[3], const float* density_g_cm3,
                  const uint8_t* material_id, const oracle_material* mats, int n_mats,
                  const oracle_params* p);
int oracle_run(oracle_dose* d, const oracle_spot* spots, int n_spots, uint64_t seed);
/* As oracle_run for the histories with global ids in [first, first + count) of the plan
 * only (ids run over the spots in order); disjoint ranges with one seed add up to the
 * whole run exactly. */
int oracle_run_range(oracle_dose* d, const oracle_spot* spots, int n_spots, uint64_t seed, uint64_t first,
                     uint64_t count);
int oracle_fetch(oracle_dose* d, double* dose_Gy, uint64_t* edep_fixed, oracle_balance* bal);
int oracle_reset(oracle_dose* d);
void oracle_destroy(oracle_dose* d);

/* ---- probes used by the pin tests ---- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int oracle_element(int Z, double* A, double* I_eV);
int oracle_physics(const oracle_material* m, double rho, const oracle_params* p, double E,
                   oracle_physics_out* out);
/* CSDA range (cm) at density rho: integral of dE / varsigma_1 from e_min to E0. */
int oracle_csda_range(const oracle_material* m, double rho, const oracle_params* p, double E0,
                      double* range_cm);
/* One Euler-Maruyama step in an unbounded homogeneous medium, for n independent
 * histories h = h0 .. h0+n-1 at step index 0, all starting at energy E along +z.
 * Outputs (any may be NULL): E_out (post-step energy, after any inelastic loss),
 * cos_out (Omega_{n+1} . Omega_n), jump_out (0 none, 1 elastic, 2 inelastic),
 * ux_out/uy_out (components of Omega_{n+1}). */
int oracle_single_step(const oracle_material* m, double rho, const oracle_params* p, double E,
                       uint64_t seed, uint64_t h0, int n, double* E_out, double* cos_out,
                       int* jump_out, double* ux_out, double* uy_out);
/* As oracle_single_step, with what the branching model emits: per history 10 values
 * (jump kind, E1 = energy after the continuous loss, energy after the event, spawned
 * (0/1), secondary energy, secondary direction x/y/z, continuing direction x/y). */
int oracle_single_step_secondary(const oracle_material* m, double rho, const oracle_params* p, double E,
                                 uint64_t seed, uint64_t h0, int n, double* out);
/* Y_0 of histories h = h0 .. h0+n-1 of one spot (the source sampling of a run): energy,
 * entry point (mm, 3 per history) and direction (3 per history); any output may be NULL. */
int oracle_sample_source(const oracle_spot* s, const oracle_params* p, uint64_t seed, uint64_t h0, int n,
                         double* E_out, double* r_out, double* u_out);
/* Samplers of the large-angle laws (U in (0,1)): CM cosine. */
double oracle_sample_mu_rutherford(double U, double mu_c);
double oracle_sample_mu_mott(double U, double eta, double mu_lo, double mu_c);
double oracle_mott_antiderivative(double mu, double eta);
double oracle_mott_dsigma(double mu, double eta, double k_fm);
double oracle_rutherford_dsigma(double mu, double eta, double k_fm);
double oracle_sample_mu_kalbach(double U, double a, double r);
double oracle_kalbach_a(double E, double u, double A);
double oracle_cm_to_lab(double E_in, double E_out, double m2, double cos_cm);
/* eta and k (fm^-1) of the two-body Coulomb problem for element Z at lab energy E. */
int oracle_coulomb_eta_k(int Z, double E, double* eta, double* k_fm);
double oracle_sigma_ne_element_mb(int Z, double E);

#ifdef __cplusplus
}
#endif
#endif
