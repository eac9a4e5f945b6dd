"""Single-step and whole-track pins of the oracle's Euler-Maruyama scheme (Eq. VSDE).

The single-step statistics are compared with what the scheme fixes in closed form: the
mean continuous loss is varsigma_1 Delta exactly (the clamp is symmetric), the variance
is that of a Gaussian clamped at +-varsigma_1 Delta, the spherical Brownian increment has
E[Omega' . Omega] = exp(-t), and a jump happens with probability 1 - exp(-Delta sigma).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from sde_workloads import WATER, BONE, water100

N = 400_000


def _clamped_gauss_var(s, c):
    a = c / s
    return s * s * ((2 * stats.norm.cdf(a) - 1) - 2 * a * stats.norm.pdf(a)) + 2 * c * c * stats.norm.sf(a)


@pytest.mark.parametrize("E,step", [(100.0, 0.05), (200.0, 0.0005), (30.0, 0.05)])
def test_energy_step_mean_and_variance(oracle_lib, E, step):
    ph = O.physics(WATER, 1.0, E, step_cm=step)
    out = O.single_step(WATER, 1.0, E, N, seed=11, physics_mask=O.PHYS_STRAGGLING, step_cm=step)
    loss = E - out["E"]
    assert np.all(loss >= 0.0)
    c = ph.s1 * step
    s = math.sqrt(ph.s2sq * step)
    se = loss.std() / math.sqrt(N)
    assert abs(loss.mean() - c) < 3.5 * se
    var = _clamped_gauss_var(s, c)
    dev = loss - c
    se_var = math.sqrt((np.mean(dev ** 4) - var ** 2) / N)
    assert abs(dev.var() - var) < 3.5 * se_var
    assert np.all(loss <= 2 * c * (1 + 1e-12))


@pytest.mark.parametrize("E", [15.0, 100.0])
def test_sbm_increment_cosine_and_tangent_variance(oracle_lib, E):
    t = O.physics(WATER, 1.0, E).t_sbm
    out = O.single_step(WATER, 1.0, E, N, seed=3, physics_mask=O.PHYS_MCS)
    cosv = out["cos"]
    se = cosv.std() / math.sqrt(N)
    # exact spherical BM: E[cos] = e^-t; the small-time sampler is off by t^2/6
    assert abs(cosv.mean() - math.exp(-t)) < 3.5 * se + t * t / 6
    for comp in ("ux", "uy"):
        x2 = out[comp] ** 2
        assert abs(x2.mean() - t) < 3.5 * x2.std() / math.sqrt(N) + t * t
    # the azimuth is uniform: the tangent components are uncorrelated with equal variance
    assert abs(np.mean(out["ux"] * out["uy"])) < 4 * t / math.sqrt(N)


@pytest.mark.parametrize("clock", [0, 1])
@pytest.mark.parametrize("E", [5.0, 20.0])
def test_jump_probability(oracle_lib, clock, E):
    mask = O.PHYS_ELASTIC | O.PHYS_INELASTIC
    ph = O.physics(BONE, 1.85, E, physics_mask=mask)
    p = -math.expm1(-0.05 * (ph.sig_e + ph.sig_ne))
    out = O.single_step(BONE, 1.85, E, N, seed=5, physics_mask=mask, jump_clock=clock)
    j = out["jump"]
    frac = np.mean(j > 0)
    assert abs(frac - p) < 3.5 * math.sqrt(p * (1 - p) / N)
    q = ph.sig_ne / (ph.sig_e + ph.sig_ne)
    k = np.sum(j > 0)
    assert abs(np.mean(j[j > 0] == 2) - q) < 3.5 * math.sqrt(q * (1 - q) / k) + 1e-12


def test_inelastic_energy_fraction_law(oracle_lib):
    """u ~ U(u_lo, u_hi) multiplies the post-loss energy by (1 - u) (Eq. VSDE)."""
    mask = O.PHYS_INELASTIC
    E = 150.0
    ph = O.physics(WATER, 1.0, E, physics_mask=mask)
    out = O.single_step(WATER, 1.0, E, 200_000, seed=9, physics_mask=mask, inel_u_lo=0.2,
                        inel_u_hi=0.6, step_cm=5.0)
    j = out["jump"] == 2
    E1 = E - ph.s1 * 5.0
    u = 1.0 - out["E"][j] / E1
    assert u.min() >= 0.2 - 1e-12 and u.max() <= 0.6 + 1e-12
    assert stats.kstest(u, stats.uniform(0.2, 0.4).cdf).pvalue > 1e-3


def test_energy_never_increases_and_step_is_deterministic_without_noise(oracle_lib):
    out = O.single_step(WATER, 1.0, 80.0, 1000, seed=1, physics_mask=0)
    ph = O.physics(WATER, 1.0, 80.0)
    assert np.all(out["E"] == out["E"][0])
    assert out["E"][0] == pytest.approx(80.0 - ph.s1 * 0.05, rel=1e-15)
    assert np.all(out["cos"] == 1.0)


@pytest.mark.parametrize("E0", [100.0, 150.0])
def test_deterministic_track_range_converges_to_csda(oracle_lib, E0):
    """With straggling, scattering and jumps off, the Euler track's length exceeds the CSDA
    range by the scheme's first-order bias, about (Delta/2) ln(varsigma_1(e_min)/varsigma_1(E0))
    (the explicit step under-estimates the loss while the stopping power rises), give or take
    one step for the discrete end."""
    R = O.csda_range(WATER, 1.0, E0)
    c = 0.5 * math.log(O.physics(WATER, 1.0, 0.05).s1 / O.physics(WATER, 1.0, E0).s1)
    wl = water100(1)
    wl.spots["E_MeV"] = E0
    wl = wl.__class__(wl.name, (40, 40, 200), wl.voxel_mm, wl.origin_mm,
                      np.ones((200, 40, 40), np.float32), np.zeros((200, 40, 40), np.uint8),
                      wl.materials, wl.spots)
    errs = []
    for D in (0.05, 0.025, 0.0125, 0.00625):
        _, _, b = O.run_workload(wl, physics_mask=0, step_cm=D)
        e = b["steps"] * D - R
        assert abs(e / D - c) <= 1.0, (D, e / D, c)
        errs.append(e)
    assert errs[-1] < errs[0] / 4


def test_survival_against_nonelastic_removal(oracle_lib):
    """With only non-elastic jumps on and u = 1 (an event ends the track), the fraction of
    tracks with an event is 1 - exp(-sum_n Delta sigma_ne(E_n)) along the deterministic
    Euler energy sequence (Bernoulli clock of Eq. VSDE, step by step)."""
    E = 160.0
    Es = []
    while E >= 0.05:
        Es.append(E)
        E = O.single_step(WATER, 1.0, E, 1, physics_mask=0)["E"][0]
    tau = sum(0.05 * O.physics(WATER, 1.0, e, physics_mask=O.PHYS_INELASTIC).sig_ne for e in Es)
    p = -math.expm1(-tau)
    n = 40_000
    wl = water100(n)
    wl.spots["E_MeV"] = 160.0
    wl = wl.__class__(wl.name, (40, 40, 200), wl.voxel_mm, wl.origin_mm,
                      np.ones((200, 40, 40), np.float32), np.zeros((200, 40, 40), np.uint8),
                      wl.materials, wl.spots)
    _, _, b = O.run_workload(wl, physics_mask=O.PHYS_INELASTIC, inel_u_lo=1.0, inel_u_hi=1.0)
    frac = b["jumps_inelastic"] / n
    assert abs(frac - p) < 3.5 * math.sqrt(p * (1 - p) / n), (frac, p)


OXYGEN = {"name": "oxygen", "elements": [(8, 1.0)], "I_eV": 0.0}


@pytest.mark.parametrize("mat,rho", [(WATER, 1.0), (BONE, 1.85), (WATER, 0.26)])
@pytest.mark.parametrize("E", [1.0, 10.0, 100.0])
def test_energy_dependent_cut_off_is_the_fixed_law_at_that_angle(oracle_lib, mat, rho, E):
    """Sec. 2.1.3 cut-off 2.5 sigma(E): the rates with theta_cut_sigmas = 2.5 equal those of
    the fixed-cut law evaluated at the angle the mode chose, element by element."""
    a = O.physics(mat, rho, E, theta_cut_sigmas=2.5)
    b = O.physics(mat, rho, E, theta_cut_rad=a.theta_cut)
    assert 1e-4 <= a.theta_cut <= 1.0
    assert a.sig_e == b.sig_e and a.sig_ne == b.sig_ne
    assert list(a.sig_e_el) == list(b.sig_e_el)


def test_cut_off_scales_with_sigma_and_rutherford_rate_with_its_inverse_square(oracle_lib):
    """Doubling k doubles theta_c; the Rutherford rate of a hydrogen-free material,
    proportional to 1/(1 - cos theta_c) - 1/2 ~ 2/theta_c^2, falls by a factor of 4."""
    a = O.physics(OXYGEN, 1.0, 100.0, theta_cut_sigmas=2.5)
    b = O.physics(OXYGEN, 1.0, 100.0, theta_cut_sigmas=5.0)
    assert b.theta_cut == pytest.approx(2.0 * a.theta_cut, rel=1e-14)
    assert a.sig_e / b.sig_e == pytest.approx(4.0, rel=2e-5)
    # the cut-off falls with energy (sigma ~ 1/(p beta)) and widens in denser media
    assert O.physics(WATER, 1.0, 150.0, theta_cut_sigmas=2.5).theta_cut < a.theta_cut * 1.2
    assert O.physics(WATER, 1.0, 30.0, theta_cut_sigmas=2.5).theta_cut > \
        O.physics(WATER, 1.0, 100.0, theta_cut_sigmas=2.5).theta_cut
    assert O.physics(BONE, 1.85, 100.0, theta_cut_sigmas=2.5).theta_cut > \
        O.physics(BONE, 1.0, 100.0, theta_cut_sigmas=2.5).theta_cut


def test_cut_off_clamps(oracle_lib):
    assert O.physics(WATER, 1.0, 0.06, theta_cut_sigmas=2.5).theta_cut == 1.0
    vac = O.physics(WATER, 0.0, 50.0, theta_cut_sigmas=2.5)
    assert vac.theta_cut == 1e-4 and vac.sig_e == 0.0 and vac.sig_ne == 0.0


def test_jumps_with_the_energy_dependent_cut_off(oracle_lib):
    """Single steps at 100 MeV with only large-angle elastic and non-elastic events:
    the jump probability is 1 - exp(-Delta sigma) at the mode's rates, and elastic
    deflections on oxygen start at the cut-off (the lab angle of a small CM angle is
    about A/(A+1) = 0.94 of it; the fixed cut-off would put them near 0.019 rad)."""
    mask = O.PHYS_ELASTIC | O.PHYS_INELASTIC
    for mat in (BONE, OXYGEN):
        ph = O.physics(mat, 1.0, 100.0, physics_mask=mask, theta_cut_sigmas=2.5)
        p = -math.expm1(-0.05 * (ph.sig_e + ph.sig_ne))
        out = O.single_step(mat, 1.0, 100.0, N, seed=9, physics_mask=mask, jump_clock=1, theta_cut_sigmas=2.5)
        frac = np.mean(out["jump"] > 0)
        assert abs(frac - p) < 3.5 * math.sqrt(p * (1 - p) / N)
        if mat is OXYGEN:
            el = out["jump"] == 1
            assert el.sum() > 100
            smallest = np.arccos(out["cos"][el].max())
            assert 0.9 * ph.theta_cut <= smallest <= ph.theta_cut
