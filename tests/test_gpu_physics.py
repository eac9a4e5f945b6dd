"""GPU physics against the oracle: the FP32 tables built on the device (FP64 evaluation)
at their grid points, and the transport kernel's step function (through the single-step
probe) on the same random streams as the oracle (its exponential jump clock)."""
import math

import numpy as np
import pytest

import oracle as O
from sde_workloads import BONE, TISSUE, WATER, Workload, pencil

pytestmark = pytest.mark.gpu


def _tiny(materials):
    n = len(materials)
    dens = np.ones((2, 2, 2), np.float32)
    mid = (np.arange(8) % n).astype(np.uint8).reshape(2, 2, 2)
    return Workload("tiny", (2, 2, 2), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), dens, mid, materials,
                    pencil(100.0, 1))


@pytest.mark.parametrize("mat_index", [0, 1, 2])
def test_tables_equal_the_oracle_at_grid_points(sde_gpu, oracle_lib, mat_index):
    mats = [WATER, BONE, TISSUE]
    with sde_gpu.SdeDose(_tiny(mats)) as d:
        t = d.tables(mat_index)
    mat = mats[mat_index]
    for k in range(0, len(t["E"]), 7):
        E = t["E"][k]
        ph = O.physics(mat, 1.0, E)
        assert t["s1"][k] == pytest.approx(ph.s1, rel=2e-6)
        assert t["s2sq"][k] == pytest.approx(ph.s2sq, rel=2e-6)
        assert t["chi_c2"][k] == pytest.approx(ph.chi_c2, rel=2e-6)
        assert t["bfac"][k] == pytest.approx(1.0 / (2.0 * ph.chi_a2 * (1 - 0.98)), rel=2e-6)
        assert t["sig_jump"][k] == pytest.approx(ph.sig_e + ph.sig_ne, rel=2e-6)
        n = len(mat["elements"])
        for i in range(n):
            assert t["rates"][k, 0, i] == pytest.approx(ph.sig_e_el[i], rel=2e-6, abs=1e-30)
            assert t["rates"][k, 1, i] == pytest.approx(ph.sig_ne_el[i], rel=2e-6, abs=1e-30)
        if k > 0:
            assert t["csda"][k] == pytest.approx(O.csda_range(mat, 1.0, E), rel=1e-8)


@pytest.mark.parametrize("cut_k", [0.0, 2.5])
def test_probe_step_follows_the_oracle_on_common_random_numbers(sde_gpu, oracle_lib, cut_k):
    """Same (seed, history, step) keys, same draw layout, exponential clock in both: the
    GPU step (FP32 tables) and the oracle step (FP64 formulas) give nearly the same
    sample, history by history -- with the fixed cut-off and with theta_c = 2.5 sigma(E)."""
    n = 100_000
    with sde_gpu.SdeDose(_tiny([WATER]), theta_cut_sigmas=cut_k) as d:
        for E in (150.0, 12.0):
            g = d.probe_steps(0, 1.0, E, n, seed=42, h0=1000)
            o = O.single_step(WATER, 1.0, E, n, seed=42, h0=1000, jump_clock=1, theta_cut_sigmas=cut_k)
            same_jump = g["jump"] == o["jump"]
            assert same_jump.mean() > 0.999
            nj = same_jump & (o["jump"] == 0)
            assert np.max(np.abs(g["E"][nj] - o["E"][nj])) < 2e-6 * E + 1e-5
            assert np.max(np.abs(g["cos"][nj] - o["cos"][nj])) < 2e-6
            assert np.max(np.abs(g["ux"][nj] - o["ux"][nj])) < 1e-3 * np.abs(o["ux"][nj]).max()
            el = same_jump & (o["jump"] == 1)
            if el.sum():
                assert np.percentile(np.abs(g["cos"][el] - o["cos"][el]), 99) < 1e-4
            ine = same_jump & (o["jump"] == 2)
            if ine.sum():
                assert np.percentile(np.abs(g["E"][ine] - o["E"][ine]) / E, 99) < 1e-4


@pytest.mark.parametrize("E", [100.0, 20.0])
def test_probe_step_statistics_against_closed_forms(sde_gpu, oracle_lib, E):
    n = 1_000_000
    ph = O.physics(WATER, 1.0, E)
    with sde_gpu.SdeDose(_tiny([WATER]), physics_mask=sde_gpu.PHYS_STRAGGLING) as d:
        g = d.probe_steps(0, 1.0, E, n, seed=7)
    loss = E - g["E"].astype(np.float64)
    c = ph.s1 * 0.05
    se = loss.std() / math.sqrt(n)
    assert abs(loss.mean() - c) < 3.5 * se + 4e-6 * E  # plus FP32 rounding of E
    with sde_gpu.SdeDose(_tiny([WATER]), physics_mask=sde_gpu.PHYS_MCS) as d:
        g = d.probe_steps(0, 1.0, E, n, seed=8)
    cosv = g["cos"].astype(np.float64)
    t = ph.t_sbm
    assert abs(cosv.mean() - math.exp(-t)) < 3.5 * cosv.std() / math.sqrt(n) + t * t / 6 + 1e-7
    mask = sde_gpu.PHYS_ELASTIC | sde_gpu.PHYS_INELASTIC
    with sde_gpu.SdeDose(_tiny([WATER]), physics_mask=mask) as d:
        g = d.probe_steps(0, 1.0, E, n, seed=9)
    p = -math.expm1(-0.05 * (ph.sig_e + ph.sig_ne))
    frac = np.mean(g["jump"] > 0)
    assert abs(frac - p) < 3.5 * math.sqrt(p * (1 - p) / n)
