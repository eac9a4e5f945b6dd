"""Inputs of the CT-like phantom and spread-out Bragg peak workloads (CPU), and an oracle
run through them.

The HU calibration is pinned at its anchor points (air, water, a bone value) and by
monotonicity; the spread-out Bragg peak weighting by the property that defines it: the
weighted sum of ideal pristine curves D_R(z) ~ (R - z)^(1/p - 1) (Bragg-Kleeman power
law), smeared by range straggling, is flat across the modulated depths.
"""
import math

import numpy as np
import pytest

import sde_workloads as W


def test_hu_calibration_anchor_points_and_monotonicity():
    rho = W.hu_to_density([-1000.0, -500.0, 0.0, 1000.0])
    assert rho[0] == pytest.approx(0.0012) and rho[1] == pytest.approx(0.5)
    assert rho[2] == pytest.approx(1.0) and rho[3] == pytest.approx(1.58)
    hu = np.linspace(-1024, 3000, 4025)
    assert np.all(np.diff(W.hu_to_density(hu)) >= 0)
    mats = W.hu_to_material([-1000, -950, -500, -100, 40, 500, 1500])
    names = [W.CT_MATERIALS[m]["name"] for m in mats]
    assert names == ["air", "air", "lung", "adipose", "soft tissue", "cortical bone", "cortical bone"]
    for m in W.CT_MATERIALS:  # mass fractions close to 1 before the engines renormalise
        assert abs(sum(w for _, w in m["elements"]) - 1.0) < 0.01


def test_bragg_kleeman_energies_match_known_water_ranges():
    # CSDA ranges of 100 and 150 MeV protons in water are 77.2 and 157.7 mm (PSTAR-type)
    E = W.bragg_kleeman_energy([77.2, 157.7])
    assert E[0] == pytest.approx(100.0, rel=0.02) and E[1] == pytest.approx(150.0, rel=0.02)


def test_sobp_weighting_gives_a_flat_plateau_for_ideal_bragg_curves():
    p = 1.77
    r_lo, r_hi, n = 90.0, 140.0, 16
    R, w = W.sobp_layer_weights(r_lo, r_hi, n, p=p)
    assert w.sum() == pytest.approx(1.0) and np.all(np.diff(w) > 0)  # deeper layers weigh more
    z = np.linspace(0.0, 150.0, 3001)
    dose = np.zeros_like(z)
    for Rk, wk in zip(R, w):
        # pristine curve (R - z)^(1/p - 1) smeared by a Gaussian range spread of 1.2 % of R
        # (straggling and the beam's energy spread)
        s = 0.012 * Rk
        rr = Rk + s * np.linspace(-4, 4, 161)
        g = np.exp(-0.5 * np.linspace(-4, 4, 161) ** 2)
        g /= g.sum()
        for Rj, gj in zip(rr, g):
            m = z < Rj - 0.05
            dose[m] += wk * gj * (Rj - z[m]) ** (1.0 / p - 1.0)
    plateau = (z >= r_lo + 6.0) & (z <= r_hi - 8.0)  # clear of the blurred distal edge
    flat = dose[plateau]
    assert flat.max() / flat.min() < 1.06, flat.max() / flat.min()
    # a single layer would not be flat at all
    assert dose[z < 20].mean() < 0.7 * flat.mean()  # proximal dose below the plateau


def test_thorax_phantom_is_seeded_and_has_every_material():
    a = W.thorax_hu((40, 40, 80), 3.0, seed=1)
    b = W.thorax_hu((40, 40, 80), 3.0, seed=1)
    c = W.thorax_hu((40, 40, 80), 3.0, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    wl = W.ct_sobp(1000, seed=1)
    assert set(np.unique(wl.material_id)) == {0, 1, 2, 3, 4}
    assert wl.density.dtype == np.float32 and wl.n_histories == 1000
    assert np.all(wl.spots["E_MeV"] > 100) and np.all(wl.spots["E_MeV"] < 145) and len(wl.spots) == 16 * 16


def test_oracle_runs_the_ct_phantom_with_exact_balance(oracle_lib):
    wl = W.ct_sobp(1500, seed=3, shape=(40, 40, 80), h=3.0)
    _, edep, bal = oracle_lib.run_workload(wl, seed=5)
    assert bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"]
    assert bal["histories"] == 1500 and int(edep.sum()) == bal["deposited"]
    # energy lands in every tissue class the beam crosses
    per_mat = np.bincount(wl.material_id.ravel(), weights=edep.ravel().astype(float), minlength=5)
    assert per_mat[3] > 0 and per_mat[1] > 0
