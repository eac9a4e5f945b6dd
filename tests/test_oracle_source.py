"""Pins of the oracle's source sampling (Y_0 of a history from its spot; Sec. 2.2.2 beam,
with the Gaussian spot of the workloads): the moments a Gaussian pencil beam must have,
measured in a frame built here, independently of the oracle's own basis.

A spot with lateral sigma s_xy, energy spread s_E and angular sigma s_a, aimed along an
oblique unit vector u, must give: entry points in the plane through the spot position
perpendicular to u, with variance s_xy^2 along any two orthonormal axes of that plane
and no correlation between them; energies of mean E and variance s_E^2; directions of
unit length whose tangent components along the two axes have variance s_a^2 (the
small-angle Gaussian, per axis).  A sigma-for-variance mix-up, a factor sqrt(2) on a
width, or a basis not perpendicular to u fails one of these checks."""
import math

import numpy as np
import pytest

import oracle as O
from sde_workloads import pencil

N = 1_000_000


def _frame(u):
    """Two orthonormal axes perpendicular to u by Gram-Schmidt from the coordinate axis
    least aligned with u (not the oracle's construction)."""
    e = np.eye(3)[int(np.argmin(np.abs(u)))]
    a = e - np.dot(e, u) * u
    a /= np.linalg.norm(a)
    b = np.cross(u, a)
    return a, b


def _var_within(x, sigma2, k=3.0):
    """Sample variance equals sigma2 within k standard errors of the variance estimate of a
    Gaussian sample (sigma2 sqrt(2/(n-1)))."""
    v = float(np.var(x, ddof=1))
    se = sigma2 * math.sqrt(2.0 / (len(x) - 1))
    return abs(v - sigma2) <= k * se, v, se


@pytest.fixture(scope="module")
def oblique_spot():
    u = np.array([0.3, -0.2, 0.93])
    u /= np.linalg.norm(u)
    spot = pencil(150.0, N, x=3.0, y=-2.0, z=1.0, sigma_xy=2.5, sigma_E=1.5, sigma_angle=0.01, u=tuple(u))
    E, r, w = O.sample_source(spot[0], N, seed=7)
    return spot[0], u, E, r, w


def test_entry_points_lie_in_the_plane_perpendicular_to_the_beam(oracle_lib, oblique_spot):
    spot, u, _, r, _ = oblique_spot
    d = r - np.array([spot["x_mm"], spot["y_mm"], spot["z_mm"]])
    assert np.max(np.abs(d @ u)) < 1e-12 * max(1.0, np.max(np.abs(d)))


def test_lateral_offsets_have_variance_sigma_xy_squared_on_both_axes(oracle_lib, oblique_spot):
    spot, u, _, r, _ = oblique_spot
    a, b = _frame(u)
    d = r - np.array([spot["x_mm"], spot["y_mm"], spot["z_mm"]])
    s2 = float(spot["sigma_xy_mm"]) ** 2
    for axis in (a, b):
        x = d @ axis
        ok, v, se = _var_within(x, s2)
        assert ok, (v, s2, se)
        assert abs(x.mean()) <= 3.0 * math.sqrt(s2 / N)
    # no correlation between the two axes: E[xa xb] = 0 within 3 standard errors (s^2/sqrt(n))
    assert abs(np.mean((d @ a) * (d @ b))) <= 3.0 * s2 / math.sqrt(N)


def test_energies_have_mean_E_and_variance_sigma_E_squared(oracle_lib, oblique_spot):
    spot, _, E, _, _ = oblique_spot
    sE = float(spot["sigma_E_MeV"])
    assert abs(E.mean() - float(spot["E_MeV"])) <= 3.0 * sE / math.sqrt(N)
    ok, v, se = _var_within(E, sE * sE)
    assert ok, (v, sE * sE, se)


def test_directions_have_per_axis_tangent_variance_sigma_angle_squared(oracle_lib, oblique_spot):
    spot, u, _, _, w = oblique_spot
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    a, b = _frame(u)
    sa2 = float(spot["sigma_angle_rad"]) ** 2
    along = w @ u
    assert np.all(along > 0.99)
    for axis in (a, b):
        t = (w @ axis) / along
        # tan(theta) ~ theta: the relative bias of the variance is 8/3 s_a^2 ~ 3e-4, well
        # inside the 3-standard-error band (4e-3 relative) of 10^6 samples
        ok, v, se = _var_within(t, sa2)
        assert ok, (v, sa2, se)
        assert abs(t.mean()) <= 3.0 * math.sqrt(sa2 / N)


def test_spot_without_spreads_is_a_point_source(oracle_lib):
    u = np.array([0.0, 0.6, 0.8])
    spot = pencil(100.0, 10, x=1.0, y=2.0, z=0.5, u=tuple(u))
    E, r, w = O.sample_source(spot[0], 1000, seed=3)
    assert np.all(E == 100.0)
    assert np.allclose(r, [1.0, 2.0, 0.5], atol=0, rtol=0)
    assert np.allclose(w, u, atol=1e-15)


def test_energy_below_the_absorption_energy_is_raised_to_it(oracle_lib):
    """A spread that reaches below e_min draws no negative or sub-threshold energy."""
    spot = pencil(0.2, 10, sigma_E=0.5)
    E, _, _ = O.sample_source(spot[0], 20000, seed=1)
    assert E.min() == pytest.approx(0.05) and np.mean(E == 0.05) > 0.3
