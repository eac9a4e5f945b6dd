"""Reference dose metrics (Sec. 2.2.3 of arXiv 2511.03115), plain numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each function is the
plain definition: integrated depth dose, distal range at a dose level by linear
interpolation, central-axis and lateral profiles, D99-normalised voxel
differences in the 1 % region of interest, and a brute-force 3D gamma index
with local dose normalisation and sub-voxel search.
"""
from __future__ import annotations

import numpy as np


def idd(dose: np.ndarray) -> np.ndarray:
    """Integrated depth dose: sum over x and y for every z slice (dose shape (nz, ny, nx))."""
    return dose.sum(axis=(1, 2))


def z_centres(nz: int, hz: float, oz: float = 0.0) -> np.ndarray:
    return oz + (np.arange(nz) + 0.5) * hz


def distal_range(curve: np.ndarray, z: np.ndarray, level: float = 0.8) -> float:
    """Depth beyond the maximum where ``curve`` falls to ``level`` x max (Sec. 2.2.3: R90 on the
    integrated depth dose, linear interpolation between voxel centres).  Returns nan when the
    curve never falls below the level after its maximum."""
    c = np.asarray(curve, dtype=np.float64)
    i = int(np.argmax(c))
    thr = level * c[i]
    for j in range(i, len(c) - 1):
        if c[j] >= thr > c[j + 1]:
            return float(z[j] + (thr - c[j]) / (c[j + 1] - c[j]) * (z[j + 1] - z[j]))
    return float("nan")


def dose_difference_d99(ref: np.ndarray, ev: np.ndarray, roi_frac: float = 0.01):
    """Voxel differences in the region receiving >= 1 % of the maximum reference dose,
    normalised to the 99th percentile of the reference dose within that region."""
    roi = ref >= roi_frac * ref.max()
    d99 = np.percentile(ref[roi], 99.0)
    return (ev - ref)[roi] / d99, roi, d99


def _trilinear(vol: np.ndarray, pz, py, px):
    """Trilinear interpolation of ``vol`` (nz, ny, nx) at fractional voxel-centre indices;
    points outside the grid take the nearest edge value."""
    nz, ny, nx = vol.shape
    pz = np.clip(pz, 0.0, nz - 1.0)
    py = np.clip(py, 0.0, ny - 1.0)
    px = np.clip(px, 0.0, nx - 1.0)
    z0 = np.minimum(np.floor(pz).astype(np.int64), nz - 2 if nz > 1 else 0)
    y0 = np.minimum(np.floor(py).astype(np.int64), ny - 2 if ny > 1 else 0)
    x0 = np.minimum(np.floor(px).astype(np.int64), nx - 2 if nx > 1 else 0)
    fz, fy, fx = pz - z0, py - y0, px - x0
    z1 = np.minimum(z0 + 1, nz - 1)
    y1 = np.minimum(y0 + 1, ny - 1)
    x1 = np.minimum(x0 + 1, nx - 1)
    c = 0.0
    for zi, wz in ((z0, 1 - fz), (z1, fz)):
        for yi, wy in ((y0, 1 - fy), (y1, fy)):
            for xi, wx in ((x0, 1 - fx), (x1, fx)):
                c = c + vol[zi, yi, xi] * (wz * wy * wx)
    return c


def gamma_pass_rate(ref: np.ndarray, ev: np.ndarray, spacing_mm, dd: float = 0.02,
                    dta_mm: float = 0.5, threshold: float = 0.01, step_frac: int = 10,
                    return_map: bool = False):
    """3D gamma index, local normalisation (Sec. 2.2.3).

    For each reference voxel with dose >= ``threshold`` x max(ref), gamma is the minimum over
    evaluated positions within the DTA ball (searched on a grid of step DTA/step_frac, the
    evaluated dose trilinearly interpolated) of sqrt(|dr|^2/DTA^2 + (D_e - D_r)^2/(dd D_r)^2).
    A voxel passes when gamma <= 1; points beyond the DTA can never pass, so the ball suffices.
    Returns the pass fraction (and the boolean pass map over the evaluated voxels)."""
    hz, hy, hx = spacing_mm[2], spacing_mm[1], spacing_mm[0]
    mask = ref >= threshold * ref.max()
    idx = np.argwhere(mask)
    r = ref[mask]
    e0 = ev[mask]
    tol = dd * r
    passed = np.abs(e0 - r) <= tol
    todo = np.nonzero(~passed)[0]
    if len(todo):
        step = dta_mm / step_frac
        g = np.arange(-step_frac, step_frac + 1) * step
        oz, oy, ox = np.meshgrid(g, g, g, indexing="ij")
        d2 = (oz ** 2 + oy ** 2 + ox ** 2) / dta_mm ** 2
        sel = d2 <= 1.0
        oz, oy, ox, d2 = oz[sel], oy[sel], ox[sel], d2[sel]
        for chunk in np.array_split(todo, max(1, len(todo) // 256)):
            iz, iy, ix = idx[chunk, 0], idx[chunk, 1], idx[chunk, 2]
            pz = iz[:, None] + oz[None, :] / hz
            py = iy[:, None] + oy[None, :] / hy
            px = ix[:, None] + ox[None, :] / hx
            de = _trilinear(ev, pz, py, px) - r[chunk, None]
            g2 = d2[None, :] + (de / tol[chunk, None]) ** 2
            passed[chunk] = g2.min(axis=1) <= 1.0
    rate = float(passed.mean()) if len(passed) else 1.0
    if return_map:
        pm = np.zeros(ref.shape, bool)
        pm[mask] = passed
        return rate, pm, mask
    return rate
