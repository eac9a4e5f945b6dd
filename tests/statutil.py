"""Helpers of the parity tests: batch statistics of dose grids and the agreement
criterion between the CUDA path and the oracle.

Agreement criterion (per-voxel dose): with B independent batches per side (disjoint
random streams: one seed per batch), each voxel's mean dose carries a standard error
from the batch spread.  In the region where either mean exceeds 1 % of D_max a voxel
agrees when |D_gpu - D_oracle| <= max(3 sqrt(SE_gpu^2 + SE_oracle^2), 0.005 D_max).
The tests require at least 98.5 % of the region to agree (with B = 16 batches per side
the z-score follows a t distribution with about 30 degrees of freedom, so about 0.5 %
of voxels exceed 3 by chance), the mean squared z-score to stay near 1 (about 1.1 for
that t distribution; a systematic offset raises it) and no voxel to lie beyond 8
combined standard errors (a local error that the fractions would average away).  The
oracle against itself with independent seeds, at the per-voxel sizes of the tests
(10^6 histories per side; 1 mm and 0.5 mm voxels), gives 99.6-99.7 % agreement, mean z^2
1.08 and a largest z of 5.1-6.3 over 5e4-3e5 voxels; its largest |difference| is 5-6 % of
D_max there, which is why 0.5 % of D_max serves as the floor of the tolerance rather than
as a bound on every voxel.
"""
import numpy as np


def batch_stats(batches):
    b = np.asarray(batches, dtype=np.float64)
    n = b.shape[0]
    return b.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(n)


def compare(gpu_batches, ora_batches, roi_frac=0.01, floor_frac=0.005):
    mg, sg = batch_stats(gpu_batches)
    mo, so = batch_stats(ora_batches)
    return compare_moments(mg, sg, mo, so, roi_frac, floor_frac)


def compare_moments(mg, sg, mo, so, roi_frac=0.01, floor_frac=0.005):
    """The agreement statistics from per-voxel means and standard errors of both sides."""
    dmax = max(mg.max(), mo.max())
    roi = (mg >= roi_frac * dmax) | (mo >= roi_frac * dmax)
    diff = np.abs(mg - mo)[roi]
    se = np.sqrt(sg ** 2 + so ** 2)[roi]
    tol = np.maximum(3.0 * se, floor_frac * dmax)
    ok = diff <= tol
    z = diff / np.where(se > 0, se, np.inf)
    return {
        "n_roi": int(roi.sum()),
        "pass_frac": float(ok.mean()),
        "mean_z2": float(np.mean(np.minimum(z, 50.0) ** 2)),
        "max_z": float(np.max(np.where(np.isfinite(z), z, 0.0))) if z.size else 0.0,
        "max_abs_over_dmax": float(diff.max() / dmax),
        "dmax": float(dmax),
        "mean_gpu": mg,
        "mean_ora": mo,
    }


class Moments:
    """Running per-voxel sum and sum of squares of batch results (one batch at a time, so
    16 batches of a 12 M-voxel grid need two grids of memory, not sixteen)."""

    def __init__(self):
        self.n = 0
        self.s1 = None
        self.s2 = None

    def add(self, x):
        x = np.asarray(x, dtype=np.float64)
        if self.s1 is None:
            self.s1 = np.zeros_like(x)
            self.s2 = np.zeros_like(x)
        self.s1 += x
        self.s2 += x * x
        self.n += 1

    def mean_se(self):
        m = self.s1 / self.n
        var = np.maximum(self.s2 - self.n * m * m, 0.0) / (self.n - 1)
        return m, np.sqrt(var / self.n)


def balanced(b):
    """Exact balance, and no counter above the incident energy (a wrapped unsigned
    difference would still balance modulo 2^64)."""
    parts = (b["deposited"], b["escaped"], b["removed"])
    return b["incident"] == sum(parts) and all(p <= b["incident"] for p in parts)
