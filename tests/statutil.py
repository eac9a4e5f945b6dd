"""Helpers of the parity tests: batch statistics of dose grids and the agreement
criterion between the CUDA path and the oracle.

Agreement criterion (per-voxel dose): with B independent batches per side (disjoint
random streams: one seed per batch), each voxel's mean dose carries a standard error
from the batch spread.  In the region where either mean exceeds 1 % of D_max a voxel
agrees when |D_gpu - D_oracle| <= max(3 sqrt(SE_gpu^2 + SE_oracle^2), 0.005 D_max).
The tests require at least 98.5 % of the region to agree (with B = 16 batches per side
the z-score follows a t distribution with about 30 degrees of freedom, so about 0.5 %
of voxels exceed 3 by chance) and the mean squared z-score to stay near 1 (about 1.1 for
that t distribution; a systematic offset raises it).
"""
import numpy as np


def batch_stats(batches):
    b = np.asarray(batches, dtype=np.float64)
    n = b.shape[0]
    return b.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(n)


def compare(gpu_batches, ora_batches, roi_frac=0.01, floor_frac=0.005):
    mg, sg = batch_stats(gpu_batches)
    mo, so = batch_stats(ora_batches)
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
        "max_abs_over_dmax": float(diff.max() / dmax),
        "dmax": float(dmax),
        "mean_gpu": mg,
        "mean_ora": mo,
    }


def balanced(b):
    """Exact balance, and no counter above the incident energy (a wrapped unsigned
    difference would still balance modulo 2^64)."""
    parts = (b["deposited"], b["escaped"], b["removed"])
    return b["incident"] == sum(parts) and all(p <= b["incident"] for p in parts)
