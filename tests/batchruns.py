"""Batch runners of the parity tests: per-voxel moments of the dose per history over
independent batches (one seed each) on the CUDA path and on the oracle, the per-voxel
criterion, and the distal ranges of the batches' depth curves."""
import math

import numpy as np

import oracle as O
from oracle import analysis as A
from statutil import Moments, balanced, compare_moments

B = 16  # independent batches per side


def _gpu_moments(S, wl, per_batch, seeds, **kw):
    """Per-voxel moments of the dose per history over batches of ``per_batch`` histories
    (one seed each), and each batch's depth curve of deposited energy per history (the two
    sides run different numbers of histories per batch)."""
    wl = wl.with_histories(per_batch)
    acc, idds = Moments(), []
    rho = wl.density.astype(np.float64)
    with S.SdeDose(wl, **kw) as d:
        for s in seeds:
            d.reset()
            d.run(wl.spots, seed=s)
            dose, edep, bal = d.fetch()
            assert balanced(bal) and int(edep.sum(dtype=np.uint64)) == bal["deposited"]
            assert bal["histories"] == wl.n_histories
            acc.add(dose / wl.n_histories)
            idds.append(A.idd(dose * rho) / wl.n_histories)
    return acc, np.array(idds)


def _oracle_moments(wl, per_batch, seeds, **kw):
    wl = wl.with_histories(per_batch)
    acc, idds = Moments(), []
    rho = wl.density.astype(np.float64)
    d = O.OracleDose(wl, **kw)
    try:
        for s in seeds:
            d.reset()
            d.run(seed=s)
            dose, _, bal = d.fetch()
            assert balanced(bal) and bal["histories"] == wl.n_histories
            acc.add(dose / wl.n_histories)
            idds.append(A.idd(dose * rho) / wl.n_histories)
    finally:
        d.close()
    return acc, np.array(idds)


def _range_of_idds(idds, hz, level):
    z = A.z_centres(idds.shape[1], hz)
    per = np.array([A.distal_range(x, z, level) for x in idds])
    return A.distal_range(idds.mean(0), z, level), per.std(ddof=1) / math.sqrt(len(per))


def _check_range_idds(gi, oi, hz, tol_mm=0.05):
    out = {}
    for level in (0.8, 0.9):
        rg, sg = _range_of_idds(gi, hz, level)
        ro, so = _range_of_idds(oi, hz, level)
        out[f"R{int(level * 100)}"] = (rg, ro)
        assert abs(rg - ro) <= max(tol_mm, 3.0 * math.hypot(sg, so)), (level, rg, ro, sg, so)
    return out


def _per_voxel(g, o, label):
    mg, sg = g.mean_se()
    mo, so = o.mean_se()
    c = compare_moments(mg, sg, mo, so)
    print(label, {k: v for k, v in c.items() if not k.startswith("mean_")}, c["mean_z2"])
    assert c["pass_frac"] >= 0.985, (label, c)
    assert 0.6 < c["mean_z2"] < 1.5, (label, c)
    assert c["max_z"] <= 8.0, (label, c)
    return c


# GPU batches of 640 000 histories: 20 000 cohorts of 32, more than three rounds of the
# 6 080 persistent warps of the default launch, so warps refill from the queue many times.
GPU_BATCH = 640_000
