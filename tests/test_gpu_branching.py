"""The branching model on the GPU (secondary_fraction kappa > 0; Sec. 2.1.1's extension to
secondary protons, one generation): primaries queue the secondaries of their non-elastic
events, a second launch transports them.  Checked against the oracle's branching model
per voxel and on common random numbers; the tally is bit-identical across launch shapes
and history ranges (the queue's chunking and order do not matter: every track's random
streams are keyed by (history, segment, step))."""
import numpy as np
import pytest

import oracle as O
from oracle import analysis as A
from sde_workloads import slab150, water100
from statutil import balanced
from batchruns import B, GPU_BATCH, _gpu_moments, _oracle_moments, _per_voxel

pytestmark = pytest.mark.gpu

KAPPA = 0.6


def test_branching_per_voxel_parity_on_the_slab_phantom(sde_gpu, oracle_lib):
    """Slab phantom (150 MeV beam) at 0.5 mm with secondaries (bone and lung slabs change the
    secondaries' ranges): GPU 16 x 640 000 against the oracle 16 x 62 500."""
    wl = slab150()
    g, _ = _gpu_moments(sde_gpu, wl, GPU_BATCH, range(B), secondary_fraction=KAPPA)
    o, _ = _oracle_moments(wl, 62_500, range(200, 200 + B), secondary_fraction=KAPPA)
    _per_voxel(g, o, "slab150 branching")


def test_branching_moves_removed_energy_into_the_tally(sde_gpu):
    wl = water100(200_000)
    _, e0, b0 = sde_gpu.run_workload(wl, seed=4)
    _, e1, b1 = sde_gpu.run_workload(wl, seed=4, secondary_fraction=KAPPA)
    for b in (b0, b1):
        assert balanced(b) and b["histories"] == 200_000
    assert b1["incident"] == b0["incident"]
    assert b1["removed"] < b0["removed"] and b1["steps"] > b0["steps"]
    assert int(e1.sum(dtype=np.uint64)) == b1["deposited"] > b0["deposited"]
    # the primaries' tracks are the same draws: the first-generation part of the tally can
    # only grow (secondaries add deposits, never remove any)
    assert np.all(e1 >= e0)


@pytest.mark.parametrize("cut_k", [0.0, 2.5])
def test_branching_common_random_numbers(sde_gpu, oracle_lib, cut_k):
    """With the oracle on the exponential clock both sides draw the same numbers for every
    track, secondaries included: counts and depth curves agree far more tightly than
    independent runs would."""
    wl = water100(20_000)
    _, eg, bg = sde_gpu.run_workload(wl, seed=3, theta_cut_sigmas=cut_k, secondary_fraction=KAPPA)
    _, eo, bo = O.run_workload(wl, seed=3, jump_clock=1, theta_cut_sigmas=cut_k, secondary_fraction=KAPPA)
    assert balanced(bg) and balanced(bo)
    ig, io = A.idd(eg.astype(float)), A.idd(eo.astype(float))
    assert np.max(np.abs(ig - io)) / io.max() < 0.01
    assert abs(bg["jumps_inelastic"] - bo["jumps_inelastic"]) <= 0.01 * bo["jumps_inelastic"] + 5
    assert abs(bg["steps"] - bo["steps"]) <= 1e-3 * bo["steps"]
    assert abs(bg["removed"] - bo["removed"]) <= 0.02 * bo["removed"]


def test_branching_tally_is_independent_of_chunks_and_launch_shape(sde_gpu):
    """3e6 histories span two chunks of the secondary queue (2^21 histories each); the same
    plan split into two ranges, and run with another launch shape, gives the same tally."""
    from paper_2511_03115_gb300 import history_shard
    wl = water100(3_000_000)
    with sde_gpu.SdeDose(wl, secondary_fraction=KAPPA) as d:
        d.run(wl.spots, seed=8)
        _, ref, rb = d.fetch(dose=False)
        assert balanced(rb) and rb["histories"] == 3_000_000
        d.reset()
        for r in range(2):
            first, count = history_shard(wl.n_histories, r, 2)
            d.run(wl.spots, seed=8, first=first, count=count)
        _, e, b = d.fetch(dose=False)
        assert np.array_equal(e, ref) and b == rb
    with sde_gpu.SdeDose(wl, secondary_fraction=KAPPA, tuning={"warps_per_block": 4, "batch": 64}) as d:
        d.run(wl.spots, seed=8)
        _, e, b = d.fetch(dose=False)
        assert np.array_equal(e, ref) and b == rb


def test_branching_is_rejected_by_the_allocation_free_entry(sde_gpu):
    import ctypes as C
    import torch
    S = sde_gpu
    wl = water100(10)
    vox = torch.zeros(wl.n_voxels, dtype=torch.int32, device="cuda")
    spots = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
    m = S._Materials(wl.materials)
    p = S.default_params(secondary_fraction=KAPPA)
    nx, ny, nz = wl.shape
    rc = S.lib().sde_transport_noalloc(nx, ny, nz, (C.c_double * 3)(*wl.voxel_mm), (C.c_double * 3)(*wl.origin_mm),
                                       vox.data_ptr(), m.arr, 1, C.byref(p), spots.data_ptr(), 1, C.c_uint64(0),
                                       out.data_ptr(), None, None, None)
    assert rc == S.SDE_EINVAL and "branching" in S.lib().sde_last_error().decode()
