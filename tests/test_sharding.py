"""Splitting one plan's histories across ranks (the multi-GPU path) on the CPU.

Every history's random stream is keyed by its global id, and tallies are integers, so
disjoint history ranges run with one seed must add up to the whole run exactly.  The
ranges are produced by ``history_shard``; two ``gloo`` ranks run the oracle on their
shards and sum their tallies with ``combine_shards`` (the integer all-reduce the
benchmark's multi-GPU path uses on NCCL), as GPUs would with their dose grids.
"""
import os
import socket

import numpy as np
import pytest

from sde_workloads import water100

BAL_KEYS = ("incident", "deposited", "escaped", "removed", "histories", "steps", "jumps_elastic", "jumps_inelastic")


def _shard():
    # pure-Python helper of the package; importing the package does not load the CUDA library
    from paper_2511_03115_gb300 import history_shard
    return history_shard


@pytest.mark.parametrize("total,world", [(0, 1), (1, 2), (7, 3), (1000, 4), (10**8 + 3, 8)])
def test_history_shards_are_disjoint_and_cover_the_plan(total, world):
    shard = _shard()
    parts = [shard(total, r, world) for r in range(world)]
    assert parts[0][0] == 0
    for (f0, c0), (f1, _) in zip(parts, parts[1:]):
        assert f0 + c0 == f1
    assert parts[-1][0] + parts[-1][1] == total
    counts = [c for _, c in parts]
    assert max(counts) - min(counts) <= 1


def test_history_shard_rejects_bad_ranks():
    shard = _shard()
    with pytest.raises(ValueError):
        shard(10, 2, 2)
    with pytest.raises(ValueError):
        shard(10, 0, 0)


def _full_run(oracle_lib, wl, seed):
    d = oracle_lib.OracleDose(wl)
    try:
        d.run(seed=seed)
        _, edep, bal = d.fetch()
        return edep, bal
    finally:
        d.close()


def test_oracle_ranges_on_one_handle_equal_the_whole_run(oracle_lib):
    wl = water100(1500)
    edep, bal = _full_run(oracle_lib, wl, 11)
    d = oracle_lib.OracleDose(wl)
    try:
        d.run(seed=11, first=0, count=517)
        d.run(seed=11, first=517, count=10**9)  # clipped at the plan's end
        d.run(seed=11, first=1500, count=5)     # beyond the plan: nothing
        _, edep2, bal2 = d.fetch()
    finally:
        d.close()
    assert np.array_equal(edep, edep2)
    assert {k: bal[k] for k in BAL_KEYS} == {k: bal2[k] for k in BAL_KEYS}
    assert bal2["histories"] == 1500


def _rank_main(rank, world, port, n_hist, seed, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2511_03115_gb300 import history_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        oracle.set_threads(2)
        wl = water100(n_hist)
        first, count = history_shard(wl.n_histories, rank, world)
        d = oracle.OracleDose(wl)
        d.run(seed=seed, first=first, count=count)
        _, edep, bal = d.fetch()
        d.close()
        # the combine of the benchmark's multi-GPU path, on CPU tensors over gloo
        from paper_2511_03115_gb300 import combine_shards
        t = torch.from_numpy(edep.view(np.int64).ravel().copy())
        tot = combine_shards(t, bal)
        if rank == 0:
            np.savez(out_path, edep=t.numpy(), bal=np.array([tot[k] for k in BAL_KEYS], np.int64))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_to_the_single_run(oracle_lib, tmp_path):
    import torch.multiprocessing as mp
    n_hist, seed = 2000, 23
    out = str(tmp_path / "reduced.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), n_hist, seed, out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    edep, bal = _full_run(oracle_lib, water100(n_hist), seed)
    assert np.array_equal(got["edep"], edep.astype(np.int64).ravel())
    assert list(got["bal"]) == [int(bal[k]) for k in BAL_KEYS]
    assert bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"]
