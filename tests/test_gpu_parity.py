"""Whole-transport parity of the CUDA path against the oracle on the seeded workloads.

Agreement is statistical (the dose is a random field; see tests/statutil.py for the
per-voxel criterion), the energy balance is exact, and the tally of a seed is
bit-identical across runs and launch shapes."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import analysis as A
from sde_workloads import WATER, insert150, plan2000, slab150, water100
from batchruns import B, GPU_BATCH, _check_range_idds, _gpu_moments, _oracle_moments, _per_voxel
from statutil import balanced, compare

pytestmark = pytest.mark.gpu

def _gpu_batches(S, wl, n_total, seeds, **kw):
    wl = wl.with_histories(n_total // len(seeds))
    out, bals = [], []
    with S.SdeDose(wl, **kw) as d:
        for s in seeds:
            d.reset()
            d.run(wl.spots, seed=s)
            dose, edep, bal = d.fetch()
            assert balanced(bal) and int(edep.sum(dtype=np.uint64)) == bal["deposited"]
            assert bal["histories"] == wl.n_histories
            out.append(dose)
            bals.append(bal)
    return np.array(out), bals


def _oracle_batches(wl, n_total, seeds, **kw):
    wl = wl.with_histories(n_total // len(seeds))
    out = []
    d = O.OracleDose(wl, **kw)
    try:
        for s in seeds:
            d.reset()
            d.run(seed=s)
            dose, _, bal = d.fetch()
            assert balanced(bal)
            out.append(dose)
    finally:
        d.close()
    return np.array(out)


def _r_levels(batches, hz, level, density):
    """Distal range of the depth curve of deposited energy (dose x density summed over
    x, y): with heterogeneous densities the dose-to-medium maximum can sit in a
    low-density slab, while the energy curve peaks at the Bragg peak."""
    z = A.z_centres(batches.shape[1], hz)
    per = np.array([A.distal_range(A.idd(b * density), z, level) for b in batches])
    full = A.distal_range(A.idd(batches.mean(0) * density), z, level)
    return full, per.std(ddof=1) / math.sqrt(len(per))


def _check_range(g, o, hz, density, tol_mm=0.05):
    for level in (0.8, 0.9):
        rg, sg = _r_levels(g, hz, level, density)
        ro, so = _r_levels(o, hz, level, density)
        assert abs(rg - ro) <= max(tol_mm, 3.0 * math.hypot(sg, so)), (level, rg, ro, sg, so)


def test_water100_dose_parity(sde_gpu, oracle_lib):
    """Water workload: 100 MeV pencil beam in water, 40x40x120 mm at 1 mm, per voxel:
    GPU 16 x 640 000 histories against the oracle 16 x 20 000."""
    wl = water100()
    g, gi = _gpu_moments(sde_gpu, wl, GPU_BATCH, range(B))
    o, oi = _oracle_moments(wl, 20_000, range(100, 100 + B))
    _per_voxel(g, o, "water100 1 mm")
    print(_check_range_idds(gi, oi, 1.0))


def test_water100_at_its_stated_size(sde_gpu, oracle_lib):
    """The workload exactly as stated (10^4 protons, seed 0): exact balance, determinism,
    and a depth-dose range consistent with the oracle's run of the same size."""
    wl = water100()
    d1, e1, b1 = sde_gpu.run_workload(wl)
    d2, e2, b2 = sde_gpu.run_workload(wl)
    assert np.array_equal(e1, e2) and b1 == b2 and balanced(b1)
    assert b1["histories"] == 10_000
    _, eo, bo = O.run_workload(wl)
    z = A.z_centres(120, 1.0)
    rg = A.distal_range(A.idd(e1.astype(float)), z, 0.8)
    ro = A.distal_range(A.idd(eo.astype(float)), z, 0.8)
    assert abs(rg - ro) < 0.25  # 10^4 histories: statistical spread of R80 ~0.05 mm
    assert abs(b1["incident"] - bo["incident"]) / bo["incident"] < 1e-9 + 1e-6


@pytest.mark.parametrize("cut_k", [0.0, 2.5])
def test_water100_common_random_numbers(sde_gpu, oracle_lib, cut_k):
    """With the oracle on the exponential jump clock both sides draw identical numbers for
    every history; the tallies then agree far more tightly than independent runs.  Also
    with the energy-dependent cut-off theta_c = 2.5 sigma(E) (Sec. 2.1.3)."""
    wl = water100(20_000)
    _, eg, bg = sde_gpu.run_workload(wl, seed=3, theta_cut_sigmas=cut_k)
    _, eo, bo = O.run_workload(wl, seed=3, jump_clock=1, theta_cut_sigmas=cut_k)
    ig, io = A.idd(eg.astype(float)), A.idd(eo.astype(float))
    assert np.max(np.abs(ig - io)) / io.max() < 0.01
    assert abs(bg["jumps_inelastic"] - bo["jumps_inelastic"]) <= 0.01 * bo["jumps_inelastic"] + 5
    assert abs(bg["jumps_elastic"] - bo["jumps_elastic"]) <= 0.01 * bo["jumps_elastic"] + 5
    assert abs(bg["steps"] - bo["steps"]) <= 1e-3 * bo["steps"]


def test_tally_is_independent_of_launch_shape(sde_gpu):
    wl = water100(30_000)
    outs = []
    for tune in ({"warps_per_block": 8, "batch": 256}, {"warps_per_block": 2, "batch": 32, "refill_min": 1},
                 {"warps_per_block": 4, "batch": 1024, "blocks_per_sm": 1, "table_smem": 1},
                 {"warps_per_block": 8, "batch": 64, "refill_min": 16, "table_smem": 2, "aggregate": 1},
                 {"warps_per_block": 8, "aggregate": 2, "refill_min": 8}):
        with sde_gpu.SdeDose(wl, tuning=tune) as d:
            d.run(wl.spots, seed=11)
            outs.append(d.fetch()[1:])
    for e, b in outs[1:]:
        assert np.array_equal(e, outs[0][0]) and b == outs[0][1]


def test_slab150_per_voxel_parity(sde_gpu, oracle_lib):
    """Slab phantom (water / bone-like / lung-like / water slabs) at its own 0.5 mm
    voxels: every voxel above 1 % of D_max, GPU 16 x 640 000 histories against the oracle
    16 x 62 500; distal R80/R90 of the energy depth curve."""
    wl = slab150()
    g, gi = _gpu_moments(sde_gpu, wl, GPU_BATCH, range(B))
    o, oi = _oracle_moments(wl, 62_500, range(200, 200 + B))
    _per_voxel(g, o, "slab150 0.5 mm")
    print(_check_range_idds(gi, oi, 0.5))


def test_insert150_per_voxel_parity(sde_gpu, oracle_lib):
    """Insert phantom (bone half-space x > 0, z 30-80 mm; edge on the beam axis) at its
    own 1 mm voxels: every voxel above 1 % of D_max (which includes the lateral profiles at
    every depth), GPU 16 x 640 000 against the oracle 16 x 62 500; the bone side stops
    earlier on both sides; distal R80/R90 of the whole beam's energy depth curve."""
    wl = insert150()
    g, gi = _gpu_moments(sde_gpu, wl, GPU_BATCH, range(B))
    o, oi = _oracle_moments(wl, 62_500, range(300, 300 + B))
    c = _per_voxel(g, o, "insert150 1 mm")
    mg, mo = c["mean_gpu"], c["mean_ora"]
    left = mg[:, :, :40].sum(axis=(1, 2))
    right = mg[:, :, 40:].sum(axis=(1, 2))
    assert int(np.argmax(right)) < int(np.argmax(left))  # the bone side stops earlier
    assert int(np.argmax(mo[:, :, 40:].sum(axis=(1, 2)))) < int(np.argmax(mo[:, :, :40].sum(axis=(1, 2))))
    print(_check_range_idds(gi, oi, 1.0))


def test_plan2000_per_voxel_parity(sde_gpu, oracle_lib):
    """The 2000-spot plan on the 200 x 200 x 300 sphere phantom at its own 1 mm
    voxels, all spots in one launch: every voxel above 1 % of D_max, GPU 16 x 640 000
    histories against the oracle 16 x 200 000 (each spot's count scaled in proportion: ~100
    histories per spot and batch, so the oracle's batch spread, not the GPU's, sets the
    standard errors)."""
    wl = plan2000()  # the plan's own spot weights; each batch rescales them
    g, _ = _gpu_moments(sde_gpu, wl, GPU_BATCH, range(B))
    o, _ = _oracle_moments(wl, 200_000, range(400, 400 + B))
    _per_voxel(g, o, "plan2000 1 mm")


def test_chord_split_tally_parity(sde_gpu, oracle_lib):
    wl = water100()
    n = 64_000
    g, _ = _gpu_batches(sde_gpu, wl, n, range(B), tally_mode=1)
    o = _oracle_batches(wl, n, range(500, 500 + B), tally_mode=1)
    c = compare(g, o)
    print({k: v for k, v in c.items() if not k.startswith("mean_")})
    assert c["pass_frac"] >= 0.985, c
    assert 0.6 < c["mean_z2"] < 1.5, c
    _check_range(g, o, 1.0, wl.density)


def test_device_resident_spots_on_a_torch_stream(sde_gpu):
    import torch
    wl = water100(20_000)
    raw = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    st = torch.cuda.Stream()
    with sde_gpu.SdeDose(wl, stream=st) as d:
        d.run_device(raw.data_ptr(), len(wl.spots), seed=5)
        dose_t = torch.empty(wl.n_voxels, dtype=torch.float64, device="cuda")
        edep_t = torch.empty(wl.n_voxels, dtype=torch.int64, device="cuda")
        bal = d.fetch_device(dose_t.data_ptr(), edep_t.data_ptr(), balance=True)
        st.synchronize()
        dose_h, edep_h, bal_h = d.fetch()
    assert balanced(bal) and bal == bal_h
    assert np.array_equal(edep_t.cpu().numpy().view(np.uint64).reshape(edep_h.shape), edep_h)
    assert np.array_equal(dose_t.cpu().numpy().reshape(dose_h.shape), dose_h)
    _, e_host, _ = sde_gpu.run_workload(wl, seed=5)
    assert np.array_equal(e_host, edep_h)


def test_step_cap_is_reported_and_balance_stays_exact(sde_gpu):
    wl = water100(2000)
    with sde_gpu.SdeDose(wl, max_steps=20) as d:
        d.run(wl.spots, seed=1)
        with pytest.raises(sde_gpu.SdeError) as ei:
            d.sync()
        assert ei.value.code == sde_gpu.SDE_EDEVICE and "step cap" in str(ei.value)
        _, _, b = d.fetch()
        # every history stops at the cap unless a non-elastic event ended it earlier
        assert balanced(b) and 0.99 * 20 * 2000 <= b["steps"] <= 20 * 2000
        assert b["histories"] == 2000


def test_invalid_device_spot_is_flagged(sde_gpu):
    import torch
    wl = water100(100)
    bad = wl.spots.copy()
    bad["E_MeV"] = -5.0
    raw = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    with sde_gpu.SdeDose(wl) as d:
        d.run_device(raw.data_ptr(), 1, seed=0)
        with pytest.raises(sde_gpu.SdeError) as ei:
            d.sync()
        assert "invalid device-resident spot" in str(ei.value)
        _, _, b = d.fetch()
        assert b["histories"] == 0 and b["incident"] == 0


def test_host_spot_validation(sde_gpu):
    wl = water100(10)
    with sde_gpu.SdeDose(wl) as d:
        bad = wl.spots.copy()
        bad["E_MeV"] = 400.0
        with pytest.raises(sde_gpu.SdeError):
            d.run(bad)
        bad = wl.spots.copy()
        bad["uz"] = 0.0
        with pytest.raises(sde_gpu.SdeError):
            d.run(bad)


def test_empty_spot_and_escape_only_beams(sde_gpu):
    """A spot with zero histories runs nothing; a beam aimed away from the phantom only
    escapes."""
    wl = water100(1000)
    sp = np.concatenate([wl.spots, wl.spots])
    sp["n_hist"][0] = 0
    _, e, b = sde_gpu.run_workload(wl, spots=sp)
    assert b["histories"] == 1000 and balanced(b)
    away = wl.spots.copy()
    away["uz"] = -1.0
    away["z_mm"] = -1.0
    _, e, b = sde_gpu.run_workload(wl, spots=away)
    assert e.sum() == 0 and b["escaped"] == b["incident"] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_straight_track_tally_matches_the_oracle(sde_gpu, oracle_lib, mode):
    """All noise off: one oblique deterministic track.  The GPU tally (midpoint or chord
    split) must match the oracle's voxel by voxel up to FP32 rounding of the energies."""
    from sde_workloads import Workload, pencil
    nx, ny, nz = 20, 20, 30
    u = np.array([0.35, 0.2, 1.0])
    u /= np.linalg.norm(u)
    wl = Workload("track", (nx, ny, nz), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0),
                  np.ones((nz, ny, nx), np.float32), np.zeros((nz, ny, nx), np.uint8), [WATER],
                  pencil(25.0, 1, x=6.3, y=4.7, z=0.0, u=tuple(u)))
    _, eg, bg = sde_gpu.run_workload(wl, physics_mask=0, tally_mode=mode)
    _, eo, bo = O.run_workload(wl, physics_mask=0, tally_mode=mode)
    assert bg["steps"] == bo["steps"] and balanced(bg)
    assert np.allclose(eg.astype(float), eo.astype(float), rtol=2e-5, atol=2e-5 * eo.max())


def test_autotune_and_graph_launch_keep_the_tally(sde_gpu):
    wl = water100(20_000)
    with sde_gpu.SdeDose(wl) as d:
        d.run(wl.spots, seed=11)
        _, ref, rb = d.fetch(dose=False)
        d.reset()
        d.run(wl.spots, seed=12)
        _, ref12, _ = d.fetch(dose=False)
        best = d.autotune(wl.spots, seed=99, max_histories=8000)
        assert best == d.get_tuning()
        _, e0, b0 = d.fetch(dose=False)
        assert e0.sum() == 0 and b0["histories"] == 0  # autotune leaves a clean tally
        d.run(wl.spots, seed=11)
        _, e1, b1 = d.fetch(dose=False)
        assert np.array_equal(e1, ref) and b1 == rb
        d.set_tuning(graph=2)
        for seed, want in ((11, ref), (12, ref12), (11, ref)):
            d.reset()
            d.run(wl.spots, seed=seed)
            _, e, _ = d.fetch(dose=False)
            assert np.array_equal(e, want)


@pytest.mark.parametrize("graph", [0, 2])
def test_history_ranges_add_up_to_the_whole_run(sde_gpu, graph):
    """The multi-GPU split of a plan: shards of its global history ids (run here one after
    the other on one handle, which accumulates) give the whole run's integer tally and
    balance bit for bit, in plain and graph launch mode; a range past the plan runs
    nothing and an over-long range is clipped."""
    from sde_workloads import plan_spots
    spots = plan_spots(6, 30_000, seed=4, e_range=(70.0, 110.0), pitch=5.0, half_width=10.0)
    wl = water100(30_000)
    with sde_gpu.SdeDose(wl) as d:
        if graph:
            d.set_tuning(graph=graph)
        d.run(spots, seed=5)
        _, ref, rb = d.fetch(dose=False)
        d.reset()
        total = int(spots["n_hist"].sum())
        for r in range(3):
            first, count = sde_gpu.history_shard(total, r, 3)
            d.run(spots, seed=5, first=first, count=count)
        d.run(spots, seed=5, first=total, count=100)
        _, e, b = d.fetch(dose=False)
        assert np.array_equal(e, ref) and b == rb
        # the same shards with device-resident spots (the path the benchmark times)
        import torch
        raw = torch.from_numpy(spots.view(np.uint8).copy()).cuda()
        d.reset()
        for r in range(3):
            first, count = sde_gpu.history_shard(total, r, 3)
            d.run_device(raw.data_ptr(), len(spots), seed=5, first=first, count=count)
        _, e, b = d.fetch(dose=False)
        assert np.array_equal(e, ref) and b == rb
        d.reset()
        d.run(spots, seed=5, first=total - 10, count=10**12)
        _, e, b = d.fetch(dose=False)
        assert b["histories"] == 10 and b["incident"] == b["deposited"] + b["escaped"] + b["removed"]


def test_ct_sobp_dose_parity(sde_gpu, oracle_lib):
    """Thorax-like synthetic CT (air outside and in the airway, lung, adipose, soft tissue,
    cortical bone; HU -> density and material) under a 16-layer spread-out Bragg peak, at
    2 mm voxels: GPU and oracle doses agree voxel by voxel, with exact balance."""
    from sde_workloads import ct_sobp
    wl = ct_sobp(1000, seed=2, shape=(60, 60, 120), h=2.0)
    n = 192_000
    g, bals = _gpu_batches(sde_gpu, wl, n, range(B))
    o = _oracle_batches(wl, n, range(100, 100 + B))
    rho = wl.density.astype(np.float64)
    # Energy per voxel (dose x density) over the whole grid; dose-to-medium where the
    # medium is not air: in air (1.2 mg/cm^3) a rare deposit divided by a tiny mass gives a
    # heavy-tailed dose whose batch standard error is not a usable scale.
    for name, a, b in (("energy", g * rho, o * rho), ("dose, rho > 0.05", g * (rho > 0.05), o * (rho > 0.05))):
        c = compare(a, b)
        print(name, {k: v for k, v in c.items() if not k.startswith("mean_")}, c["mean_z2"])
        assert c["pass_frac"] >= 0.985, (name, c)
        assert 0.6 < c["mean_z2"] < 1.5, (name, c)
    assert all(b["escaped"] > 0 for b in bals)  # lateral and distal escape through air


def test_sobp_plateau_in_water(sde_gpu):
    """The 16-layer spread-out Bragg peak in water (Bragg-Kleeman energies, Bortfeld-Schlegel
    layer weights): the depth dose is flat over the modulated depths."""
    from sde_workloads import sobp_water
    wl = sobp_water(2_000_000)
    _, edep, bal = sde_gpu.run_workload(wl, seed=1)
    assert balanced(bal)
    idd = A.idd(edep.astype(float))
    z = A.z_centres(200, 1.0)
    pl = (z >= 96) & (z <= 132)
    ratio = idd[pl].max() / idd[pl].min()
    print("SOBP plateau max/min", ratio, "R90", A.distal_range(idd, z, 0.9))
    assert ratio < 1.10
    # the distal 90 % level sits a few mm short of the deepest layer's nominal 140 mm range
    # (energy spread and straggling soften the edge of the top layer, which carries 1/6 of
    # the fluence)
    assert 130.0 < A.distal_range(idd, z, 0.9) < 142.0


def test_insert150_gamma_at_one_million_protons(sde_gpu, oracle_lib):
    """Insert phantom: 3D gamma (2 %/0.5 mm, local, 1 % threshold) of the GPU dose against the
    oracle at 10^6 protons.  Both doses are noisy, so the pass rate is compared with the pass
    rate of the oracle against itself (another seed): equal distributions give equal rates."""
    wl = insert150(1_000_000)
    dg, eg, bg = sde_gpu.run_workload(wl, seed=21)
    do1, _, bo = O.run_workload(wl, seed=22)
    do2, _, _ = O.run_workload(wl, seed=23)
    assert balanced(bg) and balanced(bo)
    g_go = A.gamma_pass_rate(do1, dg, wl.voxel_mm)
    g_oo = A.gamma_pass_rate(do1, do2, wl.voxel_mm)
    print({"gamma_gpu_vs_oracle": g_go, "gamma_oracle_vs_oracle": g_oo})
    assert g_go > 0.9
    assert abs(g_go - g_oo) < 0.01
