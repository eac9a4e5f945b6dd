"""The transport entry point that allocates nothing (sde_transport_noalloc), checked
against the handle-based entry point on the same inputs.

Callers inside a framework that owns every device allocation through its own pool, or
services that must not allocate after start-up, use this call: it keeps its tables,
spot records, prefix and counters in a fixed device array compiled into the library.
This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from sde_workloads import slab150, water100

pytestmark = pytest.mark.gpu

ERR_STEP_CAP, ERR_BAD_SPOT, ERR_BAD_VOXEL = 1, 2, 8


def _packed_voxels(wl):
    """The documented voxel word: ((bits(density) + 8) & ~15) | material id."""
    bits = np.ascontiguousarray(wl.density, np.float32).view(np.uint32).ravel()
    mid = np.ascontiguousarray(wl.material_id).ravel().astype(np.uint32)
    return ((bits + np.uint32(8)) & np.uint32(0xFFFFFFF0)) | mid


def _call(S, wl, vox, spots, out, seed, bal=None, n_spots=None, mats=None, status=None, **param_kw):
    L = S.lib()
    nx, ny, nz = wl.shape
    m = S._Materials(wl.materials if mats is None else mats)
    p = S.default_params(**param_kw)
    return L.sde_transport_noalloc(nx, ny, nz, (C.c_double * 3)(*wl.voxel_mm), (C.c_double * 3)(*wl.origin_mm),
                                   vox.data_ptr(), m.arr, len(m._keep), C.byref(p), spots.data_ptr(),
                                   len(wl.spots) if n_spots is None else n_spots, C.c_uint64(seed),
                                   out.data_ptr(), C.byref(bal) if bal is not None else None,
                                   status.data_ptr() if status is not None else None, None)


def test_noalloc_transport_matches_the_handle_path_on_two_calls_in_a_row(sde_gpu):
    import torch
    S = sde_gpu
    wl = slab150(40_000)
    vox = torch.from_numpy(_packed_voxels(wl).view(np.int32)).cuda()
    spots = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    for seed in (3, 4):
        out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
        bal = S.Balance()
        rc = _call(S, wl, vox, spots, out, seed, bal)
        assert rc == S.SDE_OK, S.lib().sde_last_error().decode()
        with S.SdeDose(wl) as d:
            d.run_device(spots.data_ptr(), len(wl.spots), seed=seed)
            _, ref, ref_bal = d.fetch(dose=False)
        got = out.cpu().numpy().view(np.uint64)
        # same kernels, tables and random streams: the tally is bit-identical
        assert np.array_equal(got, ref.ravel())
        assert bal.as_dict() == ref_bal
        assert ref_bal["incident"] == ref_bal["deposited"] + ref_bal["escaped"] + ref_bal["removed"]


def test_noalloc_balance_is_per_call_on_an_accumulating_tally(sde_gpu):
    """The tally is added to; the balance of each call is that call's own, so it stays exact
    when the caller accumulates several calls in one buffer."""
    import torch
    S = sde_gpu
    wl = water100(5000)
    vox = torch.from_numpy(_packed_voxels(wl).view(np.int32)).cuda()
    spots = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 0x55, dtype=torch.int32, device="cuda")
    deposited = 0
    for seed in (1, 2):
        bal = S.Balance()
        assert _call(S, wl, vox, spots, out, seed, bal, status=status) == S.SDE_OK
        b = bal.as_dict()
        assert b["histories"] == 5000 and b["incident"] == b["deposited"] + b["escaped"] + b["removed"]
        deposited += b["deposited"]
        assert int(status.item()) == 0
    assert int(out.cpu().numpy().view(np.uint64).sum(dtype=np.uint64)) == deposited


def test_noalloc_rejects_bad_voxel_words_on_the_device(sde_gpu):
    """A material id >= n_mats (or a bad density) in the caller's voxel words is caught before
    any table is read with it: no history runs, the tally is untouched, and the error is
    reported through the balance call and through the status word of a call without one."""
    import torch
    S = sde_gpu
    wl = water100(2000)
    words = _packed_voxels(wl)
    bad_id = words.copy()
    bad_id[12345] = (bad_id[12345] & np.uint32(0xFFFFFFF0)) | np.uint32(7)  # id 7 with n_mats = 1
    bad_rho = words.copy()
    bad_rho[777] = np.float32(np.nan).view(np.uint32) & np.uint32(0xFFFFFFF0)
    spots = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    for w in (bad_id, bad_rho):
        vox = torch.from_numpy(w.view(np.int32)).cuda()
        out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
        bal = S.Balance()
        rc = _call(S, wl, vox, spots, out, 0, bal)
        assert rc == S.SDE_EDEVICE and "voxel word" in S.lib().sde_last_error().decode()
        assert bal.histories == 0 and bal.incident == 0 and int(out.abs().sum()) == 0
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert _call(S, wl, vox, spots, out, 0, status=status) == S.SDE_OK  # asynchronous: no balance
        torch.cuda.synchronize()
        assert int(status.item()) & ERR_BAD_VOXEL and int(out.abs().sum()) == 0


def test_noalloc_status_word_reports_an_invalid_spot_without_a_balance(sde_gpu):
    import torch
    S = sde_gpu
    wl = water100(100)
    vox = torch.from_numpy(_packed_voxels(wl).view(np.int32)).cuda()
    bad = wl.spots.copy()
    bad["E_MeV"] = -5.0
    spots = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call(S, wl, vox, spots, out, 0, status=status) == S.SDE_OK
    torch.cuda.synchronize()
    assert int(status.item()) == ERR_BAD_SPOT and int(out.abs().sum()) == 0
    # the next good call clears the flag
    good = torch.from_numpy(wl.spots.view(np.uint8).copy()).cuda()
    assert _call(S, wl, vox, good, out, 0, status=status) == S.SDE_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(out.sum()) > 0


def test_noalloc_rejects_inputs_beyond_its_scratch_limits(sde_gpu):
    import torch
    S = sde_gpu
    wl = water100(10)
    vox = torch.from_numpy(_packed_voxels(wl).view(np.int32)).cuda()
    spots = torch.from_numpy(np.repeat(wl.spots, 4097).view(np.uint8).copy()).cuda()
    out = torch.zeros(wl.n_voxels, dtype=torch.int64, device="cuda")
    rc = _call(S, wl, vox, spots, out, 0, n_spots=4097)
    assert rc == S.SDE_EINVAL and "4096" in S.lib().sde_last_error().decode()
    rc = _call(S, wl, vox, spots, out, 0, n_spots=1, mats=[wl.materials[0]] * 5)
    assert rc == S.SDE_EINVAL and "n_mats" in S.lib().sde_last_error().decode()
    rc = _call(S, wl, vox, spots, out, 0, n_spots=1, theta_cut_sigmas=2.5)  # needs a handle's tables
    assert rc == S.SDE_EINVAL and "cut-off" in S.lib().sde_last_error().decode()
    assert int(out.abs().sum()) == 0
