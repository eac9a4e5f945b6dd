"""The transport entry point that allocates nothing (sde_transport_noalloc), checked
against the handle-based entry point on the same inputs.

Callers inside a framework that owns every device allocation, or that must not
allocate while a CUDA graph is being built or after start-up, use this call: it keeps
its tables, spot records, prefix and counters in a fixed device array compiled into the
library.  This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from sde_workloads import slab150, water100

pytestmark = pytest.mark.gpu


def _packed_voxels(wl):
    """The documented voxel word: ((bits(density) + 8) & ~15) | material id."""
    bits = np.ascontiguousarray(wl.density, np.float32).view(np.uint32).ravel()
    mid = np.ascontiguousarray(wl.material_id).ravel().astype(np.uint32)
    return ((bits + np.uint32(8)) & np.uint32(0xFFFFFFF0)) | mid


def _call(S, wl, vox, spots, out, seed, bal=None, n_spots=None, mats=None, **param_kw):
    L = S.lib()
    nx, ny, nz = wl.shape
    m = S._Materials(wl.materials if mats is None else mats)
    p = S.default_params(**param_kw)
    return L.sde_transport_noalloc(nx, ny, nz, (C.c_double * 3)(*wl.voxel_mm), (C.c_double * 3)(*wl.origin_mm),
                                   vox.data_ptr(), m.arr, len(m._keep), C.byref(p), spots.data_ptr(),
                                   len(wl.spots) if n_spots is None else n_spots, C.c_uint64(seed),
                                   out.data_ptr(), C.byref(bal) if bal is not None else None, None)


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
