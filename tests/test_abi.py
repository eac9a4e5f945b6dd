"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, exports every
symbol declared in include/*.h, and rejects bad arguments on the host before touching
the device.  No compute call is made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sde():
    from paper_2511_03115_gb300 import _build
    _build.build()
    import paper_2511_03115_gb300 as S
    S.lib()
    return S


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"\b(sde_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("sde_dose_create", "sde_dose_run", "sde_dose_fetch", "sde_dose_destroy", "sde_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(sde):
    L = sde.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(sde.EXPORTED) == _declared_functions()


def test_default_params_are_the_papers(sde):
    p = sde.default_params()
    assert p.step_cm == 0.05 and p.msc_z_cm == 0.05 and p.F == 0.98
    assert p.theta_cut_rad == 0.02 and p.backscatter_rad == 0.04 and p.e_min_MeV == 0.05
    assert p.K == 0.3072 and p.tally_mode == 0 and p.fixed_point_shift == 24
    assert p.physics_mask == sde.PHYS_ALL


def _create(sde, nx=2, ny=2, nz=2, dens=None, mid=None, mats=None, params=None):
    L = sde.lib()
    n = nx * ny * nz
    dens = np.ones(max(n, 1), np.float32) if dens is None else dens
    mid = np.zeros(max(n, 1), np.uint8) if mid is None else mid
    mats = mats if mats is not None else [{"elements": [(1, 0.1119), (8, 0.8881)], "I_eV": 75.0}]
    m = sde._Materials(mats)
    h = C.c_void_p()
    p = params if params is not None else sde.default_params()
    rc = L.sde_dose_create(C.byref(h), nx, ny, nz, (C.c_double * 3)(1, 1, 1), (C.c_double * 3)(0, 0, 0),
                           dens.ctypes.data, mid.ctypes.data, m.arr, len(mats), C.byref(p))
    return rc, L.sde_last_error().decode()


def test_create_rejects_bad_arguments_on_the_host(sde):
    assert _create(sde, nx=0)[0] == sde.SDE_EINVAL
    rc, msg = _create(sde, mid=np.full(8, 3, np.uint8))
    assert rc == sde.SDE_EINVAL and "material id" in msg
    rc, msg = _create(sde, dens=np.full(8, -1.0, np.float32))
    assert rc == sde.SDE_EINVAL and "density" in msg
    rc, msg = _create(sde, mats=[{"elements": [(99, 1.0)], "I_eV": 0.0}])
    assert rc == sde.SDE_EINVAL and "Z=99" in msg
    rc, msg = _create(sde, params=sde.default_params(F=1.5))
    assert rc == sde.SDE_EINVAL and "params" in msg
    rc, msg = _create(sde, params=sde.default_params(table_points=8))
    assert rc == sde.SDE_EINVAL


@pytest.mark.parametrize("bad", [dict(theta_cut_sigmas=-1.0), dict(e_max_MeV=1500.0),
                                 dict(fixed_point_shift=31), dict(step_cm=2.0), dict(physics_mask=16),
                                 dict(tally_mode=2), dict(max_steps=0), dict(km_r=1.0)])
def test_params_outside_their_ranges_are_rejected_on_the_host(sde, bad):
    # the fixed-point tally relies on E <= 1000 MeV and S <= 30 (every Q(E) below 2^40)
    rc, msg = _create(sde, params=sde.default_params(**bad))
    assert rc == sde.SDE_EINVAL and "params" in msg, bad


def test_energy_dependent_cut_off_is_off_by_default(sde):
    assert sde.default_params().theta_cut_sigmas == 0.0


def test_null_handle_calls_fail_cleanly(sde):
    L = sde.lib()
    assert L.sde_dose_run(None, None, 0, 0) == sde.SDE_EINVAL
    assert L.sde_dose_fetch(None, None, None, None) == sde.SDE_EINVAL
    assert L.sde_dose_reset(None) == sde.SDE_EINVAL
    assert L.sde_dose_set_tuning(None, None) == sde.SDE_EINVAL
    assert L.sde_dose_run_range(None, None, 0, 0, 0, 0) == sde.SDE_EINVAL
    assert L.sde_dose_run_device_range(None, None, 0, 0, 0, 0) == sde.SDE_EINVAL
    assert L.sde_dose_fetch_device_f32(None, None) == sde.SDE_EINVAL
    L.sde_dose_destroy(None)


def test_spot_record_layout(sde):
    from sde_workloads import SPOT_DTYPE
    assert SPOT_DTYPE.itemsize == C.sizeof(sde.Spot) == 88
    for name, _ in sde.Spot._fields_:
        assert getattr(sde.Spot, name).offset == SPOT_DTYPE.fields[name][1]


def test_binding_fails_loudly_without_the_library(sde, tmp_path, monkeypatch):
    import paper_2511_03115_gb300 as S
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(S.SdeError):
        S.lib()
