"""Python handle on the FP64 CPU oracle (``sde_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, direct evaluation of
the jump-SDE proton transport of arXiv 2511.03115 (Eq. VSDE with the
parameterisations of Secs. 2.1.3-2.1.5).  Only ``tests/``, the smoke check and
the benchmark's CPU-baseline leg may import this package; the CUDA library
and its Python binding never do.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sde_oracle.c")
_HDR = os.path.join(_HERE, "sde_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libsde_oracle.so")
_lock = threading.Lock()
_lib = None

PHYS_STRAGGLING, PHYS_MCS, PHYS_ELASTIC, PHYS_INELASTIC, PHYS_ALL = 1, 2, 4, 8, 15


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host code only; no GPU involved)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = force or not os.path.exists(_OUT) or any(
        os.path.getmtime(f) > os.path.getmtime(_OUT) for f in (_SRC, _HDR))
    if stale:
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", _SRC, "-lm", "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class ElementFrac(C.Structure):
    _fields_ = [("Z", C.c_int), ("mass_fraction", C.c_double)]


class Material(C.Structure):
    _fields_ = [("el", C.POINTER(ElementFrac)), ("n_el", C.c_int), ("I_eV", C.c_double)]


class Spot(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E_MeV", "sigma_E_MeV", "x_mm", "y_mm", "z_mm", "ux",
                                          "uy", "uz", "sigma_xy_mm", "sigma_angle_rad")] + [
        ("n_hist", C.c_uint64)]


class Params(C.Structure):
    _fields_ = [("step_cm", C.c_double), ("msc_z_cm", C.c_double), ("F", C.c_double),
                ("theta_cut_rad", C.c_double), ("backscatter_rad", C.c_double),
                ("e_min_MeV", C.c_double), ("K", C.c_double), ("inel_u_lo", C.c_double),
                ("inel_u_hi", C.c_double), ("km_r", C.c_double), ("tally_mode", C.c_int),
                ("fixed_point_shift", C.c_int), ("jump_clock", C.c_int), ("max_steps", C.c_int),
                ("physics_mask", C.c_int), ("theta_cut_sigmas", C.c_double),
                ("secondary_fraction", C.c_double)]


class Balance(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("incident", "deposited", "escaped", "removed",
                                          "histories", "steps", "jumps_elastic",
                                          "jumps_inelastic")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


MAX_EL = 16


class PhysicsOut(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("beta2", "gamma", "p_MeV", "I_eV", "s1", "s2sq", "chi_c2",
                                          "chi_a2", "w", "sigma_msc", "t_sbm", "sig_e",
                                          "sig_ne", "theta_cut")] + [
        ("n_el", C.c_int), ("sig_e_el", C.c_double * MAX_EL), ("sig_ne_el", C.c_double * MAX_EL)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, i, d, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
            L.oracle_default_params.argtypes = [C.POINTER(Params)]
            L.oracle_last_error.restype = C.c_char_p
            L.oracle_set_threads.argtypes = [i]
            L.oracle_create.argtypes = [C.POINTER(dp), i, i, i, C.POINTER(d), C.POINTER(d), dp, dp,
                                        C.POINTER(Material), i, C.POINTER(Params)]
            L.oracle_run.argtypes = [dp, C.POINTER(Spot), i, u64]
            L.oracle_run_range.argtypes = [dp, C.POINTER(Spot), i, u64, u64, u64]
            L.oracle_fetch.argtypes = [dp, dp, dp, C.POINTER(Balance)]
            L.oracle_reset.argtypes = [dp]
            L.oracle_destroy.argtypes = [dp]
            L.oracle_destroy.restype = None
            L.oracle_philox4x32_10.argtypes = [dp, dp, dp]
            L.oracle_philox4x32_10.restype = None
            L.oracle_element.argtypes = [i, C.POINTER(d), C.POINTER(d)]
            L.oracle_physics.argtypes = [C.POINTER(Material), d, C.POINTER(Params), d,
                                         C.POINTER(PhysicsOut)]
            L.oracle_csda_range.argtypes = [C.POINTER(Material), d, C.POINTER(Params), d,
                                            C.POINTER(d)]
            L.oracle_single_step_secondary.argtypes = [C.POINTER(Material), d, C.POINTER(Params), d, u64, u64,
                                                       i, dp]
            L.oracle_sample_source.argtypes = [C.POINTER(Spot), C.POINTER(Params), u64, u64, i, dp, dp, dp]
            L.oracle_single_step.argtypes = [C.POINTER(Material), d, C.POINTER(Params), d, u64, u64,
                                             i, dp, dp, dp, dp, dp]
            for name, nargs in (("oracle_sample_mu_rutherford", 2), ("oracle_sample_mu_mott", 4),
                                ("oracle_mott_antiderivative", 2), ("oracle_mott_dsigma", 3),
                                ("oracle_rutherford_dsigma", 3), ("oracle_sample_mu_kalbach", 3),
                                ("oracle_kalbach_a", 3), ("oracle_cm_to_lab", 4)):
                f = getattr(L, name)
                f.argtypes = [d] * nargs
                f.restype = d
            L.oracle_coulomb_eta_k.argtypes = [i, d, C.POINTER(d), C.POINTER(d)]
            L.oracle_sigma_ne_element_mb.argtypes = [i, d]
            L.oracle_sigma_ne_element_mb.restype = d
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {lib().oracle_last_error().decode()}")


def params(**kw) -> Params:
    p = Params()
    lib().oracle_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class _MaterialBlock:
    """Keeps the ctypes element arrays alive for the material structs."""

    def __init__(self, materials):
        self._keep = []
        self.arr = (Material * len(materials))()
        for i, m in enumerate(materials):
            els = (ElementFrac * len(m["elements"]))(*[ElementFrac(z, w) for z, w in m["elements"]])
            self._keep.append(els)
            self.arr[i] = Material(C.cast(els, C.POINTER(ElementFrac)), len(m["elements"]),
                                   float(m.get("I_eV", 0.0)))


def _spots(spots: np.ndarray):
    arr = (Spot * len(spots))()
    for i, s in enumerate(spots):
        arr[i] = Spot(*[float(s[n]) for n in spots.dtype.names[:-1]], int(s["n_hist"]))
    return arr


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


class OracleDose:
    """Oracle dose engine with the same call shape as the CUDA library."""

    def __init__(self, wl, **param_kw):
        L = lib()
        self.wl = wl
        self.shape = wl.shape
        self._dens = np.ascontiguousarray(wl.density, dtype=np.float32)
        self._mid = np.ascontiguousarray(wl.material_id, dtype=np.uint8)
        self._mats = _MaterialBlock(wl.materials)
        self.params = params(**param_kw)
        h = C.c_void_p()
        vox = (C.c_double * 3)(*wl.voxel_mm)
        org = (C.c_double * 3)(*wl.origin_mm)
        nx, ny, nz = wl.shape
        _check(L.oracle_create(C.byref(h), nx, ny, nz, vox, org, self._dens.ctypes.data,
                               self._mid.ctypes.data, self._mats.arr, len(wl.materials),
                               C.byref(self.params)))
        self.h = h

    def run(self, spots=None, seed=None, first=None, count=None):
        """Transport the plan (or, with first/count, the histories with global ids in
        [first, first + count))."""
        spots = self.wl.spots if spots is None else spots
        seed = self.wl.seed if seed is None else seed
        arr = _spots(spots)
        if first is None and count is None:
            _check(lib().oracle_run(self.h, arr, len(spots), C.c_uint64(seed)))
        else:
            _check(lib().oracle_run_range(self.h, arr, len(spots), C.c_uint64(seed), C.c_uint64(first or 0),
                                          C.c_uint64(2**64 - 1 if count is None else count)))

    def fetch(self):
        nx, ny, nz = self.shape
        dose = np.empty((nz, ny, nx), np.float64)
        edep = np.empty((nz, ny, nx), np.uint64)
        bal = Balance()
        _check(lib().oracle_fetch(self.h, dose.ctypes.data, edep.ctypes.data, C.byref(bal)))
        return dose, edep, bal.as_dict()

    def reset(self):
        _check(lib().oracle_reset(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_workload(wl, seed=None, threads=0, **param_kw):
    """Run a workload on the oracle; returns (dose_Gy, edep_fixed, balance)."""
    if threads:
        set_threads(threads)
    d = OracleDose(wl, **param_kw)
    try:
        d.run(seed=seed)
        return d.fetch()
    finally:
        d.close()


# ------------------------------------------------------------------ probes
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(C.cast(c, C.c_void_p), C.cast(k, C.c_void_p), C.cast(o, C.c_void_p))
    return [int(x) for x in o]


def element(Z):
    A, I = C.c_double(), C.c_double()
    _check(lib().oracle_element(Z, C.byref(A), C.byref(I)))
    return A.value, I.value


def physics(material, rho, E, **param_kw) -> PhysicsOut:
    blk = _MaterialBlock([material])
    out = PhysicsOut()
    p = params(**param_kw)
    _check(lib().oracle_physics(blk.arr, float(rho), C.byref(p), float(E), C.byref(out)))
    return out


def csda_range(material, rho, E0, **param_kw) -> float:
    blk = _MaterialBlock([material])
    p = params(**param_kw)
    r = C.c_double()
    _check(lib().oracle_csda_range(blk.arr, float(rho), C.byref(p), float(E0), C.byref(r)))
    return r.value


def single_step(material, rho, E, n, seed=0, h0=0, **param_kw):
    blk = _MaterialBlock([material])
    p = params(**param_kw)
    E_out = np.empty(n)
    cos_out = np.empty(n)
    jump = np.empty(n, np.int32)
    ux = np.empty(n)
    uy = np.empty(n)
    _check(lib().oracle_single_step(blk.arr, float(rho), C.byref(p), float(E), C.c_uint64(seed),
                                    C.c_uint64(h0), int(n), E_out.ctypes.data, cos_out.ctypes.data,
                                    jump.ctypes.data, ux.ctypes.data, uy.ctypes.data))
    return {"E": E_out, "cos": cos_out, "jump": jump, "ux": ux, "uy": uy}


def single_step_secondary(material, rho, E, n, seed=0, h0=0, **param_kw):
    """One step per history with the branching model's emission (see the C header)."""
    blk = _MaterialBlock([material])
    p = params(**param_kw)
    out = np.empty((n, 10))
    _check(lib().oracle_single_step_secondary(blk.arr, float(rho), C.byref(p), float(E), C.c_uint64(seed),
                                              C.c_uint64(h0), int(n), out.ctypes.data))
    keys = ("jump", "E1", "E2", "spawn", "sec_E", "sec_ux", "sec_uy", "sec_uz", "ux", "uy")
    return {k: out[:, i] for i, k in enumerate(keys)}


def sample_source(spot, n, seed=0, h0=0, **param_kw):
    """Y_0 of n histories of one spot (a numpy spot record): energy, entry point, direction."""
    arr = _spots(np.asarray([spot], dtype=spot.dtype) if hasattr(spot, "dtype") else spot)
    p = params(**param_kw)
    E = np.empty(n)
    r = np.empty((n, 3))
    u = np.empty((n, 3))
    _check(lib().oracle_sample_source(arr, C.byref(p), C.c_uint64(seed), C.c_uint64(h0), int(n),
                                      E.ctypes.data, r.ctypes.data, u.ctypes.data))
    return E, r, u


def coulomb_eta_k(Z, E):
    eta, k = C.c_double(), C.c_double()
    _check(lib().oracle_coulomb_eta_k(Z, float(E), C.byref(eta), C.byref(k)))
    return eta.value, k.value


def fn(name):
    """A scalar probe function of the oracle by name (samplers, laws, kinematics)."""
    return getattr(lib(), name)
