"""Python binding of the GB300 jump-SDE proton dose engine (``libsde_dose.so``).

Argument marshalling only: every step of the transport runs in the library's
CUDA kernels.  The C functions keep their names (``sde_dose_create``,
``sde_dose_run``, ``sde_dose_fetch`` ...; see ``include/sde_dose.h``); the
``SdeDose`` class wraps a handle for numpy / torch callers.  Importing this
package does not build or load anything; the first call that needs the
library loads it and raises ``SdeError`` if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SDE_DOSE_LIB") or os.path.join(_PKG, "_lib", "libsde_dose.so")
_lock = threading.Lock()
_lib = None

SDE_OK, SDE_EINVAL, SDE_ENOMEM, SDE_ECUDA, SDE_EDEVICE = 0, -1, -2, -3, -4
PHYS_STRAGGLING, PHYS_MCS, PHYS_ELASTIC, PHYS_INELASTIC, PHYS_ALL = 1, 2, 4, 8, 15
MAX_ELEMENTS = 16

EXPORTED = [
    "sde_default_params", "sde_last_error", "sde_dose_create", "sde_dose_set_stream",
    "sde_dose_set_tuning", "sde_dose_get_tuning", "sde_dose_autotune", "sde_dose_run", "sde_dose_run_range",
    "sde_dose_run_device", "sde_dose_run_device_range",
    "sde_dose_sync", "sde_dose_fetch", "sde_dose_fetch_device", "sde_dose_fetch_device_f32", "sde_dose_reset",
    "sde_dose_destroy", "sde_dose_info", "sde_dose_tables", "sde_dose_probe_steps",
    "sde_transport_noalloc", "sde_gemm_bf16", "sde_conv3d_forward", "sde_conv3d_wgrad",
    "sde_conv3d_flip_weights", "sde_denoise_status", "sde_denoiser_create", "sde_denoiser_destroy",
    "sde_denoiser_set_stream", "sde_denoiser_num_params", "sde_denoiser_infer", "sde_denoiser_train_step",
    "sde_denoiser_gradients", "sde_denoiser_get_params", "sde_denoiser_set_params", "sde_gamma3d",
    "sde_scale_f32", "sde_conv3d_plan", "sde_conv3d_wgrad_plan",
]


def history_shard(total: int, rank: int, world: int):
    """(first, count) of the contiguous block of global history ids that rank ``rank`` of
    ``world`` transports when one plan of ``total`` histories is split across GPUs: the
    blocks are disjoint, cover [0, total) and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    first = total * rank // world
    return first, total * (rank + 1) // world - first


BALANCE_KEYS = ("incident", "deposited", "escaped", "removed", "histories", "steps", "jumps_elastic",
                "jumps_inelastic")


def combine_shards(tally, balance, group=None):
    """The one exchange step of a plan split across GPUs by global history id: an exact
    integer sum over the ranks of the 64-bit tallies and of the balance counters.

    ``tally`` is this rank's tally as a torch int64 tensor (the library's unsigned words
    viewed as signed: two's-complement addition gives the same bits as unsigned addition
    modulo 2^64), on the rank's GPU for NCCL or on the CPU for gloo; it is summed in place.
    ``balance`` is this rank's balance dict.  Integer addition is exact and does not
    depend on the order of the ranks, so the result is the single-GPU run's bit for bit.
    Returns the summed balance (counters must stay below 2^63, i.e. < 5.5e11 MeV of
    incident energy at the default 2^-24 MeV unit)."""
    import torch
    import torch.distributed as dist
    b = torch.tensor([int(balance[k]) for k in BALANCE_KEYS], dtype=torch.int64, device=tally.device)
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
    return {k: int(v) for k, v in zip(BALANCE_KEYS, b.tolist())}


class SdeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sde error {code}: {msg}")
        self.code = code


class ElementFrac(C.Structure):
    _fields_ = [("Z", C.c_int), ("mass_fraction", C.c_double)]


class Material(C.Structure):
    _fields_ = [("el", C.POINTER(ElementFrac)), ("n_el", C.c_int), ("I_eV", C.c_double)]


class Spot(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E_MeV", "sigma_E_MeV", "x_mm", "y_mm", "z_mm", "ux",
                                          "uy", "uz", "sigma_xy_mm", "sigma_angle_rad")] + [
        ("n_hist", C.c_uint64)]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("step_cm", "msc_z_cm", "F", "theta_cut_rad",
                                          "backscatter_rad", "e_min_MeV", "K", "inel_u_lo",
                                          "inel_u_hi", "km_r", "e_max_MeV")] + [
        (n, C.c_int) for n in ("tally_mode", "fixed_point_shift", "max_steps", "physics_mask",
                               "table_points")] + [("theta_cut_sigmas", C.c_double),
                                                   ("secondary_fraction", C.c_double)]


class Balance(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("incident", "deposited", "escaped", "removed",
                                          "histories", "steps", "jumps_elastic",
                                          "jumps_inelastic")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int), ("warps_per_block", C.c_int), ("batch", C.c_int),
                ("refill_min", C.c_int), ("table_smem", C.c_int), ("aggregate", C.c_int), ("graph", C.c_int)]


assert C.sizeof(Spot) == 88


def lib():
    """Load ``libsde_dose.so`` (raises SdeError when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise SdeError(SDE_ECUDA, f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i, d, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
        L.sde_default_params.argtypes = [C.POINTER(Params)]
        L.sde_last_error.restype = C.c_char_p
        L.sde_dose_create.argtypes = [C.POINTER(vp), i, i, i, C.POINTER(d), C.POINTER(d), vp, vp,
                                      C.POINTER(Material), i, C.POINTER(Params)]
        L.sde_dose_set_stream.argtypes = [vp, vp]
        L.sde_dose_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.sde_dose_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.sde_dose_autotune.argtypes = [vp, C.POINTER(Spot), i, u64, u64, C.POINTER(Tuning)]
        L.sde_dose_run.argtypes = [vp, C.POINTER(Spot), i, u64]
        L.sde_dose_run_range.argtypes = [vp, C.POINTER(Spot), i, u64, u64, u64]
        L.sde_dose_run_device.argtypes = [vp, vp, i, u64]
        L.sde_dose_run_device_range.argtypes = [vp, vp, i, u64, u64, u64]
        L.sde_dose_sync.argtypes = [vp]
        L.sde_dose_fetch.argtypes = [vp, vp, vp, C.POINTER(Balance)]
        L.sde_dose_fetch_device.argtypes = [vp, vp, vp, C.POINTER(Balance)]
        L.sde_dose_fetch_device_f32.argtypes = [vp, vp]
        L.sde_dose_reset.argtypes = [vp]
        L.sde_dose_destroy.argtypes = [vp]
        L.sde_dose_destroy.restype = None
        L.sde_dose_info.argtypes = [vp, C.POINTER(u64), C.POINTER(i), C.POINTER(d), C.POINTER(d),
                                    C.POINTER(i)]
        L.sde_dose_tables.argtypes = [vp, i, vp, vp, vp]
        L.sde_dose_probe_steps.argtypes = [vp, i, d, d, u64, u64, i, vp, vp, vp, vp, vp]
        L.sde_transport_noalloc.argtypes = [i, i, i, C.POINTER(d), C.POINTER(d), vp, C.POINTER(Material), i,
                                            C.POINTER(Params), vp, i, u64, vp, C.POINTER(Balance), vp, vp]
        L.sde_gemm_bf16.argtypes = [vp, vp, vp, i, i, i, vp]
        L.sde_conv3d_forward.argtypes = [vp, i, i, i, i, i, vp, vp, i, vp, i, i, i, i, vp]
        L.sde_conv3d_wgrad.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp]
        L.sde_conv3d_flip_weights.argtypes = [vp, vp, i, i, vp]
        L.sde_conv3d_plan.argtypes = [i, i, i, i, i, i, C.POINTER(C.c_int32), i, C.POINTER(u64)]
        L.sde_conv3d_wgrad_plan.argtypes = [i, i, i, i, i, i, i, C.POINTER(C.c_int32), i, C.POINTER(u64)]
        L.sde_denoise_status.argtypes = [vp]
        L.sde_denoiser_create.argtypes = [C.POINTER(vp), i, i, i, i, u64]
        L.sde_denoiser_destroy.argtypes = [vp]
        L.sde_denoiser_destroy.restype = None
        L.sde_denoiser_set_stream.argtypes = [vp, vp]
        L.sde_denoiser_num_params.argtypes = [vp, C.POINTER(u64)]
        L.sde_denoiser_infer.argtypes = [vp, vp, vp, i, vp]
        L.sde_denoiser_train_step.argtypes = [vp, vp, vp, vp, C.c_float, i, C.c_float, C.POINTER(C.c_float)]
        L.sde_denoiser_gradients.argtypes = [vp, vp, vp, vp, C.c_float, i, vp, u64, C.POINTER(C.c_float)]
        L.sde_scale_f32.argtypes = [vp, u64, C.c_float, vp]
        L.sde_denoiser_get_params.argtypes = [vp, vp, u64]
        L.sde_denoiser_set_params.argtypes = [vp, vp, u64]
        L.sde_gamma3d.argtypes = [vp, vp, i, i, i, C.POINTER(d), d, d, d, i, C.POINTER(u64), C.POINTER(u64), vp]
        _lib = L
        return L


def _check(rc):
    if rc != SDE_OK:
        raise SdeError(rc, lib().sde_last_error().decode())


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().sde_default_params(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class _Materials:
    def __init__(self, materials):
        self._keep = []
        self.arr = (Material * len(materials))()
        for n, m in enumerate(materials):
            els = (ElementFrac * len(m["elements"]))(*[ElementFrac(z, w) for z, w in m["elements"]])
            self._keep.append(els)
            self.arr[n] = Material(C.cast(els, C.POINTER(ElementFrac)), len(m["elements"]),
                                   float(m.get("I_eV", 0.0)))


def spots_to_ctypes(spots: np.ndarray):
    """A numpy structured spot array (88-byte records) viewed as ``Spot`` records."""
    a = np.ascontiguousarray(spots)
    if a.dtype.itemsize != C.sizeof(Spot):
        raise ValueError("spot records must be 88 bytes (10 float64 + uint64)")
    return a, C.cast(a.ctypes.data, C.POINTER(Spot))


class SdeDose:
    """One engine handle: phantom, tables and tally on the current CUDA device.

    ``wl`` is a workload with ``shape`` (nx, ny, nz), ``voxel_mm``, ``origin_mm``,
    ``density`` / ``material_id`` (x-fastest, shape (nz, ny, nx)), ``materials``.
    """

    def __init__(self, wl, stream=None, tuning=None, **param_kw):
        L = lib()
        self.shape = tuple(wl.shape)
        self.wl = wl
        dens = np.ascontiguousarray(wl.density, np.float32)
        mid = np.ascontiguousarray(wl.material_id, np.uint8)
        mats = _Materials(wl.materials)
        self.params = default_params(**param_kw)
        h = C.c_void_p()
        nx, ny, nz = self.shape
        _check(L.sde_dose_create(C.byref(h), nx, ny, nz, (C.c_double * 3)(*wl.voxel_mm),
                                 (C.c_double * 3)(*wl.origin_mm), dens.ctypes.data, mid.ctypes.data,
                                 mats.arr, len(wl.materials), C.byref(self.params)))
        self.h = h
        if stream is not None:
            self.set_stream(stream)
        if tuning:
            self.set_tuning(**tuning)

    # -- configuration
    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        _check(lib().sde_dose_set_stream(self.h, C.c_void_p(ptr)))

    def set_tuning(self, blocks_per_sm=0, warps_per_block=0, batch=0, refill_min=0, table_smem=0,
                   aggregate=0, graph=0):
        t = Tuning(blocks_per_sm, warps_per_block, batch, refill_min, table_smem, aggregate, graph)
        _check(lib().sde_dose_set_tuning(self.h, C.byref(t)))

    def autotune(self, spots, seed=0, max_histories=200_000):
        """Pick the fastest launch shape for this plan (resets the tally)."""
        a, ptr = spots_to_ctypes(spots)
        t = Tuning()
        _check(lib().sde_dose_autotune(self.h, ptr, len(a), C.c_uint64(seed), C.c_uint64(max_histories),
                                       C.byref(t)))
        return {n: getattr(t, n) for n, _ in Tuning._fields_}

    def get_tuning(self):
        t = Tuning()
        _check(lib().sde_dose_get_tuning(self.h, C.byref(t)))
        return {n: getattr(t, n) for n, _ in Tuning._fields_}

    # -- work
    def run(self, spots, seed=0, first=None, count=None):
        """Transport the plan, or with first/count the histories with global ids in
        [first, first + count) (one shard of it)."""
        a, ptr = spots_to_ctypes(spots)
        if first is None and count is None:
            _check(lib().sde_dose_run(self.h, ptr, len(a), C.c_uint64(seed)))
        else:
            _check(lib().sde_dose_run_range(self.h, ptr, len(a), C.c_uint64(seed), C.c_uint64(first or 0),
                                            C.c_uint64(2**64 - 1 if count is None else count)))

    def run_device(self, d_spots_ptr: int, n_spots: int, seed=0, first=None, count=None):
        if first is None and count is None:
            _check(lib().sde_dose_run_device(self.h, C.c_void_p(d_spots_ptr), int(n_spots), C.c_uint64(seed)))
        else:
            _check(lib().sde_dose_run_device_range(self.h, C.c_void_p(d_spots_ptr), int(n_spots), C.c_uint64(seed),
                                                   C.c_uint64(first or 0),
                                                   C.c_uint64(2**64 - 1 if count is None else count)))

    def sync(self):
        _check(lib().sde_dose_sync(self.h))

    def reset(self):
        _check(lib().sde_dose_reset(self.h))

    def fetch(self, dose=True, edep=True):
        nx, ny, nz = self.shape
        d = np.empty((nz, ny, nx), np.float64) if dose else None
        e = np.empty((nz, ny, nx), np.uint64) if edep else None
        bal = Balance()
        _check(lib().sde_dose_fetch(self.h, d.ctypes.data if dose else None,
                                    e.ctypes.data if edep else None, C.byref(bal)))
        return d, e, bal.as_dict()

    def fetch_into(self, dose_ptr=None, edep_ptr=None, balance=True):
        """Host (pinned or pageable) output pointers; returns the balance dict."""
        bal = Balance()
        _check(lib().sde_dose_fetch(self.h, C.c_void_p(dose_ptr) if dose_ptr else None,
                                    C.c_void_p(edep_ptr) if edep_ptr else None,
                                    C.byref(bal) if balance else None))
        return bal.as_dict()

    def dose_into(self, tensor):
        """Write the dose (Gy) into a device tensor of n_vox float32 or float64 elements."""
        import torch
        if not tensor.is_cuda or tensor.numel() != self.wl.n_voxels or not tensor.is_contiguous():
            raise ValueError("dose_into needs a contiguous CUDA tensor with one element per voxel")
        if tensor.dtype == torch.float32:
            _check(lib().sde_dose_fetch_device_f32(self.h, C.c_void_p(tensor.data_ptr())))
        elif tensor.dtype == torch.float64:
            _check(lib().sde_dose_fetch_device(self.h, C.c_void_p(tensor.data_ptr()), None, None))
        else:
            raise ValueError("dose_into needs float32 or float64")
        return tensor

    def fetch_device(self, dose_ptr=None, edep_ptr=None, balance=False):
        """Raw device pointers: dose_ptr must hold n_vox float64, edep_ptr n_vox uint64."""
        bal = Balance()
        _check(lib().sde_dose_fetch_device(self.h, C.c_void_p(dose_ptr) if dose_ptr else None,
                                           C.c_void_p(edep_ptr) if edep_ptr else None,
                                           C.byref(bal) if balance else None))
        return bal.as_dict() if balance else None

    # -- introspection
    def info(self):
        nv, tp, n_m = C.c_uint64(), C.c_int(), C.c_int()
        emin, emax = C.c_double(), C.c_double()
        _check(lib().sde_dose_info(self.h, C.byref(nv), C.byref(tp), C.byref(emin), C.byref(emax),
                                   C.byref(n_m)))
        return {"n_vox": nv.value, "table_points": tp.value, "e_min": emin.value, "e_max": emax.value,
                "n_mats": n_m.value}

    def tables(self, m):
        inf = self.info()
        N = inf["table_points"]
        n_el = len(self.wl.materials[m]["elements"])
        raw = np.empty((N, 5), np.float32)
        rates = np.empty((N, 2, n_el), np.float32)
        csda = np.empty(N, np.float64)
        _check(lib().sde_dose_tables(self.h, int(m), raw.ctypes.data, rates.ctypes.data, csda.ctypes.data))
        E = inf["e_min"] * (inf["e_max"] / inf["e_min"]) ** (np.arange(N) / (N - 1))
        return {"E": E, "s1": raw[:, 0], "s2sq": raw[:, 1], "chi_c2": raw[:, 2], "bfac": raw[:, 3],
                "sig_jump": raw[:, 4], "rates": rates, "csda": csda}

    def probe_steps(self, m, rho, E, n, seed=0, h0=0):
        out = {k: np.empty(n, np.float32) for k in ("E", "cos", "ux", "uy")}
        out["jump"] = np.empty(n, np.int32)
        _check(lib().sde_dose_probe_steps(self.h, int(m), float(rho), float(E), C.c_uint64(seed),
                                          C.c_uint64(h0), int(n), out["E"].ctypes.data,
                                          out["cos"].ctypes.data, out["jump"].ctypes.data,
                                          out["ux"].ctypes.data, out["uy"].ctypes.data))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().sde_dose_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_bf16(A, B, D=None, stream=None):
    """D = A @ B.T on the tensor core (torch CUDA tensors: A [M,K] and B [N,K] bfloat16,
    D [M,N] float32)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if D is None:
        D = torch.empty(M, N, dtype=torch.float32, device=A.device)
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(lib().sde_gemm_bf16(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, st))
    return D


def _sp(stream):
    return None if stream is None else C.c_void_p(stream.cuda_stream)


def pcg_zeros(n, C, D, H, W, device="cuda"):
    """A zeroed BF16 tensor in the convolutions' padded channel-group-major layout:
    [n, C/8, D+2, H+2, W+2, 8] (see include/sde_dose.h)."""
    import torch
    return torch.zeros(n, C // 8, D + 2, H + 2, W + 2, 8, dtype=torch.bfloat16, device=device)


def to_pcg(x):
    """Channels-last [n, D, H, W, C] -> padded channel-group-major [n, C/8, D+2, H+2, W+2, 8]."""
    n, D, H, W, Cc = x.shape
    y = pcg_zeros(n, Cc, D, H, W, device=x.device)
    y[:, :, 1:-1, 1:-1, 1:-1, :] = x.to(y.dtype).reshape(n, D, H, W, Cc // 8, 8).permute(0, 4, 1, 2, 3, 5)
    return y


def from_pcg(y):
    """Padded channel-group-major [n, G, D+2, H+2, W+2, 8] -> channels-last [n, D, H, W, 8 G]."""
    n, G, Dp, Hp, Wp, _ = y.shape
    return y[:, :, 1:-1, 1:-1, 1:-1, :].permute(0, 2, 3, 4, 1, 5).reshape(n, Dp - 2, Hp - 2, Wp - 2, 8 * G)


def _pcg_shape(x):
    n, G, Dp, Hp, Wp, e = x.shape
    if e != 8:
        raise ValueError("expected a padded channel-group-major tensor [n, C/8, D+2, H+2, W+2, 8]")
    return n, Dp - 2, Hp - 2, Wp - 2, 8 * G


def conv3d(x, w, bias=None, relu=False, y=None, y_coffset=0, fp32=False, stream=None):
    """3x3x3 convolution: x padded channel-group-major with Cin channels, w [Cout, 27, Cin]
    bf16 -> y padded channel-group-major bf16, or with fp32 channels-last [n, D, H, W, C]."""
    import torch
    n, D, H, W, Cin = _pcg_shape(x)
    Cout = w.shape[0]
    if y is None:
        y = (torch.empty(n, D, H, W, Cout, dtype=torch.float32, device=x.device) if fp32
             else pcg_zeros(n, Cout, D, H, W, device=x.device))
    cstride = y.shape[-1] if fp32 else 8 * y.shape[1]
    _check(lib().sde_conv3d_forward(x.data_ptr(), n, D, H, W, Cin, w.data_ptr(),
                                    None if bias is None else bias.data_ptr(), Cout, y.data_ptr(),
                                    cstride, y_coffset, int(fp32), int(relu), _sp(stream)))
    return y


CONV_PLAN_FIELDS = ("Ty", "tiles", "rowtile", "fold", "nyb", "P", "Yb", "Cp", "nsplit", "plane", "w_off", "wres",
                    "stage", "nacc", "xch", "tcols", "items")
WGRAD_PLAN_FIELDS = ("Ty", "nyb", "P", "Yb", "Nc", "ntap", "ngroups", "kst", "plane_dy", "plane_x", "x_off", "stage",
                     "items", "G")


def conv3d_plan(batch, D, H, W, Cin, Cout):
    """Work decomposition sde_conv3d_forward launches for this shape (host only, no GPU):
    a dict of the plan's fields plus ``smem`` (dynamic shared memory in bytes)."""
    f = (C.c_int32 * len(CONV_PLAN_FIELDS))()
    sm = C.c_uint64()
    _check(lib().sde_conv3d_plan(batch, D, H, W, Cin, Cout, f, len(f), C.byref(sm)))
    return dict(zip(CONV_PLAN_FIELDS, list(f)), smem=sm.value)


def conv3d_wgrad_plan(batch, D, H, W, Cin, Cout, sms=152):
    """Work decomposition sde_conv3d_wgrad launches on a GPU with ``sms`` multiprocessors
    (host only, no GPU): a dict of the plan's fields plus ``smem``."""
    f = (C.c_int32 * len(WGRAD_PLAN_FIELDS))()
    sm = C.c_uint64()
    _check(lib().sde_conv3d_wgrad_plan(batch, D, H, W, Cin, Cout, sms, f, len(f), C.byref(sm)))
    return dict(zip(WGRAD_PLAN_FIELDS, list(f)), smem=sm.value)


def conv3d_wgrad(x, dy, dw, stream=None):
    """dw [Cout, 27, Cin] fp32 += weight gradient; x, dy padded channel-group-major."""
    n, D, H, W, Cin = _pcg_shape(x)
    _check(lib().sde_conv3d_wgrad(x.data_ptr(), dy.data_ptr(), dw.data_ptr(), n, D, H, W, Cin, 8 * dy.shape[1],
                                  _sp(stream)))
    return dw


def conv3d_flip_weights(w, wd=None, stream=None):
    import torch
    Cout, _, Cin = w.shape
    if wd is None:
        wd = torch.empty(Cin, 27, Cout, dtype=w.dtype, device=w.device)
    _check(lib().sde_conv3d_flip_weights(w.data_ptr(), wd.data_ptr(), Cin, Cout, _sp(stream)))
    return wd


def denoise_status(stream=None):
    _check(lib().sde_denoise_status(_sp(stream)))


class Denoiser:
    """Handle of the learned dose denoiser (see include/sde_dose.h)."""

    LAYERS = [(16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64), (64, 64), (96, 32),
              (32, 32), (32, 16)]

    def __init__(self, D, H, W, batch_max=1, seed=0, stream=None):
        h = C.c_void_p()
        _check(lib().sde_denoiser_create(C.byref(h), D, H, W, batch_max, C.c_uint64(seed)))
        self.h = h
        self.shape = (D, H, W)
        if stream is not None:
            _check(lib().sde_denoiser_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def num_params(self):
        n = C.c_uint64()
        _check(lib().sde_denoiser_num_params(self.h, C.byref(n)))
        return n.value

    def infer(self, dose_low, density, out=None):
        import torch
        b = dose_low.shape[0] if dose_low.dim() == 4 else 1
        if out is None:
            out = torch.empty_like(dose_low)
        _check(lib().sde_denoiser_infer(self.h, dose_low.data_ptr(), density.data_ptr(), b, out.data_ptr()))
        return out

    def train_step(self, dose_low, density, dose_high, lr=1e-3, want_loss=True, target_scale=1.0):
        b = dose_low.shape[0] if dose_low.dim() == 4 else 1
        loss = C.c_float()
        _check(lib().sde_denoiser_train_step(self.h, dose_low.data_ptr(), density.data_ptr(), dose_high.data_ptr(),
                                             C.c_float(target_scale), b, C.c_float(lr),
                                             C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def gradients(self, dose_low, density, dose_high, target_scale=1.0):
        b = dose_low.shape[0] if dose_low.dim() == 4 else 1
        n = self.num_params()
        g = np.empty(n, np.float32)
        loss = C.c_float()
        _check(lib().sde_denoiser_gradients(self.h, dose_low.data_ptr(), density.data_ptr(), dose_high.data_ptr(),
                                            C.c_float(target_scale), b, g.ctypes.data, n, C.byref(loss)))
        return g, loss.value

    def get_params(self):
        n = self.num_params()
        p = np.empty(n, np.float32)
        _check(lib().sde_denoiser_get_params(self.h, p.ctypes.data, n))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().sde_denoiser_set_params(self.h, p.ctypes.data, len(p)))

    def split(self, vec):
        """Per-layer (weights [Cout,27,Cin], bias [Cout]) views of a parameter vector."""
        out, o = [], 0
        for ci, co in self.LAYERS:
            n = co * 27 * ci
            out.append((vec[o:o + n].reshape(co, 27, ci), vec[o + n:o + n + co]))
            o += n + co
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().sde_denoiser_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scale_(x, factor, stream=None):
    """x *= factor in place (device FP32 tensor), in the library's kernel."""
    _check(lib().sde_scale_f32(x.data_ptr(), x.numel(), C.c_float(factor), _sp(stream)))
    return x


def gamma3d(ref, ev, voxel_mm, dd=0.02, dta_mm=0.5, threshold=0.01, steps=10, stream=None):
    """Gamma pass rate on the GPU (device FP32 grids [nz, ny, nx])."""
    nz, ny, nx = ref.shape[-3:]
    ne, npass = C.c_uint64(), C.c_uint64()
    _check(lib().sde_gamma3d(ref.data_ptr(), ev.data_ptr(), nx, ny, nz, (C.c_double * 3)(*voxel_mm), dd, dta_mm,
                             threshold, steps, C.byref(ne), C.byref(npass), _sp(stream)))
    return npass.value / max(ne.value, 1)


def run_workload(wl, seed=None, spots=None, **param_kw):
    """Create, run and fetch in one call; returns (dose_Gy, edep_fixed, balance)."""
    with SdeDose(wl, **param_kw) as d:
        d.run(wl.spots if spots is None else spots, wl.seed if seed is None else seed)
        return d.fetch()
