"""GB300 (sm_103a) MRT-Smagorinsky lattice Boltzmann solver: Python binding.

Argument marshalling only.  Every function below calls the entry point of the
same name in the in-tree CUDA library ``liblbm_gb300.so`` (C ABI declared in
``include/lbm.h``); all computation runs in that library's kernels.  There is
no CPU fallback: ``load()`` raises if the library is missing or cannot be
loaded.

Host arrays are numpy arrays (C-contiguous, x fastest): populations
``(19, nz, ny, nx)``, vectors ``(3, nz, ny, nx)``, scalars ``(nz, ny, nx)``.
A device velocity field may be a CUDA torch tensor (float64, same layout).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_UNSUPPORTED = -6

LBM_FP32, LBM_FP16_SHIFTED, LBM_BF16_SHIFTED = 0, 1, 2
LBM_FORCE_NONE, LBM_FORCE_PAPER_SIN, LBM_FORCE_CONST, LBM_FORCE_KOLMOGOROV = 0, 1, 2, 3
LBM_INIT_REST, LBM_INIT_TGV3D, LBM_INIT_TGV2D, LBM_INIT_VELOCITY = 0, 1, 2, 3
LBM_STATS_SPECTRUM, LBM_STATS_STRUCTURE = 1, 2
LBM_MAX_R = 24

EXPORTED = [
    "lbm_create", "lbm_create_batch", "lbm_destroy", "lbm_count", "lbm_init_field",
    "lbm_init_velocity_f32", "lbm_step",
    "lbm_sync", "lbm_time", "lbm_stats", "lbm_series", "lbm_spectrum", "lbm_histogram",
    "lbm_get_populations", "lbm_set_populations", "lbm_set_time", "lbm_get_fields",
    "lbm_get_theta_slice", "lbm_device_ptr", "lbm_get_params", "lbm_kernel_config",
    "lbm_last_error", "lbm_version", "lbm_structure_functions_noalloc", "lbm_debug_withhold_load",
    "lbm_energy_balance", "lbm_batch_create", "lbm_batch_step", "lbm_batch_stats", "lbm_get_velocity",
    "lbm_init_random_spectrum",
]


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("re", ctypes.c_double), ("u0", ctypes.c_double), ("nu0", ctypes.c_double),
        ("cs", ctypes.c_double), ("cf", ctypes.c_double), ("f0", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("force_mode", ctypes.c_int32), ("stats_every", ctypes.c_int32),
        ("hist_bins", ctypes.c_int32), ("device", ctypes.c_int32),
        ("hist_max", ctypes.c_double), ("stream", ctypes.c_void_p),
        ("kernel", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
        ("stages", ctypes.c_int32), ("threads", ctypes.c_int32),
        ("row_align", ctypes.c_int32), ("strain_mode", ctypes.c_int32), ("layout", ctypes.c_int32),
        ("tma_slots", ctypes.c_int32),
    ]


class LbmStats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("cells", ctypes.c_int64),
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("E_k", ctypes.c_double), ("inj", ctypes.c_double), ("eps0", ctypes.c_double),
        ("eps_sgs", ctypes.c_double), ("uu", ctypes.c_double * 6),
        ("theta_mean", ctypes.c_double), ("theta_var", ctypes.c_double),
        ("theta_min", ctypes.c_double), ("theta_max", ctypes.c_double),
        ("theta_p05", ctypes.c_double), ("theta_p50", ctypes.c_double),
        ("theta_p95", ctypes.c_double), ("theta_p99", ctypes.c_double),
        ("Kt_mean", ctypes.c_double), ("Kt_var", ctypes.c_double),
        ("L", ctypes.c_double), ("eps_spec", ctypes.c_double), ("eta", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("u_rms", ctypes.c_double), ("Re_lambda", ctypes.c_double),
        ("nr", ctypes.c_int32), ("r", ctypes.c_int32 * LBM_MAX_R),
        ("Sp", (ctypes.c_double * 6) * LBM_MAX_R), ("F4", ctypes.c_double * LBM_MAX_R),
        ("E_frac", ctypes.c_double * 3), ("b", ctypes.c_double * 6),
        ("II_b", ctypes.c_double), ("III_b", ctypes.c_double),
        ("lumley_xi", ctypes.c_double), ("lumley_eta", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name in ("momentum", "uu", "E_frac", "b"):
                v = list(v)
            elif name in ("r", "Sp", "F4"):
                continue
            out[name.rstrip("_")] = v
        n = self.nr
        out["r"] = list(self.r)[:n]
        out["Sp"] = np.array([list(self.Sp[i]) for i in range(n)]).reshape(n, 6)
        out["F4"] = np.array(list(self.F4)[:n])
        return out


class LbmRecord(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("E_k", ctypes.c_double), ("inj", ctypes.c_double), ("eps0", ctypes.c_double),
        ("eps_sgs", ctypes.c_double), ("theta_mean", ctypes.c_double),
        ("theta_var", ctypes.c_double), ("theta_min", ctypes.c_double),
        ("theta_max", ctypes.c_double),
    ]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    """liblbm_gb300.so, or its bounds-checked build when the environment sets
    LBM_LIBRARY=checked."""
    return _build.LIB_CHECKED if os.environ.get("LBM_LIBRARY") == "checked" else _build.LIB


def load():
    """Load the library (library_path()); raises if it has not been built (no
    fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "lbm_create": ([ctypes.POINTER(LbmParams), ctypes.POINTER(H)], ctypes.c_int),
        "lbm_create_batch": ([ctypes.POINTER(LbmParams), i32, ctypes.POINTER(H)], ctypes.c_int),
        "lbm_destroy": ([H], ctypes.c_int),
        "lbm_count": ([H], ctypes.c_int),
        "lbm_init_field": ([H, i32, i32, ctypes.c_double, ctypes.c_void_p, i32], ctypes.c_int),
        "lbm_init_velocity_f32": ([H, i32, ctypes.c_void_p, i32], ctypes.c_int),
        "lbm_step": ([H, i64], ctypes.c_int),
        "lbm_sync": ([H], ctypes.c_int),
        "lbm_time": ([H], i64),
        "lbm_stats": ([H, i32, i32, ctypes.POINTER(LbmStats)], ctypes.c_int),
        "lbm_series": ([H, i32, ctypes.POINTER(LbmRecord), i32, ctypes.POINTER(i32)], ctypes.c_int),
        "lbm_spectrum": ([H, i32, _D, i32], ctypes.c_int),
        "lbm_histogram": ([H, i32, ctypes.POINTER(ctypes.c_uint64), i32], ctypes.c_int),
        "lbm_get_populations": ([H, i32, _D, i32], ctypes.c_int),
        "lbm_set_populations": ([H, i32, _D, i32], ctypes.c_int),
        "lbm_set_time": ([H, i64], ctypes.c_int),
        "lbm_get_fields": ([H, i32, _D, _D, _D, _D], ctypes.c_int),
        "lbm_get_theta_slice": ([H, i32, i32, i32, _D], ctypes.c_int),
        "lbm_device_ptr": ([H, i32, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t),
                            ctypes.POINTER(i32)], ctypes.c_int),
        "lbm_get_params": ([H, i32, _D, _D, _D, _D], ctypes.c_int),
        "lbm_kernel_config": ([H] + [ctypes.POINTER(i32)] * 7, ctypes.c_int),
        "lbm_last_error": ([H], ctypes.c_char_p),
        "lbm_version": ([], ctypes.c_char_p),
        "lbm_structure_functions_noalloc": ([ctypes.c_void_p, i32, i32, i32, ctypes.POINTER(i32), i32,
                                             ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "lbm_debug_withhold_load": ([H, ctypes.c_double], ctypes.c_int),
        "lbm_energy_balance": ([ctypes.POINTER(LbmRecord), i32, _D, ctypes.POINTER(i64)], ctypes.c_int),
        "lbm_batch_create": ([ctypes.POINTER(LbmParams), i32, ctypes.POINTER(H)], ctypes.c_int),
        "lbm_batch_step": ([H, i64], ctypes.c_int),
        "lbm_batch_stats": ([H, i32, ctypes.POINTER(LbmStats)], ctypes.c_int),
        "lbm_get_velocity": ([H, i32, _D], ctypes.c_int),
        "lbm_init_random_spectrum": ([H, i32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_void_p, i32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(h, rc: int):
    if rc != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LbmError(rc, msg.decode() if msg else "")


def _f64(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


# ---- entry points (same names as include/lbm.h) ---------------------------------

def make_params(nx, ny=None, nz=None, *, precision=LBM_FP32, re=0.0, u0=0.0, nu0=0.0, cs=0.0,
                cf=0.2, f0=0.0, body_force=(0.0, 0.0, 0.0), force_mode=LBM_FORCE_NONE,
                stats_every=0, hist_bins=0, hist_max=0.0, device=0, stream=None, kernel=0,
                tile_rows=0, stages=0, threads=0, row_align=0, strain_mode=0, layout=0,
                tma_slots=0) -> LbmParams:
    p = LbmParams()
    p.nx, p.ny, p.nz = nx, nx if ny is None else ny, nx if nz is None else nz
    p.precision = precision
    p.re, p.u0, p.nu0, p.cs, p.cf, p.f0 = re, u0, nu0, cs, cf, f0
    for i in range(3):
        p.body_force[i] = body_force[i]
    p.force_mode, p.stats_every = force_mode, stats_every
    p.hist_bins, p.hist_max, p.device = hist_bins, hist_max, device
    p.stream = stream
    p.kernel, p.tile_rows = kernel, tile_rows
    p.stages, p.threads = stages, threads
    p.row_align = row_align
    p.strain_mode = strain_mode
    p.layout = layout
    p.tma_slots = tma_slots
    return p


def lbm_create(params: LbmParams) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(None, load().lbm_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def lbm_create_batch(params: list) -> ctypes.c_void_p:
    arr = (LbmParams * len(params))(*params)
    h = ctypes.c_void_p()
    _check(None, load().lbm_create_batch(arr, len(params), ctypes.byref(h)))
    return h


def lbm_destroy(h) -> None:
    _check(None, load().lbm_destroy(h))


def lbm_count(h) -> int:
    return int(load().lbm_count(h))


def lbm_init_field(h, inst: int, mode: int, amplitude: float = 0.0, u=None) -> None:
    """u: None, a host numpy array (3, nz, ny, nx) (staged copies), a
    page-locked CPU torch tensor (read in place by the kernel: keep it alive
    until the next synchronising call), or a CUDA torch tensor.  float32 data
    go through lbm_init_velocity_f32 (same populations, half the bytes), any
    other dtype is taken as float64."""
    lib = load()
    if u is None:
        _check(h, lib.lbm_init_field(h, inst, mode, amplitude, None, 0))
        return

    def call(ptr, where, f32):
        if f32:
            if mode != LBM_INIT_VELOCITY:
                raise ValueError("an FP32 field is only accepted for LBM_INIT_VELOCITY")
            _check(h, lib.lbm_init_velocity_f32(h, inst, ptr, where))
        else:
            _check(h, lib.lbm_init_field(h, inst, mode, amplitude, ptr, where))

    if hasattr(u, "is_cuda"):
        import torch
        where = 1 if u.is_cuda else (2 if u.is_pinned() else None)
        if where is not None:
            if u.dtype not in (torch.float64, torch.float32) or not u.is_contiguous():
                raise ValueError("velocity tensor must be a contiguous float64 or float32 tensor")
            if u.is_cuda:
                # the handle's stream does not wait for torch's: the field must be
                # complete before the initialisation kernel reads it
                torch.cuda.current_stream(u.device).synchronize()
            call(ctypes.c_void_p(u.data_ptr()), where, u.dtype == torch.float32)
            return
        u = u.numpy()
    f32 = getattr(u, "dtype", None) == np.float32
    ua = np.ascontiguousarray(u, dtype=np.float32 if f32 else np.float64)
    call(ua.ctypes.data_as(ctypes.c_void_p), 0, f32)


def lbm_init_random_spectrum(h, inst: int = 0, seed: int = 1, urms: float = 0.05, k0: float = 4.0,
                             u_out=None) -> None:
    """Seeded random solenoidal field generated on the device (include/lbm.h).
    u_out: None, a float32 numpy array (3, nz, ny, nx), or a contiguous float32
    torch tensor of that shape (CUDA: device copy; CPU: host copy)."""
    where, ptr = 0, None
    if u_out is not None:
        if hasattr(u_out, "is_cuda"):
            import torch
            if u_out.dtype != torch.float32 or not u_out.is_contiguous():
                raise ValueError("u_out must be a contiguous float32 tensor")
            where, ptr = (1 if u_out.is_cuda else 0), ctypes.c_void_p(u_out.data_ptr())
        else:
            if u_out.dtype != np.float32 or not u_out.flags["C_CONTIGUOUS"]:
                raise ValueError("u_out must be a C-contiguous float32 array")
            ptr = u_out.ctypes.data_as(ctypes.c_void_p)
    _check(h, load().lbm_init_random_spectrum(h, inst, int(seed), float(urms), float(k0), ptr, where))


def lbm_step(h, n: int) -> None:
    _check(h, load().lbm_step(h, int(n)))


def lbm_sync(h) -> None:
    _check(h, load().lbm_sync(h))


def lbm_time(h) -> int:
    return int(load().lbm_time(h))


def lbm_stats(h, inst: int = 0, what: int = 0) -> dict:
    s = LbmStats()
    _check(h, load().lbm_stats(h, inst, what, ctypes.byref(s)))
    return s.as_dict()


def lbm_series(h, inst: int = 0, max_records: int = 1024) -> list:
    buf = (LbmRecord * max_records)()
    n = ctypes.c_int32()
    _check(h, load().lbm_series(h, inst, buf, max_records, ctypes.byref(n)))
    out = []
    for i in range(n.value):
        r = buf[i]
        out.append({"step": r.step, "mass": r.mass, "momentum": list(r.momentum), "E_k": r.E_k,
                    "inj": r.inj, "eps0": r.eps0, "eps_sgs": r.eps_sgs,
                    "theta_mean": r.theta_mean, "theta_var": r.theta_var,
                    "theta_min": r.theta_min, "theta_max": r.theta_max})
    return out


def lbm_spectrum(h, inst: int, kmax: int) -> np.ndarray:
    E = np.zeros(kmax + 1)
    _check(h, load().lbm_spectrum(h, inst, _ptr(E), kmax))
    return E


def lbm_histogram(h, inst: int, bins: int) -> np.ndarray:
    c = np.zeros(bins + 1, dtype=np.uint64)
    _check(h, load().lbm_histogram(h, inst, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), bins))
    return c


def lbm_get_populations(h, inst: int, shape, shifted: bool = True) -> np.ndarray:
    nz, ny, nx = shape
    out = np.zeros((19, nz, ny, nx))
    _check(h, load().lbm_get_populations(h, inst, _ptr(out), 1 if shifted else 0))
    return out


def lbm_set_populations(h, inst: int, f: np.ndarray, shifted: bool = True) -> None:
    a = np.ascontiguousarray(f, dtype=np.float64)
    _check(h, load().lbm_set_populations(h, inst, _ptr(a), 1 if shifted else 0))


def lbm_set_time(h, t: int) -> None:
    _check(h, load().lbm_set_time(h, int(t)))


def lbm_get_fields(h, inst: int, shape) -> dict:
    nz, ny, nx = shape
    drho = np.zeros((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    sn = np.zeros((nz, ny, nx))
    th = np.zeros((nz, ny, nx))
    _check(h, load().lbm_get_fields(h, inst, _ptr(drho), _ptr(u), _ptr(sn), _ptr(th)))
    return {"drho": drho, "u": u, "snorm": sn, "theta": th}


def lbm_get_velocity(h, inst: int, shape) -> np.ndarray:
    nz, ny, nx = shape
    u = np.zeros((3, nz, ny, nx))
    _check(h, load().lbm_get_velocity(h, inst, _ptr(u)))
    return u


def lbm_batch_create(params: list) -> ctypes.c_void_p:
    arr = (LbmParams * len(params))(*params)
    h = ctypes.c_void_p()
    _check(None, load().lbm_batch_create(arr, len(params), ctypes.byref(h)))
    return h


def lbm_batch_step(h, n: int) -> None:
    _check(h, load().lbm_batch_step(h, n))


def lbm_batch_stats(h, count: int, what: int = 0) -> list:
    out = (LbmStats * max(count, 1))()
    _check(h, load().lbm_batch_stats(h, what, out))
    return [out[i].as_dict() for i in range(count)]


def lbm_get_theta_slice(h, inst: int, axis: int, index: int, shape) -> np.ndarray:
    nz, ny, nx = shape
    dims = {0: (nz, ny), 1: (nz, nx), 2: (ny, nx)}.get(axis, (1,))
    out = np.zeros(dims)
    _check(h, load().lbm_get_theta_slice(h, inst, axis, index, _ptr(out)))
    return out


def lbm_device_ptr(h, inst: int = 0):
    p = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    nxp = ctypes.c_int32()
    _check(h, load().lbm_device_ptr(h, inst, ctypes.byref(p), ctypes.byref(nbytes), ctypes.byref(nxp)))
    return p.value, nbytes.value, nxp.value


def lbm_get_params(h, inst: int = 0) -> dict:
    v = [ctypes.c_double() for _ in range(4)]
    _check(h, load().lbm_get_params(h, inst, *[ctypes.byref(x) for x in v]))
    return dict(zip(("nu0", "s_nu0", "F0", "C"), [x.value for x in v]))


def lbm_kernel_config(h) -> dict:
    v = [ctypes.c_int32() for _ in range(7)]
    _check(h, load().lbm_kernel_config(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(("kind", "tile_rows", "stages", "threads", "blocks_per_sm", "layout", "slot_bytes"),
                    [x.value for x in v]))


def lbm_structure_functions_noalloc(u, r, sp, stream=None) -> None:
    """S_p(r) of a device velocity field without any device allocation.

    u: CUDA float32 tensor (3, nz, ny, nx); r: separations (<= 24 of them);
    sp: CUDA float64 tensor with len(r) * 6 elements, written asynchronously on
    `stream` (a torch stream, or None for the default stream)."""
    import torch
    if not (u.is_cuda and sp.is_cuda) or u.device != sp.device:
        raise ValueError("u and sp must be CUDA tensors on the same device")
    if u.dtype != torch.float32 or not u.is_contiguous() or u.dim() != 4 or u.shape[0] != 3:
        raise ValueError("u must be a contiguous float32 tensor of shape (3, nz, ny, nx)")
    if sp.dtype != torch.float64 or not sp.is_contiguous() or sp.numel() < 6 * len(r):
        raise ValueError("sp must be a contiguous float64 tensor of at least 6 * len(r) elements")
    _, nz, ny, nx = u.shape
    ra = (ctypes.c_int32 * max(1, len(r)))(*r)
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    with torch.cuda.device(u.device):  # the entry point works on the current device
        _check(None, load().lbm_structure_functions_noalloc(
            ctypes.c_void_p(u.data_ptr()), nx, ny, nz, ra, len(r), ctypes.c_void_p(sp.data_ptr()), st))


def lbm_energy_balance(records: list):
    """(times, relative residuals) of Eq. (energy_balance) along a record series
    (the dicts of lbm_series)."""
    n = len(records)
    buf = (LbmRecord * max(1, n))()
    for i, r in enumerate(records):
        buf[i].step = r["step"]
        buf[i].E_k, buf[i].inj, buf[i].eps0, buf[i].eps_sgs = r["E_k"], r["inj"], r["eps0"], r["eps_sgs"]
    res = np.zeros(max(1, n - 2))
    at = (ctypes.c_int64 * max(1, n - 2))()
    _check(None, load().lbm_energy_balance(buf, n, _ptr(res), at))
    return np.array(list(at)[:n - 2]), res[:n - 2]


def lbm_debug_withhold_load(h, wait_seconds: float) -> None:
    _check(h, load().lbm_debug_withhold_load(h, float(wait_seconds)))


def lbm_last_error(h=None) -> str:
    m = load().lbm_last_error(h)
    return m.decode() if m else ""


def lbm_version() -> str:
    return load().lbm_version().decode()


# ---- convenience wrapper ---------------------------------------------------------

class Lattice:
    """One handle (one or more instances) with numpy-friendly methods."""

    def __init__(self, params):
        plist = params if isinstance(params, (list, tuple)) else [params]
        self.params = list(plist)
        self.h = lbm_create_batch(self.params) if len(plist) > 1 else lbm_create(plist[0])
        self.shapes = [(p.nz, p.ny, p.nx) for p in self.params]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def time(self) -> int:
        return lbm_time(self.h)

    def init(self, mode=LBM_INIT_VELOCITY, amplitude=0.0, u=None, inst=0):
        lbm_init_field(self.h, inst, mode, amplitude, u)

    def init_random(self, seed=1, urms=0.05, k0=4.0, inst=0, u_out=None):
        lbm_init_random_spectrum(self.h, inst, seed, urms, k0, u_out)

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def populations(self, inst=0, shifted=True):
        return lbm_get_populations(self.h, inst, self.shapes[inst], shifted)

    def set_populations(self, f, inst=0, shifted=True):
        lbm_set_populations(self.h, inst, f, shifted)

    def fields(self, inst=0):
        return lbm_get_fields(self.h, inst, self.shapes[inst])

    def stats(self, inst=0, what=0):
        return lbm_stats(self.h, inst, what)

    def spectrum(self, kmax, inst=0):
        return lbm_spectrum(self.h, inst, kmax)

    def theta_slice(self, axis, index, inst=0):
        return lbm_get_theta_slice(self.h, inst, axis, index, self.shapes[inst])

    def series(self, inst=0):
        return lbm_series(self.h, inst)

    def config(self):
        return lbm_kernel_config(self.h)

    def derived(self, inst=0):
        return lbm_get_params(self.h, inst)
