"""ctypes binding of liblbm_rd3q81 (include/lbm.h): the same entry points, same names,
argument marshalling only.  Every step of the method runs in the library's CUDA kernels.

Arrays: host arguments are C-contiguous numpy float64 arrays; device arguments are
contiguous CUDA float64 torch tensors (passed by data_ptr()).  A status other than LBM_OK
raises LbmError (LbmUnstable for LBM_EUNSTABLE) carrying the library's message.
If the shared library is missing the import fails loudly: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbm_rd3q81.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUSY, LBM_ENOTFOUND = range(8)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSTABLE",
                5: "LBM_ETIMEOUT", 6: "LBM_EBUSY", 7: "LBM_ENOTFOUND"}
LBM_RD3Q81 = 1
LBM_BC_PERIODIC, LBM_BC_ZERO_GRADIENT, LBM_BC_EQ_INFLOW, LBM_BC_BOUNCE_BACK = 0, 1, 2, 3
LBM_F64, LBM_F32, LBM_F16_OFFSET, LBM_BF16_OFFSET = 0, 1, 2, 3
LBM_EQ_SERIES, LBM_EQ_ENTROPIC, LBM_EQ_SERIES_EXACT_W = 0, 1, 2
EQUILIBRIUM = {"series": LBM_EQ_SERIES, "entropic": LBM_EQ_ENTROPIC, "series_exact_w": LBM_EQ_SERIES_EXACT_W}
LBM_COLLISION_BGK, LBM_COLLISION_ENTROPIC = 0, 1
COLLISION = {"bgk": LBM_COLLISION_BGK, "entropic": LBM_COLLISION_ENTROPIC}
LBM_STREAM_PINGPONG, LBM_STREAM_AA = 0, 1
STREAMING = {"pingpong": LBM_STREAM_PINGPONG, "aa": LBM_STREAM_AA}
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16_OFFSET, "bf16": LBM_BF16_OFFSET}
Q = 81


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class LbmUnstable(LbmError):
    pass


class lbm_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rho", ctypes.c_double), ("ux", ctypes.c_double),
                ("uy", ctypes.c_double), ("uz", ctypes.c_double), ("theta", ctypes.c_double)]


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("velset", ctypes.c_int),
                ("tau", ctypes.c_double), ("face", lbm_bc * 6), ("storage", ctypes.c_int),
                ("fp64_moments", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("equilibrium", ctypes.c_int),
                ("collision", ctypes.c_int), ("streaming", ctypes.c_int)]


class lbm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("unstable", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("site_updates", ctypes.c_longlong), ("ticks", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("graph_launches", ctypes.c_longlong),
                ("resident_cases", ctypes.c_int), ("resident_bytes", ctypes.c_size_t),
                ("peak_resident_bytes", ctypes.c_size_t), ("busy_seconds", ctypes.c_double),
                ("resident_byte_seconds", ctypes.c_double), ("backlog_seconds", ctypes.c_double),
                ("backlog_byte_seconds", ctypes.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built; run __graft_entry__.build() "
                          "(python -m paper_2409_05114_gb300.build_lib)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, LL, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    sigs = {
        "lbm_footprint": ([ctypes.POINTER(lbm_config), ctypes.POINTER(ctypes.c_size_t)], I),
        "lbm_create": ([ctypes.POINTER(lbm_config), ctypes.POINTER(P)], I),
        "lbm_init": ([P, P, P, P, I], I),
        "lbm_step": ([P, LL], I),
        "lbm_moments": ([P, P, P, P, I], I),
        "lbm_advance_fields": ([P, P, P, P, LL, P, P, P, I], I),
        "lbm_totals": ([P, P], I),
        "lbm_diagnostics": ([P, P], I),
        "lbm_selftest_log1p": ([LL, ctypes.POINTER(D)], I),
        "lbm_get_populations": ([P, P, I], I),
        "lbm_set_populations": ([P, P, I], I),
        "lbm_probe": ([P, P, LL, P], I),
        "lbm_sync": ([P], I),
        "lbm_launch_count": ([P, ctypes.POINTER(LL)], I),
        "lbm_destroy": ([P], I),
        "lbm_last_error": ([P], ctypes.c_char_p),
        "lbm_velocities": ([P, P], I),
        "lbm_server_create": ([ctypes.c_size_t, I, ctypes.POINTER(P)], I),
        "lbm_submit": ([P, ctypes.POINTER(lbm_config), P, P, P, LL, ctypes.POINTER(LL)], I),
        "lbm_poll": ([P, LL, P, P, P, ctypes.POINTER(D)], I),
        "lbm_wait": ([P, LL, D], I),
        "lbm_server_get_stats": ([P, ctypes.POINTER(lbm_server_stats)], I),
        "lbm_server_last_error": ([P], ctypes.c_char_p),
        "lbm_server_destroy": ([P], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def library_path() -> str:
    return _LIB_PATH


def _check(status: int, ctx=None):
    if status != LBM_OK:
        msg = _lib.lbm_last_error(ctx).decode()
        raise (LbmUnstable if status == LBM_EUNSTABLE else LbmError)(status, msg)


def _ptr(a, writable: bool = False):
    """(pointer, on_device) of a float64 array: numpy (host) or CUDA torch tensor (device)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or (writable and not a.flags.writeable):
            raise ValueError("host arrays must be C-contiguous, writable float64 numpy arrays")
        return ctypes.c_void_p(a.ctypes.data), 0
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float64 CUDA tensors")
        return ctypes.c_void_p(a.data_ptr()), 1
    raise TypeError(f"expected a numpy float64 array or a CUDA float64 tensor, got {type(a)}")


def make_config(nx: int, ny: int, nz: int, tau: float, storage="f32", faces=None, fp64_moments=False,
                stream=None, equilibrium="series", collision="bgk", streaming="pingpong") -> lbm_config:
    """Builds an lbm_config.  ``faces``: up to 6 face specs (-x, +x, -y, +y, -z, +z), each
    "periodic", "zero_gradient", "bounce_back" or ("eq_inflow", rho, ux, uy, uz, theta); default
    periodic.
    ``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None.
    ``equilibrium``: "series" (App. B), "series_exact_w" (App. B with the exact weights W(theta))
    or "entropic" (Sec. III, exact).
    ``collision``: "bgk" (alpha = 2) or "entropic" (alpha from Eq. (delH); needs the entropic
    equilibrium).  ``streaming``: "pingpong" (two buffers) or "aa" (one buffer, in place)."""
    cfg = lbm_config()
    cfg.equilibrium = EQUILIBRIUM[equilibrium] if isinstance(equilibrium, str) else int(equilibrium)
    cfg.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    cfg.streaming = STREAMING[streaming] if isinstance(streaming, str) else int(streaming)
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    cfg.velset = LBM_RD3Q81
    cfg.tau = float(tau)
    cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    cfg.fp64_moments = 1 if fp64_moments else 0
    faces = list(faces or [])
    for f in range(6):
        spec = faces[f] if f < len(faces) else "periodic"
        b = cfg.face[f]
        if isinstance(spec, str):
            spec = (spec,)
        kind = spec[0]
        b.kind = {"periodic": LBM_BC_PERIODIC, "zero_gradient": LBM_BC_ZERO_GRADIENT,
                  "eq_inflow": LBM_BC_EQ_INFLOW, "bounce_back": LBM_BC_BOUNCE_BACK}.get(kind, -1) \
            if isinstance(kind, str) else int(kind)
        if kind == "eq_inflow":
            b.rho, b.ux, b.uy, b.uz, b.theta = (float(v) for v in spec[1:6])
    if stream is None:
        cfg.cuda_stream = None
    elif hasattr(stream, "cuda_stream"):
        cfg.cuda_stream = ctypes.c_void_p(stream.cuda_stream)
    else:
        cfg.cuda_stream = ctypes.c_void_p(int(stream))
    return cfg


def lbm_footprint(cfg: lbm_config) -> int:
    out = ctypes.c_size_t()
    _check(_lib.lbm_footprint(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def lbm_create(cfg: lbm_config):
    ctx = ctypes.c_void_p()
    _check(_lib.lbm_create(ctypes.byref(cfg), ctypes.byref(ctx)))
    return ctx


def lbm_init(ctx, rho, u, theta):
    (pr, d0), (pu, d1), (pt, d2) = _ptr(rho), _ptr(u), _ptr(theta)
    if not d0 == d1 == d2:
        raise ValueError("rho, u, theta must all be host arrays or all device tensors")
    _check(_lib.lbm_init(ctx, pr, pu, pt, d0), ctx)


def lbm_step(ctx, n: int):
    _check(_lib.lbm_step(ctx, int(n)), ctx)


def lbm_moments(ctx, rho, u, theta):
    (pr, d0), (pu, d1), (pt, d2) = _ptr(rho, True), _ptr(u, True), _ptr(theta, True)
    if not d0 == d1 == d2:
        raise ValueError("rho, u, theta must all be host arrays or all device tensors")
    _check(_lib.lbm_moments(ctx, pr, pu, pt, d0), ctx)


def lbm_advance_fields(ctx, rho, u, theta, n: int, rho_out, u_out, theta_out):
    ptrs = [_ptr(rho), _ptr(u), _ptr(theta), _ptr(rho_out, True), _ptr(u_out, True), _ptr(theta_out, True)]
    if len({d for _, d in ptrs}) != 1:
        raise ValueError("all six fields must be host arrays or all device tensors")
    (pr, d0), (pu, _), (pt, _), (qr, _), (qu, _), (qt, _) = ptrs
    _check(_lib.lbm_advance_fields(ctx, pr, pu, pt, int(n), qr, qu, qt, d0), ctx)


def lbm_totals(ctx) -> np.ndarray:
    out = np.zeros(5)
    _check(_lib.lbm_totals(ctx, ctypes.c_void_p(out.ctypes.data)), ctx)
    return out


def lbm_diagnostics(ctx):
    """(KE, enstrophy): mean rho u.u/2 and mean rho |curl u|^2/2 of the stored state (Sec. IV C)."""
    out = np.zeros(2)
    _check(_lib.lbm_diagnostics(ctx, ctypes.c_void_p(out.ctypes.data)), ctx)
    return float(out[0]), float(out[1])


def lbm_selftest_log1p(n: int = 1 << 24) -> float:
    """Largest relative difference of the entropic-alpha FP32 log(1 + y) from CUDA's log1pf."""
    out = ctypes.c_double(0.0)
    _check(_lib.lbm_selftest_log1p(n, ctypes.byref(out)), None)
    return out.value


def lbm_get_populations(ctx, f):
    p, dev = _ptr(f, True)
    _check(_lib.lbm_get_populations(ctx, p, dev), ctx)


def lbm_set_populations(ctx, f):
    p, dev = _ptr(f)
    _check(_lib.lbm_set_populations(ctx, p, dev), ctx)


def lbm_probe(ctx, sites) -> np.ndarray:
    """Populations [len(sites), 81] (FP64, library order) of the given site indices."""
    idx = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((idx.size, Q))
    _check(_lib.lbm_probe(ctx, ctypes.c_void_p(idx.ctypes.data), idx.size, ctypes.c_void_p(out.ctypes.data)), ctx)
    return out


def lbm_sync(ctx):
    _check(_lib.lbm_sync(ctx), ctx)


def lbm_launch_count(ctx) -> int:
    out = ctypes.c_longlong()
    _check(_lib.lbm_launch_count(ctx, ctypes.byref(out)), ctx)
    return out.value


def lbm_destroy(ctx):
    _check(_lib.lbm_destroy(ctx))


def lbm_last_error(ctx=None) -> str:
    return _lib.lbm_last_error(ctx).decode()


def lbm_velocities():
    """(h[81, 3] int32 with h = 2c, w[81] float64) in the library's direction order."""
    h = np.zeros(3 * Q, dtype=np.int32)
    w = np.zeros(Q)
    n = _lib.lbm_velocities(ctypes.c_void_p(h.ctypes.data), ctypes.c_void_p(w.ctypes.data))
    assert n == Q
    return h.reshape(Q, 3), w


# ---- serving ---------------------------------------------------------------------------

def _check_srv(status: int, srv=None):
    if status != LBM_OK:
        msg = _lib.lbm_server_last_error(srv).decode()
        raise (LbmUnstable if status == LBM_EUNSTABLE else LbmError)(status, msg)


def lbm_server_create(hbm_budget_bytes: int, max_cases: int):
    srv = ctypes.c_void_p()
    _check_srv(_lib.lbm_server_create(int(hbm_budget_bytes), int(max_cases), ctypes.byref(srv)))
    return srv


def lbm_submit(srv, cfg: lbm_config, rho, u, theta, nsteps: int) -> int:
    """Queues a case (host fields, copied before returning); returns its ticket."""
    (pr, d0), (pu, d1), (pt, d2) = _ptr(rho), _ptr(u), _ptr(theta)
    if d0 or d1 or d2:
        raise ValueError("lbm_submit takes host arrays")
    t = ctypes.c_longlong()
    _check_srv(_lib.lbm_submit(srv, ctypes.byref(cfg), pr, pu, pt, int(nsteps), ctypes.byref(t)), srv)
    return t.value


def lbm_poll(srv, ticket: int, rho=None, u=None, theta=None):
    """(status, latency_s).  status LBM_EBUSY while running; once done the fields are copied
    into the given host arrays (any may be None) and the ticket is forgotten."""
    lat = ctypes.c_double(0.0)
    ptrs = [None if a is None else _ptr(a, True)[0] for a in (rho, u, theta)]
    st = _lib.lbm_poll(srv, int(ticket), *ptrs, ctypes.byref(lat))
    return st, lat.value


def lbm_wait(srv, ticket: int, timeout_s: float) -> int:
    """LBM_OK when the case is done, LBM_ETIMEOUT after timeout_s seconds."""
    return _lib.lbm_wait(srv, int(ticket), float(timeout_s))


def lbm_server_get_stats(srv) -> dict:
    st = lbm_server_stats()
    _check_srv(_lib.lbm_server_get_stats(srv, ctypes.byref(st)), srv)
    return {name: getattr(st, name) for name, _ in st._fields_}


def lbm_server_destroy(srv):
    _check_srv(_lib.lbm_server_destroy(srv))
