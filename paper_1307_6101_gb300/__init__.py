"""Python binding of the GB300 DD-alpha-AMG library (C ABI in include/ddamg.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libddamg.so``.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA memory); complex128 arrays are passed as their interleaved
float64 storage.  There is no CPU fallback: importing fails if the library
has not been built (``python -m paper_1307_6101_gb300.build`` or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddamg.so")

DDAMG_OK = 0
DDAMG_ERR_ARG = -1
DDAMG_ERR_OOM = -2
DDAMG_ERR_NOCONV = -3
DDAMG_ERR_CUDA = -4
DDAMG_ERR_SINGULAR = -5
DDAMG_ERR_ADMISSION = -6
MAX_LEVELS = 4

EXPORTED = (
    "ddamg_default_params", "ddamg_setup", "ddamg_solve", "ddamg_free", "ddamg_last_error",
    "ddamg_set_stream", "ddamg_level_info", "ddamg_apply", "ddamg_smooth", "ddamg_restrict",
    "ddamg_prolong", "ddamg_kcycle", "ddamg_coarse_solve", "ddamg_set_testvectors",
    "ddamg_get_testvectors", "ddamg_rebuild", "ddamg_get_interpolation", "ddamg_get_coarse_operator",
    "ddamg_profile", "ddamg_profile_read", "ddamg_launch_count", "ddamg_set_option",
    "ddamg_krylov_steps", "ddamg_residual_norm_noalloc", "ddamg_get_option",
    "ddamg_device_bytes", "ddamg_estimate_bytes", "ddamg_server_create", "ddamg_server_add",
    "ddamg_server_submit", "ddamg_server_poll", "ddamg_server_wait", "ddamg_server_free",
    "ddamg_setup_times", "ddamg_autotune_times", "ddamg_cgnr", "ddamg_sigma_extremes",
    "ddamg_update_gauge",
)
DDAMG_OPT_GRAPHS = 0
DDAMG_OPT_COARSEST_CLUSTER = 1
DDAMG_OPT_SAP_CLUSTER = 2
DDAMG_OPT_HALF_STORAGE = 3
DDAMG_OPT_COARSE_TC = 4
DDAMG_OPT_SAP_SCHUR = 5
DDAMG_OPT_SAP_PERSIST = 6
DDAMG_OPT_OUTER_DF = 7
SETUP_KINDS = ("smooth", "kcycle", "rebuild")   # DDAMG_SETUP_* order
PROF_KINDS = {"fine_sap": 0, "fine_dslash": 1, "coarse_apply": 2, "coarse_sap": 3, "transfer": 4, "precond": 5,
              "outer_ortho": 6}


class DdamgParams(C.Structure):
    _fields_ = [
        ("levels", C.c_int),
        ("agg", (C.c_int * 4) * MAX_LEVELS),
        ("n_tv", C.c_int * MAX_LEVELS),
        ("sap_block", (C.c_int * 4) * MAX_LEVELS),
        ("mr_steps", C.c_int),
        ("nu", C.c_int),
        ("mu", C.c_int),
        ("n_inv", C.c_int),
        ("eta_passes", C.c_int),
        ("outer_restart", C.c_int),
        ("outer_max_cycles", C.c_int),
        ("kcycle_len", C.c_int),
        ("kcycle_cycles", C.c_int),
        ("kcycle_tol", C.c_double),
        ("coarse_tol", C.c_double),
        ("coarse_restart", C.c_int),
        ("coarse_cycles", C.c_int),
        ("precision", C.c_int),
        ("max_rhs", C.c_int),
        ("seed", C.c_uint64),
        ("sap_schur", C.c_int),
        ("setup_batch", C.c_int),
    ]


class DdamgStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cycles", C.c_int), ("converged", C.c_int),
                ("true_residual", C.c_double)]


class DdamgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ddamg error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, ip, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
    lib.ddamg_default_params.argtypes = [C.POINTER(DdamgParams)]
    lib.ddamg_default_params.restype = None
    lib.ddamg_setup.argtypes = [vp, C.POINTER(C.c_int), ip, C.c_double, C.c_double, C.POINTER(DdamgParams),
                                C.POINTER(C.c_void_p), C.POINTER(vp)]
    lib.ddamg_solve.argtypes = [vp, vp, vp, ip, C.c_double, C.POINTER(DdamgStats)]
    lib.ddamg_free.argtypes = [vp]
    lib.ddamg_update_gauge.argtypes = [vp, vp, ip]
    lib.ddamg_cgnr.argtypes = [vp, vp, vp, ip, C.c_double, ip, C.POINTER(DdamgStats)]
    lib.ddamg_sigma_extremes.argtypes = [vp, ip, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int)]
    lib.ddamg_free.restype = None
    lib.ddamg_last_error.restype = C.c_char_p
    lib.ddamg_set_stream.argtypes = [vp, vp]
    lib.ddamg_level_info.argtypes = [vp, ip, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    for name in ("ddamg_apply", "ddamg_restrict", "ddamg_prolong", "ddamg_kcycle"):
        getattr(lib, name).argtypes = [vp, ip, ip, vp, vp, ip]
    lib.ddamg_smooth.argtypes = [vp, ip, ip, vp, vp, ip, ip]
    lib.ddamg_coarse_solve.argtypes = [vp, ip, vp, vp, ip]
    lib.ddamg_set_testvectors.argtypes = [vp, ip, vp, ip]
    lib.ddamg_get_testvectors.argtypes = [vp, ip, vp, ip]
    lib.ddamg_rebuild.argtypes = [vp, ip]
    lib.ddamg_get_interpolation.argtypes = [vp, ip, vp]
    lib.ddamg_get_coarse_operator.argtypes = [vp, ip, vp]
    lib.ddamg_profile.argtypes = [vp, ip]
    lib.ddamg_profile_read.argtypes = [vp, ip, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double)]
    lib.ddamg_set_option.argtypes = [vp, ip, ip]
    lib.ddamg_get_option.argtypes = [vp, ip, C.POINTER(C.c_int)]
    lib.ddamg_krylov_steps.argtypes = [vp, ip, ip, C.POINTER(C.c_longlong)]
    lib.ddamg_residual_norm_noalloc.argtypes = [vp, vp, vp, ip, vp]
    lib.ddamg_launch_count.restype = C.c_longlong
    lib.ddamg_launch_count.argtypes = []
    sp = C.POINTER(C.c_size_t)
    lib.ddamg_device_bytes.argtypes = [vp, sp]
    lib.ddamg_setup_times.argtypes = [vp, C.POINTER(C.c_double), ip]
    lib.ddamg_autotune_times.argtypes = [vp, ip, ip, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.ddamg_estimate_bytes.argtypes = [C.POINTER(C.c_int), C.POINTER(DdamgParams), sp]
    lib.ddamg_server_create.argtypes = [C.c_size_t, C.POINTER(vp)]
    lib.ddamg_server_add.argtypes = [vp, vp, C.POINTER(C.c_int)]
    lib.ddamg_server_submit.argtypes = [vp, ip, vp, ip, C.c_double, C.POINTER(C.c_longlong)]
    lib.ddamg_server_poll.argtypes = [vp, C.c_longlong, C.POINTER(C.c_int)]
    lib.ddamg_server_wait.argtypes = [vp, C.c_longlong, vp, C.POINTER(DdamgStats), C.POINTER(C.c_double)]
    lib.ddamg_server_free.argtypes = [vp]
    del dp
    return lib


_LIB = None


def lib():
    """The loaded libddamg.so (loaded on first use; raises if it was not built)."""
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


def _check(rc):
    if rc != DDAMG_OK:
        raise DdamgError(rc, lib().ddamg_last_error().decode())
    return rc


def _ptr(a):
    """Device or host address of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        if a.dtype not in (np.complex128, np.float64):
            raise ValueError("arrays must be complex128 or float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if a.dtype not in (torch.complex128, torch.float64):
            raise ValueError("tensors must be complex128 or float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def ddamg_default_params(**overrides) -> DdamgParams:
    p = DdamgParams()
    lib().ddamg_default_params(C.byref(p))
    for k, v in overrides.items():
        if k in ("agg", "sap_block"):
            for l, blk in enumerate(v):
                if blk is None:
                    continue
                for d in range(4):
                    getattr(p, k)[l][d] = int(blk[d])
        elif k == "n_tv":
            for l, n in enumerate(v):
                p.n_tv[l] = int(n)
        else:
            setattr(p, k, v)
    return p


class Handle:
    """An owned hierarchy (ddamg_handle*).  Methods mirror the C ABI."""

    def __init__(self, raw, params, dims):
        self._h = raw
        self.params = params
        self.dims = tuple(dims)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None):
            lib().ddamg_free(self._h)
            self._h = None

    @property
    def raw(self):
        return self._h

    def level_info(self, level):
        d = (C.c_int * 4)()
        n, t = C.c_int(), C.c_int()
        _check(lib().ddamg_level_info(self._h, level, d, C.byref(n), C.byref(t)))
        return tuple(d), n.value, t.value


def ddamg_setup(gauge, dims, bc_t, m0, csw, params: DdamgParams, tv_random=None) -> Handle:
    """tv_random = None: the library draws the setup's random vectors from params.seed."""
    d = (C.c_int * 4)(*[int(x) for x in dims])
    if tv_random is None:
        ptrs = None
    else:
        ptrs = (C.c_void_p * MAX_LEVELS)(*[_ptr(t) if t is not None else None for t in tv_random] +
                                         [None] * (MAX_LEVELS - len(tv_random)))
    out = C.c_void_p()
    _check(lib().ddamg_setup(_ptr(gauge), d, int(bc_t), float(m0), float(csw), C.byref(params), ptrs,
                            C.byref(out)))
    return Handle(out, params, dims)


def ddamg_solve(h: Handle, rhs, x, n, tol, with_stats=True, raise_noconv=False):
    stats = (DdamgStats * max(1, n))()
    rc = lib().ddamg_solve(h.raw, _ptr(rhs), _ptr(x), int(n), float(tol), stats if with_stats else None)
    if rc != DDAMG_OK and (rc != DDAMG_ERR_NOCONV or raise_noconv):
        _check(rc)
    return [dict(iterations=s.iterations, cycles=s.cycles, converged=bool(s.converged),
                 true_residual=s.true_residual) for s in stats[:n]]


def ddamg_update_gauge(h: Handle, gauge, n_inv):
    """New gauge field into the hierarchy: operators rebuilt from the current test vectors, n_inv Alg. 4 passes."""
    _check(lib().ddamg_update_gauge(h.raw, _ptr(gauge), int(n_inv)))


def ddamg_cgnr(h: Handle, rhs, x, n, tol, max_iter=100000):
    """FP64 CGNR on the handle's fine operator; per-rhs stats (iterations, converged, true residual)."""
    stats = (DdamgStats * max(1, n))()
    rc = lib().ddamg_cgnr(h.raw, _ptr(rhs), _ptr(x), int(n), float(tol), int(max_iter), stats)
    if rc not in (DDAMG_OK, DDAMG_ERR_NOCONV):
        _check(rc)
    return [dict(iterations=s.iterations, converged=bool(s.converged), true_residual=s.true_residual)
            for s in stats[:n]]


def ddamg_sigma_extremes(h: Handle, steps, seed=0):
    """(sigma_min, sigma_max, steps taken) of the fine operator from the CG Lanczos matrix of D^+ D."""
    a, b, k = C.c_double(), C.c_double(), C.c_int()
    _check(lib().ddamg_sigma_extremes(h.raw, int(steps), C.c_uint64(int(seed)), C.byref(a), C.byref(b),
                                      C.byref(k)))
    return a.value, b.value, k.value


def ddamg_free(h: Handle):
    h.free()


def ddamg_set_stream(h: Handle, stream_ptr):
    _check(lib().ddamg_set_stream(h.raw, C.c_void_p(stream_ptr) if stream_ptr else None))


def ddamg_apply(h, level, precision, inp, out, n):
    _check(lib().ddamg_apply(h.raw, level, precision, _ptr(inp), _ptr(out), n))


def ddamg_smooth(h, level, precision, b, z, n, iterations):
    _check(lib().ddamg_smooth(h.raw, level, precision, _ptr(b), _ptr(z), n, iterations))


def ddamg_restrict(h, level, precision, fine, coarse, n):
    _check(lib().ddamg_restrict(h.raw, level, precision, _ptr(fine), _ptr(coarse), n))


def ddamg_prolong(h, level, precision, coarse, fine, n):
    _check(lib().ddamg_prolong(h.raw, level, precision, _ptr(coarse), _ptr(fine), n))


def ddamg_kcycle(h, level, precision, b, z, n):
    _check(lib().ddamg_kcycle(h.raw, level, precision, _ptr(b), _ptr(z), n))


def ddamg_coarse_solve(h, precision, b, z, n):
    _check(lib().ddamg_coarse_solve(h.raw, precision, _ptr(b), _ptr(z), n))


def ddamg_set_testvectors(h, level, tv, n):
    _check(lib().ddamg_set_testvectors(h.raw, level, _ptr(tv), n))


def ddamg_get_testvectors(h, level, tv, n):
    _check(lib().ddamg_get_testvectors(h.raw, level, _ptr(tv), n))


def ddamg_rebuild(h, level):
    _check(lib().ddamg_rebuild(h.raw, level))


def ddamg_get_interpolation(h, level, P):
    _check(lib().ddamg_get_interpolation(h.raw, level, _ptr(P)))


def ddamg_get_coarse_operator(h, level, blocks):
    _check(lib().ddamg_get_coarse_operator(h.raw, level, _ptr(blocks)))


def ddamg_profile(h, enable):
    _check(lib().ddamg_profile(h.raw, int(enable)))


def ddamg_profile_read(h, kind):
    """(total ms, launches, algorithmic bytes) of a kernel class since profiling was enabled."""
    k = PROF_KINDS[kind] if isinstance(kind, str) else int(kind)
    ms, n, b = C.c_double(), C.c_longlong(), C.c_double()
    _check(lib().ddamg_profile_read(h.raw, k, C.byref(ms), C.byref(n), C.byref(b)))
    return ms.value, n.value, b.value


def ddamg_launch_count():
    return int(lib().ddamg_launch_count())


def ddamg_set_option(h, option, value):
    _check(lib().ddamg_set_option(h.raw, int(option), int(value)))


def ddamg_krylov_steps(h, level, precision):
    n = C.c_longlong()
    _check(lib().ddamg_krylov_steps(h.raw, int(level), int(precision), C.byref(n)))
    return n.value


def ddamg_residual_norm_noalloc(h, rhs, x, n, out):
    """||rhs_i - D x_i|| / ||rhs_i|| into out without any allocation (rhs, x on the device)."""
    _check(lib().ddamg_residual_norm_noalloc(h.raw, _ptr(rhs), _ptr(x), int(n), _ptr(out)))


def ddamg_get_option(h, option):
    v = C.c_int()
    _check(lib().ddamg_get_option(h.raw, int(option), C.byref(v)))
    return v.value


def ddamg_setup_times(h):
    """Setup wall-clock seconds per level: [{"smooth": s, "kcycle": s, "rebuild": s}, ...]."""
    n = MAX_LEVELS * len(SETUP_KINDS)
    buf = (C.c_double * n)()
    _check(lib().ddamg_setup_times(h.raw, buf, n))
    return [dict(zip(SETUP_KINDS, buf[l * len(SETUP_KINDS):(l + 1) * len(SETUP_KINDS)])) for l in range(MAX_LEVELS)]


TUNE_KINDS = {"coarse": 0, "restrict": 1, "prolong": 2, "sap": 3}


def ddamg_autotune_times(h, kind, level):
    """(ms per candidate, -1 where not timed; the candidate in use) of an autotuned kernel class."""
    ms = (C.c_double * 5)()
    ch = C.c_int()
    k = TUNE_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().ddamg_autotune_times(h.raw, k, int(level), ms, C.byref(ch)))
    return list(ms), ch.value


def ddamg_device_bytes(h):
    n = C.c_size_t()
    _check(lib().ddamg_device_bytes(h.raw, C.byref(n)))
    return n.value


def ddamg_estimate_bytes(dims, params):
    """Device bytes a hierarchy with these parameters would hold (host arithmetic, no device call)."""
    d = (C.c_int * 4)(*[int(x) for x in dims])
    n = C.c_size_t()
    _check(lib().ddamg_estimate_bytes(d, C.byref(params), C.byref(n)))
    return n.value


_live_servers = weakref.WeakSet()


@atexit.register
def _stop_servers():
    # worker threads must stop before the interpreter (and the CUDA runtime) shut down
    for s in list(_live_servers):
        try:
            s.free()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over resident hierarchies (ddamg_server_*)."""

    def __init__(self, hbm_budget=0):
        self.raw = C.c_void_p()
        _check(lib().ddamg_server_create(C.c_size_t(int(hbm_budget)), C.byref(self.raw)))
        self._handles = []
        _live_servers.add(self)

    def add(self, h):
        hid = C.c_int()
        _check(lib().ddamg_server_add(self.raw, h.raw, C.byref(hid)))
        self._handles.append(h)
        return hid.value

    def submit(self, hid, rhs, n, tol):
        rid = C.c_longlong()
        _check(lib().ddamg_server_submit(self.raw, int(hid), _ptr(rhs), int(n), float(tol), C.byref(rid)))
        return rid.value

    def poll(self, rid):
        d = C.c_int()
        _check(lib().ddamg_server_poll(self.raw, C.c_longlong(rid), C.byref(d)))
        return bool(d.value)

    def wait(self, rid, x, n, check=True):
        """Solutions into x; returns (per-rhs stats dicts, (queue_s, latency_s, batch_s), return code)."""
        st = (DdamgStats * int(n))()
        t = (C.c_double * 3)()
        rc = lib().ddamg_server_wait(self.raw, C.c_longlong(rid), _ptr(x), st, t)
        if check and rc not in (DDAMG_OK, DDAMG_ERR_NOCONV):
            _check(rc)
        stats = [dict(iterations=s.iterations, cycles=s.cycles, converged=bool(s.converged),
                      true_residual=s.true_residual) for s in st]
        return stats, (t[0], t[1], t[2]), rc

    def free(self):
        if self.raw:
            lib().ddamg_server_free(self.raw)
            self.raw = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
