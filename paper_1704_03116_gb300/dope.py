"""Thin Python binding of the DOPE C-ABI (include/dope.h).

Argument marshalling only: every step of the ADMM path runs in libdope.so's
CUDA kernels.  Each ``dope_*`` function here has the C function's name and
meaning; arrays may be torch CUDA tensors (passed as device pointers, on the
current torch stream unless ``stream`` is given), or numpy arrays / CPU
tensors (passed as host pointers).  There is no CPU fallback: if the library
is missing or fails to load, importing this module raises ImportError.

DOPE: Dolz, Ben Ayed, Desrosiers, "DOPE: Distributed Optimization for
Pairwise Energies" (arXiv 1704.03116), Algorithm 1.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DOPE_LIBRARY=checked selects the checked build (shared-memory index checks
# that record a bad index instead of touching memory; built by
# _build.build(checked=True)); anything else the ordinary library.
LIB_PATH = os.path.join(_HERE, "libdope_checked.so" if os.environ.get("DOPE_LIBRARY") == "checked"
                        else "libdope.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dope.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(_HERE), "include", "dope_potentials.h")]

DOPE_OK, DOPE_EINVAL, DOPE_EUNSUPPORTED, DOPE_ENOMEM = 0, 1, 2, 3
DOPE_EOVERFLOW, DOPE_ENOTCONV, DOPE_ETIMEOUT, DOPE_ECUDA = 4, 5, 6, 7
DOPE_ECANCELED = 8
DOPE_HOST, DOPE_DEVICE = 0, 1


class DopeError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {status} ({_lib.dope_strerror(status).decode()})")


class dope_params(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("mu_fact", ctypes.c_double), ("eps", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("relabel_period", ctypes.c_int),
                ("threads", ctypes.c_int), ("max_pulses", ctypes.c_int), ("fold_rounds", ctypes.c_int),
                ("launch_mode", ctypes.c_int), ("grow", ctypes.c_int * 3), ("lsa_steps", ctypes.c_int),
                ("barrier_timeout_us", ctypes.c_int)]


class dope_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("pulses_total", ctypes.c_int64), ("pulses_max", ctypes.c_int),
                ("free_nodes_total", ctypes.c_int64), ("rmax_last", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("bfs_levels_total", ctypes.c_int64),
                ("bfs_levels_max", ctypes.c_int), ("fold_rounds_max", ctypes.c_int),
                ("phase_cycles", ctypes.c_double * 4), ("loop_cycles", ctypes.c_double * 4),
                ("windows", ctypes.c_int), ("window_iterations", ctypes.c_int),
                ("window_cycles", ctypes.c_double * 8), ("solver_kernel", ctypes.c_int),
                ("reserved", ctypes.c_int), ("blocks_solved", ctypes.c_int64),
                ("blocks_updated", ctypes.c_int64), ("blocks_solved_partial", ctypes.c_int64)]


class dope_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 2), ("ms", ctypes.c_double * 2),
                ("first_iteration_launches", ctypes.c_int64), ("first_iteration_ms", ctypes.c_double),
                ("iterations", ctypes.c_int64)]


class dope_server_params(ctypes.Structure):
    _fields_ = [("hbm_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int), ("mode", ctypes.c_int),
                ("launch_iters", ctypes.c_int), ("reserved", ctypes.c_int)]


class dope_request(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("connectivity", ctypes.c_int), ("grid", ctypes.c_int64 * 3),
                ("block_shape", ctypes.c_int32 * 3), ("lambda_", ctypes.c_double), ("params", dope_params),
                ("use_params", ctypes.c_int), ("where_inputs", ctypes.c_int), ("unaries", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("where_labels", ctypes.c_int),
                ("reserved", ctypes.c_int), ("tag", ctypes.c_uint64), ("image_request", ctypes.c_void_p)]


class dope_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("reserved", ctypes.c_int),
                ("energy_int", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class dope_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "admitted", "completed", "launches", "yields",
                                              "queued", "in_flight", "max_in_flight")] + \
               [(k, ctypes.c_uint64) for k in ("bytes_limit", "bytes_in_use", "bytes_peak")] + \
               [("gpu_launch_s", ctypes.c_double)]


class dope_tune_result(ctypes.Structure):
    _fields_ = [("block_shape", ctypes.c_int32 * 3), ("params", dope_params), ("ms", ctypes.c_double),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("energy_int", ctypes.c_int64),
                ("status", ctypes.c_int), ("reserved", ctypes.c_int)]


DOPE_BATCH_MAX = 256
DOPE_TUNE_BLOCK = 1
DOPE_GMM_MAX_COMP, DOPE_GMM_MAX_CH = 8, 4
DOPE_CONTRAST_WS_BYTES = 64


class dope_gmm(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int), ("channels", ctypes.c_int),
                ("weight", ctypes.c_double * DOPE_GMM_MAX_COMP),
                ("mean", (ctypes.c_double * DOPE_GMM_MAX_CH) * DOPE_GMM_MAX_COMP),
                ("cov", ((ctypes.c_double * DOPE_GMM_MAX_CH) * DOPE_GMM_MAX_CH) * DOPE_GMM_MAX_COMP)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                          "(nvcc, sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "dope_default_params": (None, [P(dope_params)]),
        "dope_create": (i32, [P(ctypes.c_int64), i32, i32, P(ctypes.c_int32), dbl, P(dope_params), P(vp)]),
        "dope_set_unaries": (i32, [vp, vp, i64, i32, vp]),
        "dope_set_weights": (i32, [vp, vp, i64, i32, vp]),
        "dope_set_inputs": (i32, [vp, vp, vp, i64, i32, vp]),
        "dope_solve": (i32, [vp, vp, i32, P(ctypes.c_int64), P(ctypes.c_int), vp]),
        "dope_solve_begin": (i32, [vp, vp, i32, vp]),
        "dope_solve_end": (i32, [vp, P(ctypes.c_int64), P(ctypes.c_int), vp]),
        "dope_reset": (i32, [vp]),
        "dope_iterate": (i32, [vp, i32, P(ctypes.c_int), P(ctypes.c_int), vp]),
        "dope_get_state": (i32, [vp, vp, vp, vp, P(ctypes.c_double), P(ctypes.c_int), vp]),
        "dope_set_state": (i32, [vp, vp, vp, vp, dbl, i32, vp]),
        "dope_shifted_caps": (i32, [vp, vp, vp]),
        "dope_block_cuts": (i32, [vp, vp, vp, vp]),
        "dope_energy": (i32, [vp, vp, i32, P(ctypes.c_int64), vp]),
        "dope_trace": (i32, [vp, vp, i32, P(ctypes.c_int)]),
        "dope_get_stats": (i32, [vp, P(dope_stats)]),
        "dope_get_geometry": (i32, [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int), P(ctypes.c_int)]),
        "dope_set_profiling": (i32, [vp, i32]),
        "dope_get_profile": (i32, [vp, P(dope_profile)]),
        "dope_solve_noalloc": (i32, [P(ctypes.c_int64), i32, i32, P(ctypes.c_int32), dbl, P(dope_params),
                                     vp, vp, vp, P(ctypes.c_int64), P(ctypes.c_int), vp]),
        "dope_iterate_batch": (i32, [P(vp), i32, i32, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), vp]),
        "dope_labels": (i32, [vp, vp, i32, P(ctypes.c_int64), vp]),
        "dope_server_create": (i32, [P(dope_server_params), P(vp)]),
        "dope_server_submit": (i32, [vp, P(dope_request), P(ctypes.c_uint64)]),
        "dope_server_poll": (i32, [vp, P(dope_result), i32, P(ctypes.c_int), dbl]),
        "dope_server_clock": (dbl, [vp]),
        "dope_server_cancel": (i32, [vp, ctypes.c_uint64]),
        "dope_server_get_stats": (i32, [vp, P(dope_server_stats)]),
        "dope_server_destroy": (None, [vp]),
        "dope_autotune": (i32, [P(ctypes.c_int64), i32, i32, P(ctypes.c_int32), dbl, P(dope_params), vp, vp, i32,
                                i32, i32, P(dope_tune_result), i32, P(ctypes.c_int), P(dope_tune_result), vp]),
        "dope_get_block_state": (i32, [vp, vp, vp, i64, P(ctypes.c_int64), vp]),
        "dope_gmm_unaries": (i32, [vp, i64, i32, P(dope_gmm), P(dope_gmm), dbl, vp, vp]),
        "dope_contrast_weights": (i32, [vp, P(ctypes.c_int64), i32, i32, i32, dbl, i32, vp, vp,
                                        P(ctypes.c_double), vp]),
        "dope_set_image": (i32, [vp, vp, i32, P(dope_gmm), P(dope_gmm), dbl, dbl, i32, i32, P(ctypes.c_double), vp]),
        "dope_destroy": (None, [vp]),
        "dope_strerror": (ctypes.c_char_p, [i32]),
        "dope_check_status": (i32, [P(ctypes.c_uint64), i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


try:
    _lib = _load()
except OSError as e:  # pragma: no cover - a broken build must fail loudly
    raise ImportError(f"cannot load {LIB_PATH}: {e}") from e


def declared_symbols(headers=None):
    """Function names declared in include/dope.h and include/dope_potentials.h."""
    names = set()
    for h in headers or HEADERS:
        txt = open(h).read()
        names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dope_[a-z_0-9]+)\s*\(", txt, re.M))
    return sorted(names)


def _check(rc, where):
    if rc not in (DOPE_OK,):
        raise DopeError(rc, where)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(x, dtype):
    """(pointer, where, keepalive) of a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != dtype[1] or not x.is_contiguous():
                raise TypeError(f"expected contiguous {dtype[1]} tensor")
            return ctypes.c_void_p(x.data_ptr()), (DOPE_DEVICE if x.is_cuda else DOPE_HOST), x
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype[0])
    return ctypes.c_void_p(a.ctypes.data), DOPE_HOST, a


def _t(np_dtype):
    import torch
    return (np_dtype, {np.float32: torch.float32, np.int32: torch.int32, np.uint8: torch.uint8,
                       np.int64: torch.int64, np.float64: torch.float64}[np_dtype])


# --------------------------------------------------------------------------
# C-ABI functions (same names)
# --------------------------------------------------------------------------

def dope_check_status(clear=False):
    """Checked build only: (length, index) of the first shared-memory index a
    kernel found outside its array since the last clear, or None.  Raises
    DopeError(DOPE_EUNSUPPORTED) on the ordinary build."""
    w = ctypes.c_uint64(0)
    _check(_lib.dope_check_status(ctypes.byref(w), int(bool(clear))), "dope_check_status")
    if not w.value:
        return None
    v = w.value - 1
    return (v >> 32, v & 0xffffffff)


def dope_default_params():
    p = dope_params()
    _lib.dope_default_params(ctypes.byref(p))
    return p


def dope_create(grid, connectivity, block_shape, lam, params=None):
    grid = [int(g) for g in grid]
    block = [int(b) for b in block_shape]
    if len(grid) != len(block):
        raise ValueError("grid and block_shape must have the same rank")
    g = (ctypes.c_int64 * len(grid))(*grid)
    b = (ctypes.c_int32 * len(block))(*block)
    ctx = ctypes.c_void_p()
    rc = _lib.dope_create(g, len(grid), int(connectivity), b, float(lam),
                          ctypes.byref(params) if params is not None else None, ctypes.byref(ctx))
    _check(rc, "dope_create")
    return ctx


def dope_set_unaries(ctx, u, stream=None):
    p, where, keep = _ptr(u, _t(np.float32))
    _check(_lib.dope_set_unaries(ctx, p, int(np.prod(keep.shape)), where, _stream(stream)), "dope_set_unaries")


def dope_set_weights(ctx, wq, stream=None):
    p, where, keep = _ptr(wq, _t(np.int32))
    n = int(np.prod(keep.shape)) // max(1, int(keep.shape[0])) if len(keep.shape) == 2 else None
    if n is None:
        raise ValueError("wq must be [conn/2, N]")
    _check(_lib.dope_set_weights(ctx, p, n, where, _stream(stream)), "dope_set_weights")


def dope_set_inputs(ctx, u, wq, stream=None):
    """Unaries and weights together, asynchronously (the status is reported
    by the next synchronising call, e.g. dope_solve)."""
    pu, wu, ku = _ptr(u, _t(np.float32))
    pw, ww, kw = _ptr(wq, _t(np.int32))
    if wu != ww:
        raise TypeError("unaries and weights must both be host or both device arrays")
    if len(kw.shape) != 2:
        raise ValueError("wq must be [conn/2, N]")
    _check(_lib.dope_set_inputs(ctx, pu, pw, int(np.prod(ku.shape)), wu, _stream(stream)), "dope_set_inputs")
    return ku, kw


def dope_solve(ctx, labels, stream=None, allow_notconv=False):
    """Runs Algorithm 1; writes labels; returns (E_int, iterations, status)."""
    p, where, keep = _ptr(labels, _t(np.uint8))
    e = ctypes.c_int64(0)
    it = ctypes.c_int(0)
    rc = _lib.dope_solve(ctx, p, where, ctypes.byref(e), ctypes.byref(it), _stream(stream))
    if rc == DOPE_ENOTCONV and allow_notconv:
        return e.value, it.value, rc
    _check(rc, "dope_solve")
    if where == DOPE_HOST and keep is not labels and isinstance(labels, np.ndarray):
        labels[...] = keep.reshape(labels.shape)
    return e.value, it.value, rc


def dope_reset(ctx):
    _check(_lib.dope_reset(ctx), "dope_reset")


def dope_iterate(ctx, n_iter, stream=None):
    done = ctypes.c_int(0)
    conv = ctypes.c_int(0)
    _check(_lib.dope_iterate(ctx, int(n_iter), ctypes.byref(done), ctypes.byref(conv), _stream(stream)),
           "dope_iterate")
    return done.value, bool(conv.value)


def _geom(ctx):
    n, k = ctypes.c_int64(0), ctypes.c_int64(0)
    b, f = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.dope_get_geometry(ctx, ctypes.byref(n), ctypes.byref(k), ctypes.byref(b), ctypes.byref(f)),
           "dope_get_geometry")
    return n.value, k.value, b.value, f.value


def dope_get_geometry(ctx):
    return _geom(ctx)


def dope_get_state(ctx, stream=None, y_only=False):
    """State after the last iteration: y, a, yhat (image order), mu, t.  With
    y_only (required for overlapping partitions, whose a / yhat are per block
    copy: dope_get_block_state) a and yhat are None."""
    n = _geom(ctx)[0]
    y = np.empty(n, np.float64)
    a = None if y_only else np.empty(n, np.float64)
    yh = None if y_only else np.empty(n, np.uint8)
    mu = ctypes.c_double(0)
    t = ctypes.c_int(0)
    _check(_lib.dope_get_state(ctx, y.ctypes.data, None if y_only else a.ctypes.data,
                               None if y_only else yh.ctypes.data, ctypes.byref(mu), ctypes.byref(t),
                               _stream(stream)), "dope_get_state")
    return {"y": y, "a": a, "yhat": yh, "mu": mu.value, "t": t.value}


def dope_set_state(ctx, y, a, yhat, mu, t, stream=None):
    y = np.ascontiguousarray(y, np.float64)
    a = np.ascontiguousarray(a, np.float64)
    yh = np.ascontiguousarray(yhat, np.uint8)
    _check(_lib.dope_set_state(ctx, y.ctypes.data, a.ctypes.data, yh.ctypes.data, float(mu), int(t),
                               _stream(stream)), "dope_set_state")


def dope_shifted_caps(ctx, stream=None):
    n = _geom(ctx)[0]
    C = np.empty(n, np.int64)
    _check(_lib.dope_shifted_caps(ctx, C.ctypes.data, _stream(stream)), "dope_shifted_caps")
    return C


def dope_block_cuts(ctx, C, stream=None):
    C = np.ascontiguousarray(C, np.int64)
    yh = np.empty(C.shape[0], np.uint8)
    _check(_lib.dope_block_cuts(ctx, C.ctypes.data, yh.ctypes.data, _stream(stream)), "dope_block_cuts")
    return yh


def dope_energy(ctx, labels, stream=None):
    p, where, keep = _ptr(labels, _t(np.uint8))
    e = ctypes.c_int64(0)
    _check(_lib.dope_energy(ctx, p, where, ctypes.byref(e), _stream(stream)), "dope_energy")
    return e.value


def dope_trace(ctx, cap=4096):
    r = np.zeros(cap, np.float64)
    cnt = ctypes.c_int(0)
    _check(_lib.dope_trace(ctx, r.ctypes.data, cap, ctypes.byref(cnt)), "dope_trace")
    return r[:cnt.value].copy()


def dope_get_stats(ctx):
    s = dope_stats()
    _check(_lib.dope_get_stats(ctx, ctypes.byref(s)), "dope_get_stats")
    out = {f: getattr(s, f) for f, _ in s._fields_}
    out["phase_cycles"] = list(s.phase_cycles)
    out["loop_cycles"] = list(s.loop_cycles)
    out["window_cycles"] = list(s.window_cycles)
    return out


def dope_set_profiling(ctx, enable):
    _check(_lib.dope_set_profiling(ctx, int(bool(enable))), "dope_set_profiling")


def dope_get_profile(ctx):
    p = dope_profile()
    _check(_lib.dope_get_profile(ctx, ctypes.byref(p)), "dope_get_profile")
    return {"launches": list(p.launches), "ms": list(p.ms),
            "first_iteration_launches": p.first_iteration_launches,
            "first_iteration_ms": p.first_iteration_ms, "iterations": p.iterations}


def dope_solve_noalloc(grid, connectivity, block_shape, lam, u, wq, labels, params=None, stream=None,
                       allow_notconv=False):
    """Allocation-free solve (no context, no device allocation): u, wq and
    labels must be CUDA tensors on the current device with u of N elements,
    wq of shape (conn/2, N) (or conn/2 * N elements) and labels of at least N
    elements, N = prod(grid); the C function takes no lengths, so they are
    checked here before anything runs.  Returns (E_int, iterations, status)."""
    grid = [int(x) for x in grid]
    block = [int(x) for x in block_shape]
    n = int(np.prod(grid)) if grid else 0
    nh = int(connectivity) // 2
    for name, x in (("u", u), ("wq", wq), ("labels", labels)):
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            raise TypeError(f"dope_solve_noalloc takes device tensors ({name})")
    import torch
    cur = torch.cuda.current_device()
    for name, x in (("u", u), ("wq", wq), ("labels", labels)):
        if x.device.index != cur:
            raise ValueError(f"dope_solve_noalloc: {name} is on cuda:{x.device.index}, the current device is "
                             f"cuda:{cur}")
    if u.numel() != n:
        raise ValueError(f"dope_solve_noalloc: u has {u.numel()} elements, the grid {n}")
    if wq.numel() != nh * n or (wq.dim() == 2 and tuple(wq.shape) != (nh, n)):
        raise ValueError(f"dope_solve_noalloc: wq must be ({nh}, {n}), got {tuple(wq.shape)}")
    if labels.numel() < n:
        raise ValueError(f"dope_solve_noalloc: labels has {labels.numel()} elements, needs {n}")
    pu, wu, ku = _ptr(u, _t(np.float32))
    pw, ww, kw = _ptr(wq, _t(np.int32))
    pl, wl, kl = _ptr(labels, _t(np.uint8))
    if not (wu == ww == wl == DOPE_DEVICE):
        raise TypeError("dope_solve_noalloc takes device tensors")
    g = (ctypes.c_int64 * len(grid))(*grid)
    b = (ctypes.c_int32 * len(block))(*block)
    e = ctypes.c_int64(0)
    it = ctypes.c_int(0)
    rc = _lib.dope_solve_noalloc(g, len(grid), int(connectivity), b, float(lam),
                                 ctypes.byref(params) if params is not None else None,
                                 pu, pw, pl, ctypes.byref(e), ctypes.byref(it), _stream(stream))
    if not (rc == DOPE_ENOTCONV and allow_notconv):
        _check(rc, "dope_solve_noalloc")
    return e.value, it.value, rc


def dope_iterate_batch(ctxs, n_iter, stream=None):
    """One batched launch over the contexts; per context (iterations, converged, status)."""
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c if isinstance(c, int) else c.value for c in ctxs])
    it = (ctypes.c_int * n)()
    cv = (ctypes.c_int * n)()
    st = (ctypes.c_int * n)()
    rc = _lib.dope_iterate_batch(arr, n, int(n_iter), it, cv, st, _stream(stream))
    _check(rc, "dope_iterate_batch")
    return [(it[i], bool(cv[i]), st[i]) for i in range(n)]


def dope_labels(ctx, labels, stream=None):
    """Labels of the last iteration into `labels`; returns E_int."""
    p, where, keep = _ptr(labels, _t(np.uint8))
    e = ctypes.c_int64(0)
    _check(_lib.dope_labels(ctx, p, where, ctypes.byref(e), _stream(stream)), "dope_labels")
    if where == DOPE_HOST and keep is not labels and isinstance(labels, np.ndarray):
        labels[...] = keep.reshape(labels.shape)
    return e.value


def dope_server_create(hbm_bytes=0, max_batch=0, mode=0, launch_iters=0):
    p = dope_server_params(int(hbm_bytes), int(max_batch), int(mode), int(launch_iters), 0)
    out = ctypes.c_void_p()
    _check(_lib.dope_server_create(ctypes.byref(p), ctypes.byref(out)), "dope_server_create")
    return out


def dope_server_submit(srv, req):
    rid = ctypes.c_uint64(0)
    _check(_lib.dope_server_submit(srv, ctypes.byref(req), ctypes.byref(rid)), "dope_server_submit")
    return rid.value


def dope_server_poll(srv, cap=256, timeout=0.0):
    buf = (dope_result * cap)()
    n = ctypes.c_int(0)
    _check(_lib.dope_server_poll(srv, buf, cap, ctypes.byref(n), float(timeout)), "dope_server_poll")
    return [buf[i] for i in range(n.value)]


def dope_server_clock(srv):
    return _lib.dope_server_clock(srv)


def dope_server_get_stats(srv):
    st = dope_server_stats()
    _check(_lib.dope_server_get_stats(srv, ctypes.byref(st)), "dope_server_get_stats")
    return {k: getattr(st, k) for k, _ in dope_server_stats._fields_}


def dope_server_destroy(srv):
    _lib.dope_server_destroy(srv)


def _tune_dict(r, ndim):
    p = r.params
    return {"block": tuple(r.block_shape[:ndim]), "relabel_period": p.relabel_period, "threads": p.threads,
            "fold_rounds": p.fold_rounds, "launch_mode": p.launch_mode, "ms": r.ms, "iterations": r.iterations,
            "converged": bool(r.converged), "energy_int": r.energy_int, "status": r.status, "params": p}


def dope_autotune(grid, connectivity, block_shape, lam, u, wq, params=None, flags=0, reps=2, cap=256,
                  stream=None):
    """Stage-wise search of solver settings; returns (best, all_tried) as dicts."""
    grid = [int(g) for g in grid]
    block = [int(b) for b in block_shape]
    pu, wu, ku = _ptr(u, _t(np.float32))
    pw, ww, kw = _ptr(wq, _t(np.int32))
    if wu != ww:
        raise TypeError("unaries and weights must both be host or both device arrays")
    g = (ctypes.c_int64 * len(grid))(*grid)
    b = (ctypes.c_int32 * len(block))(*block)
    out = (dope_tune_result * cap)()
    best = dope_tune_result()
    n = ctypes.c_int(0)
    rc = _lib.dope_autotune(g, len(grid), int(connectivity), b, float(lam),
                            ctypes.byref(params) if params is not None else None, pu, pw, wu, int(flags),
                            int(reps), out, cap, ctypes.byref(n), ctypes.byref(best), _stream(stream))
    _check(rc, "dope_autotune")
    return _tune_dict(best, len(grid)), [_tune_dict(out[i], len(grid)) for i in range(n.value)]


def dope_get_block_state(ctx, stream=None):
    """Overlapping contexts: per-block multipliers a and labels yhat, box-major."""
    n = ctypes.c_int64(0)
    _check(_lib.dope_get_block_state(ctx, None, None, 0, ctypes.byref(n), _stream(stream)),
           "dope_get_block_state")
    a = np.empty(n.value, np.float64)
    yh = np.empty(n.value, np.uint8)
    _check(_lib.dope_get_block_state(ctx, a.ctypes.data, yh.ctypes.data, n.value, ctypes.byref(n),
                                     _stream(stream)), "dope_get_block_state")
    return a, yh


def dope_destroy(ctx):
    _lib.dope_destroy(ctx)


def dope_strerror(status):
    return _lib.dope_strerror(int(status)).decode()


# --------------------------------------------------------------------------
# Convenience object over the same calls
# --------------------------------------------------------------------------

# --------------------------------------------------------------------------
# Whole-image potentials (include/dope_potentials.h)
# --------------------------------------------------------------------------

class dope_image_request(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("channels", ctypes.c_int), ("inv_dist", ctypes.c_int),
                ("clip", ctypes.c_double), ("sigma", ctypes.c_double), ("fg", dope_gmm), ("bg", dope_gmm)]


def gmm(weights, means, covs):
    """A dope_gmm from (weights [K], means [K, C], covs [K, C, C])."""
    w = np.asarray(weights, np.float64).reshape(-1)
    m = np.asarray(means, np.float64).reshape(len(w), -1)
    S = np.asarray(covs, np.float64).reshape(len(w), m.shape[1], m.shape[1])
    if not 1 <= len(w) <= DOPE_GMM_MAX_COMP or not 1 <= m.shape[1] <= DOPE_GMM_MAX_CH:
        raise ValueError("1..8 components of 1..4 channels")
    g = dope_gmm()
    g.n_comp, g.channels = len(w), m.shape[1]
    for j in range(len(w)):
        g.weight[j] = float(w[j])
        for r in range(m.shape[1]):
            g.mean[j][r] = float(m[j, r])
            for c in range(m.shape[1]):
                g.cov[j][r][c] = float(S[j, r, c])
    return g


def _as_gmm(g):
    return g if isinstance(g, dope_gmm) else gmm(*g)


def _dev_tensor(x, what):
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float32 CUDA tensor")
    return x


def dope_gmm_unaries(image, fg, bg, clip=1.0e5, channels=None, out=None, stream=None):
    """u = clip(log p_bg(x) - log p_fg(x)) per pixel of a CUDA image [..., C]
    (pixel-major, channels interleaved); fg / bg: dope_gmm or (weights,
    means, covs).  Returns the float32 CUDA tensor u [N]."""
    import torch
    image = _dev_tensor(image, "image")
    fg, bg = _as_gmm(fg), _as_gmm(bg)
    C = fg.channels if channels is None else int(channels)
    n = image.numel() // C
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=image.device)
    _dev_tensor(out, "out")
    _check(_lib.dope_gmm_unaries(ctypes.c_void_p(image.data_ptr()), n, C, ctypes.byref(fg), ctypes.byref(bg),
                                 float(clip), ctypes.c_void_p(out.data_ptr()), _stream(stream)), "dope_gmm_unaries")
    return out


def dope_contrast_weights(image, grid, connectivity, channels=1, sigma=0.0, inv_dist=False, out=None,
                          stream=None, read_sigma=True):
    """wq [conn/2, N] int32 CUDA tensor of a CUDA image on `grid` ((H, W) or
    (D, H, W)) and the sigma used (sigma <= 0: the mean contrast).  With
    read_sigma=False the call stays asynchronous and the sigma returned is
    None."""
    import torch
    image = _dev_tensor(image, "image")
    grid = tuple(int(g) for g in grid)
    n = int(np.prod(grid))
    nh = int(connectivity) // 2
    if out is None:
        out = torch.empty((nh, n), dtype=torch.int32, device=image.device)
    ws = torch.empty(DOPE_CONTRAST_WS_BYTES // 8, dtype=torch.float64, device=image.device)
    g = (ctypes.c_int64 * len(grid))(*grid)
    sig = ctypes.c_double(0.0)
    _check(_lib.dope_contrast_weights(ctypes.c_void_p(image.data_ptr()), g, len(grid), int(channels),
                                      int(connectivity), float(sigma), int(bool(inv_dist)),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                      ctypes.byref(sig) if read_sigma else None, _stream(stream)),
           "dope_contrast_weights")
    return out, (sig.value if read_sigma else None)


def dope_set_image(ctx, image, fg, bg, clip=1.0e5, sigma=0.0, inv_dist=False, channels=None, stream=None,
                   read_sigma=True):
    """Both potentials of an image (CUDA tensor or host array, [..., C])
    straight into a context; returns the sigma used.  read_sigma=False: no
    synchronisation (returns None; the status is reported by the next
    synchronising call)."""
    fg, bg = _as_gmm(fg), _as_gmm(bg)
    C = fg.channels if channels is None else int(channels)
    p, where, keep = _ptr(image, _t(np.float32))
    sig = ctypes.c_double(0.0)
    _check(_lib.dope_set_image(ctx, p, C, ctypes.byref(fg), ctypes.byref(bg), float(clip), float(sigma),
                               int(bool(inv_dist)), where, ctypes.byref(sig) if read_sigma else None,
                               _stream(stream)), "dope_set_image")
    return sig.value if read_sigma else None


class Dope:
    """One DOPE context: grid, connectivity, block shape, lambda (Algorithm 1 inputs)."""

    def __init__(self, grid, connectivity, block_shape, lam, mu0=None, mu_fact=None, eps=None,
                 max_iter=None, relabel_period=None, threads=None, max_pulses=None, fold_rounds=None,
                 launch_mode=None, grow=None, lsa_steps=None, barrier_timeout_us=None):
        p = dope_default_params()
        for k, v in dict(mu0=mu0, mu_fact=mu_fact, eps=eps, max_iter=max_iter,
                         relabel_period=relabel_period, threads=threads, max_pulses=max_pulses,
                         fold_rounds=fold_rounds, launch_mode=launch_mode, lsa_steps=lsa_steps,
                         barrier_timeout_us=barrier_timeout_us).items():
            if v is not None:
                setattr(p, k, v)
        if grow is not None:
            for i, g in enumerate(grow):
                p.grow[i] = int(g)
        self.grid = tuple(int(g) for g in grid)
        # overlap-path contexts (overlapping partitions, larger kernels) keep
        # their multipliers per block copy
        self.overlap = (grow is not None and any(int(g) for g in grow)) or int(connectivity) not in (4, 8, 6)
        self.ctx = dope_create(grid, connectivity, block_shape, lam, p)
        self.n, self.nblocks, self.block_volume, self.face_size = _geom(self.ctx)

    @classmethod
    def from_instance(cls, inst, **kw):
        kw.setdefault("mu0", inst.get("mu0"))
        d = cls(inst["grid"], inst["conn"], inst["block"], inst["lam"], **kw)
        d.set_unaries(inst["u"])
        d.set_weights(inst["wq"])
        return d

    def set_unaries(self, u, stream=None):
        dope_set_unaries(self.ctx, u, stream)

    def set_weights(self, wq, stream=None):
        dope_set_weights(self.ctx, wq, stream)

    def set_image(self, image, fg, bg, clip=1.0e5, sigma=0.0, inv_dist=False, stream=None, read_sigma=True):
        """Unaries and weights computed on the GPU from the image; returns sigma
        (None with read_sigma=False, which does not synchronise)."""
        return dope_set_image(self.ctx, image, fg, bg, clip, sigma, inv_dist, stream=stream, read_sigma=read_sigma)

    def set_inputs(self, u, wq, stream=None):
        """Unaries and weights together, without synchronising (errors are
        reported by the next solve)."""
        self._inputs = dope_set_inputs(self.ctx, u, wq, stream)

    def solve(self, labels=None, stream=None, allow_notconv=False):
        """(labels, E = E_int / 1024, iterations)."""
        if labels is None:
            labels = np.empty(self.n, np.uint8)
        e, it, _ = dope_solve(self.ctx, labels, stream, allow_notconv)
        return labels, e / 1024.0, it

    def solve_begin(self, labels=None, stream=None):
        """Issue a solve without waiting (see solve_end); returns the labels
        buffer, valid once solve_end has returned."""
        if labels is None:
            labels = np.empty(self.n, np.uint8)
        if isinstance(labels, np.ndarray):
            if labels.dtype != np.uint8 or not labels.flags.c_contiguous:
                raise TypeError("labels must be a contiguous uint8 array")
            p, where, keep = ctypes.c_void_p(labels.ctypes.data), DOPE_HOST, labels
        else:
            p, where, keep = _ptr(labels, _t(np.uint8))
        _check(_lib.dope_solve_begin(self.ctx, p, where, _stream(stream)), "dope_solve_begin")
        self._begun = keep
        return labels

    def solve_end(self, stream=None, allow_notconv=False):
        """Wait for the solve solve_begin issued: (labels, E = E_int / 1024, iterations)."""
        e = ctypes.c_int64(0)
        it = ctypes.c_int(0)
        rc = _lib.dope_solve_end(self.ctx, ctypes.byref(e), ctypes.byref(it), _stream(stream))
        labels, self._begun = getattr(self, "_begun", None), None
        if not (rc == DOPE_ENOTCONV and allow_notconv):
            _check(rc, "dope_solve_end")
        return labels, e.value / 1024.0, it.value

    def iterate(self, n, stream=None):
        return dope_iterate(self.ctx, n, stream)

    def reset(self):
        dope_reset(self.ctx)

    def get_state(self):
        return dope_get_state(self.ctx, y_only=self.overlap)

    def set_state(self, y, a, yhat, mu, t):
        dope_set_state(self.ctx, y, a, yhat, mu, t)

    def shifted_caps(self):
        return dope_shifted_caps(self.ctx)

    def block_cuts(self, C):
        return dope_block_cuts(self.ctx, C)

    def energy_int(self, labels):
        return dope_energy(self.ctx, labels)

    def trace(self):
        return dope_trace(self.ctx)

    def stats(self):
        return dope_get_stats(self.ctx)

    def set_profiling(self, on=True):
        dope_set_profiling(self.ctx, on)

    def profile(self):
        return dope_get_profile(self.ctx)

    def block_state(self):
        """(a, yhat) per block copy, box-major (overlapping partitions)."""
        return dope_get_block_state(self.ctx)

    def energy_trace(self, max_iter=1000, stream=None):
        """Algorithm 1 from its initial state one iteration at a time (the same
        iterates as a solve), recording after each iteration t the energy
        E_int(yhat_t) (computed on the device), the number of labels that
        differ from iteration t - 1 (from all-background at t = 1), and the
        largest block residual.  Returns a dict of lists; the energy evolution
        Section 4 plots per ADMM iteration."""
        self.reset()
        energies, flips = [], []
        prev = np.zeros(self.n, np.uint8)
        lab = np.empty(self.n, np.uint8)
        for _ in range(int(max_iter)):
            _, conv = dope_iterate(self.ctx, 1, stream)
            energies.append(dope_labels(self.ctx, lab, stream))
            flips.append(int(np.count_nonzero(lab != prev)))
            prev[...] = lab
            if conv:
                break
        return {"energy_int": energies, "flips": flips, "rmax": self.trace().tolist(),
                "labels": prev.copy()}

    def labels(self, labels=None, stream=None):
        """(labels, E_int) of the last iteration run."""
        if labels is None:
            labels = np.empty(self.n, np.uint8)
        e = dope_labels(self.ctx, labels, stream)
        return labels, e

    def close(self):
        if self.ctx:
            dope_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def iterate_batch(solvers, n_iter, stream=None):
    """dope_iterate_batch over Dope objects."""
    return dope_iterate_batch([d.ctx for d in solvers], n_iter, stream)


class Server:
    """Request server (continuous batching): submit solves, poll results.

    Buffers handed to ``submit`` are kept referenced here until their result
    has been polled."""

    def __init__(self, hbm_bytes=0, max_batch=0, mode=0, launch_iters=0):
        self.srv = dope_server_create(hbm_bytes, max_batch, mode, launch_iters)
        self._keep = {}

    def submit(self, grid, connectivity, block_shape, lam, u, wq, labels, params=None, tag=0):
        grid = [int(g) for g in grid]
        block = [int(b) for b in block_shape]
        if len(grid) != len(block) or len(grid) not in (2, 3):
            raise ValueError("grid and block_shape must both have rank 2 or 3")
        pu, wu, ku = _ptr(u, _t(np.float32))
        pw, ww, kw = _ptr(wq, _t(np.int32))
        if wu != ww:
            raise TypeError("unaries and weights must both be host or both device arrays")
        if isinstance(labels, np.ndarray):
            if labels.dtype != np.uint8 or not labels.flags.c_contiguous:
                raise TypeError("labels must be a contiguous uint8 array")
            pl, wl, kl = ctypes.c_void_p(labels.ctypes.data), DOPE_HOST, labels
        else:
            pl, wl, kl = _ptr(labels, _t(np.uint8))
        r = dope_request()
        r.ndim = len(grid)
        r.connectivity = int(connectivity)
        for i in range(len(grid)):
            r.grid[i] = grid[i]
            r.block_shape[i] = block[i]
        r.lambda_ = float(lam)
        if params is not None:
            r.params = params
            r.use_params = 1
        r.where_inputs = wu
        r.unaries, r.weights, r.labels = pu, pw, pl
        r.where_labels = wl
        r.tag = int(tag)
        rid = dope_server_submit(self.srv, r)
        self._keep[rid] = (ku, kw, kl)
        return rid

    def submit_image(self, grid, connectivity, block_shape, lam, image, fg, bg, labels, clip=1.0e5, sigma=0.0,
                     inv_dist=False, params=None, tag=0):
        """Queue a solve whose potentials the server computes on the GPU from
        `image` ([..., C] float32, host array or CUDA tensor; fg / bg:
        dope_gmm or (weights, means, covs))."""
        grid = [int(g) for g in grid]
        block = [int(b) for b in block_shape]
        if len(grid) != len(block) or len(grid) not in (2, 3):
            raise ValueError("grid and block_shape must both have rank 2 or 3")
        fg, bg = _as_gmm(fg), _as_gmm(bg)
        pi, wi, ki = _ptr(image, _t(np.float32))
        if isinstance(labels, np.ndarray):
            if labels.dtype != np.uint8 or not labels.flags.c_contiguous:
                raise TypeError("labels must be a contiguous uint8 array")
            pl, wl, kl = ctypes.c_void_p(labels.ctypes.data), DOPE_HOST, labels
        else:
            pl, wl, kl = _ptr(labels, _t(np.uint8))
        q = dope_image_request()
        q.image, q.channels, q.inv_dist = pi, fg.channels, int(bool(inv_dist))
        q.clip, q.sigma, q.fg, q.bg = float(clip), float(sigma), fg, bg
        r = dope_request()
        r.ndim = len(grid)
        r.connectivity = int(connectivity)
        for i in range(len(grid)):
            r.grid[i] = grid[i]
            r.block_shape[i] = block[i]
        r.lambda_ = float(lam)
        if params is not None:
            r.params = params
            r.use_params = 1
        r.where_inputs = wi
        r.labels = pl
        r.where_labels = wl
        r.tag = int(tag)
        r.image_request = ctypes.cast(ctypes.pointer(q), ctypes.c_void_p)
        rid = dope_server_submit(self.srv, r)      # the server copies q
        self._keep[rid] = (ki, kl)
        return rid

    def poll(self, timeout=0.0, cap=256):
        out = []
        for r in dope_server_poll(self.srv, cap, timeout):
            self._keep.pop(r.id, None)
            out.append({"id": r.id, "tag": r.tag, "status": r.status, "iterations": r.iterations,
                        "converged": bool(r.converged), "energy_int": r.energy_int,
                        "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done})
        return out

    def cancel(self, rid):
        """Cancel a submitted request (its result then has status DOPE_ECANCELED,
        unless it had already finished)."""
        _check(_lib.dope_server_cancel(self.srv, ctypes.c_uint64(int(rid))), "dope_server_cancel")

    def clock(self):
        return dope_server_clock(self.srv)

    def stats(self):
        return dope_server_get_stats(self.srv)

    def close(self):
        if self.srv:
            dope_server_destroy(self.srv)
            self.srv = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
