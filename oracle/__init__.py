"""DOPE oracle -- TEST INFRASTRUCTURE ONLY.

Plain CPU implementation of the DOPE ADMM path (Dolz, Ben Ayed, Desrosiers,
arXiv 1704.03116) used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package.  It shares no code with
``paper_1704_03116_gb300``: neither imports the other.

The arithmetic lives in ``dope_oracle.c`` (FP64, one IEEE rounding per
operation, built with ``-ffp-contract=off``); this module only compiles it and
marshals numpy arrays.  ``theorem1.py`` holds the literal matrix form of
Theorem 1 / Eq. 8 / Eq. 10 / Eq. 11 (dense numpy, small grids only).

Conventions (Section 2 of the paper, Eq. 1-3):
  * grids are (D, H, W) with D = 1 for 2-D, pixel index (z*H + y)*W + x;
  * ``wq`` is int32 [conn/2, N]: weight of the edge from pixel i to its
    forward neighbour along offset k (2-D 4-conn: (0,+1), (+1,0); 8-conn adds
    (+1,+1), (+1,-1); 3-D 6-conn: (0,0,+1), (0,+1,0), (+1,0,0)), x1024;
  * U = rne(1024 u), Wl = rne(lambda * wq), E_int = U.y + sum Wl |y_i - y_j|
    (each undirected edge once), E = E_int / 1024;
  * labels: 1 = foreground = sink side.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dope_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_F64P = ctypes.POINTER(ctypes.c_double)
_F32P = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile dope_oracle.c into _liboracle.so (OpenMP if the compiler has it)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-lm"], check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    geo = [_I64P, ctypes.c_int, _I32P]
    lib.orc_quantise.argtypes = geo + [_F32P, _I32P, ctypes.c_double, _I64P, _I64P]
    lib.orc_quantise.restype = ctypes.c_int
    lib.orc_energy.argtypes = geo + [_I64P, _I64P, _U8P]
    lib.orc_energy.restype = ctypes.c_int64
    lib.orc_bk_mincut.argtypes = [ctypes.c_int, _I64P, ctypes.c_int, _I32P, _I32P, _I64P, _I64P, _U8P]
    lib.orc_bk_mincut.restype = ctypes.c_int
    lib.orc_bruteforce.argtypes = [ctypes.c_int, _I64P, ctypes.c_int, _I32P, _I32P, _I64P,
                                   _I64P, _U8P, _U8P, _I64P]
    lib.orc_bruteforce.restype = ctypes.c_int
    lib.orc_shifted_caps.argtypes = geo + [_I64P, _I64P, _F64P, _F64P, ctypes.c_double, _F64P, _I64P]
    lib.orc_shifted_caps.restype = ctypes.c_int
    lib.orc_block_cuts.argtypes = geo + [_I64P, _I64P, _U8P]
    lib.orc_block_cuts.restype = ctypes.c_int
    lib.orc_update.argtypes = geo + [_I64P, _U8P, ctypes.c_double, _F64P, _F64P, _F64P]
    lib.orc_update.restype = ctypes.c_int
    lib.orc_admm.argtypes = geo + [_I64P, _I64P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _U8P, ctypes.POINTER(ctypes.c_int), _F64P, _I64P,
                                   _F64P, _F64P, _F64P]
    lib.orc_admm.restype = ctypes.c_int
    lib.orc_admm_step.argtypes = geo + [_I64P, _I64P, ctypes.c_double, _F64P, _F64P, _U8P, _F64P]
    lib.orc_admm_step.restype = ctypes.c_int
    lib.orc_global_mincut.argtypes = geo + [_I64P, _I64P, _U8P]
    lib.orc_global_mincut.restype = ctypes.c_int64
    ov = geo + [_I32P]
    lib.orc_ov_geometry.argtypes = ov + [_I32P, _I32P, ctypes.POINTER(ctypes.c_int), _I64P]
    lib.orc_ov_geometry.restype = ctypes.c_int
    lib.orc_ov_caps.argtypes = ov + [_I64P, _I64P, _F64P, _F64P, ctypes.c_double, _F64P, _I64P]
    lib.orc_ov_caps.restype = ctypes.c_int
    lib.orc_ov_block_cuts.argtypes = ov + [_I64P, _I64P, _U8P]
    lib.orc_ov_block_cuts.restype = ctypes.c_int
    lib.orc_ov_update.argtypes = ov + [_I64P, _U8P, ctypes.c_double, _F64P, _F64P, _F64P]
    lib.orc_ov_update.restype = ctypes.c_int
    lib.orc_ov_labels.argtypes = ov + [_U8P, _U8P]
    lib.orc_ov_labels.restype = ctypes.c_int
    lib.orc_ov_admm.argtypes = ov + [_I64P, _I64P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _U8P, ctypes.POINTER(ctypes.c_int), _F64P, _F64P, _F64P,
                                     _U8P, _F64P]
    lib.orc_ov_admm.restype = ctypes.c_int
    lib.orc_quantise_signed.argtypes = geo + [_F32P, _I32P, ctypes.c_double, _I64P, _I64P]
    lib.orc_quantise_signed.restype = ctypes.c_int
    lib.orc_nsm_block_solve.argtypes = geo + [_I64P, _I64P, _U8P, ctypes.c_int]
    lib.orc_nsm_block_solve.restype = ctypes.c_int
    lib.orc_nsm_admm.argtypes = geo + [_I64P, _I64P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, _U8P, ctypes.POINTER(ctypes.c_int), _F64P,
                                       _F64P, _F64P, _F64P]
    lib.orc_nsm_admm.restype = ctypes.c_int
    lib.orc_lsa_tr_block_trace.argtypes = geo[:3] + [_I64P, ctypes.c_int64, _I64P, _U8P, ctypes.c_int,
                                                      ctypes.c_int, _U8P, _U8P, _I64P, _I64P, _I64P, _I64P,
                                                      _I64P, _I64P, ctypes.POINTER(ctypes.c_int)]
    lib.orc_lsa_tr_block_trace.restype = ctypes.c_int
    lib.orc_lsa_tr_global.argtypes = [_I64P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, _U8P]
    lib.orc_lsa_tr_global.restype = ctypes.c_int64
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_set_threads.restype = None
    _lib = lib
    return lib


def _p(arr, typ):
    return arr.ctypes.data_as(typ)


def _c(arr, dtype):
    return np.ascontiguousarray(arr, dtype=dtype)


@dataclass
class Instance:
    """A quantised DOPE instance (Eq. 1 with integer fixed-point potentials)."""
    dims: tuple          # (D, H, W), D = 1 for 2-D
    conn: int            # 4, 8 or 6
    block: tuple         # (bd, bh, bw)
    U: np.ndarray        # int64 [N]        = rne(1024 u)
    Wl: np.ndarray       # int64 [conn/2, N] = rne(lambda wq)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    @property
    def nblocks(self) -> int:
        D, H, W = self.dims
        bd, bh, bw = self.block
        return (D // bd) * (H // bh) * (W // bw)

    def _geo(self):
        d = _c(self.dims, np.int64)
        b = _c(self.block, np.int32)
        self._keep = (d, b)
        return [_p(d, _I64P), int(self.conn), _p(b, _I32P)]


def _dims3(grid):
    grid = tuple(int(g) for g in grid)
    return grid if len(grid) == 3 else (1,) + grid


def quantise(grid, conn, block, u, wq, lam, signed=False) -> Instance:
    """Instance canonicalisation: U = rne(1024 u), Wl = rne(lambda wq) (FP64).
    signed=True accepts negative weights (non-submodular instances)."""
    lib = _load()
    dims, blk = _dims3(grid), _dims3(block)
    n = int(np.prod(dims))
    u = _c(u, np.float32).reshape(-1)
    wq = _c(wq, np.int32).reshape(conn // 2, n)
    U = np.empty(n, np.int64)
    Wl = np.empty((conn // 2, n), np.int64)
    inst = Instance(dims, conn, blk, U, Wl)
    fn = lib.orc_quantise_signed if signed else lib.orc_quantise
    rc = fn(*inst._geo(), _p(u, _F32P), _p(wq, _I32P), float(lam), _p(U, _I64P), _p(Wl, _I64P))
    if rc != 0:
        raise ValueError(f"orc_quantise failed: {rc}")
    return inst


def energy(inst: Instance, labels) -> int:
    """E_int of Eq. 1 (x1024, int64)."""
    lab = _c(labels, np.uint8).reshape(-1)
    return int(_load().orc_energy(*inst._geo(), _p(_c(inst.U, np.int64), _I64P),
                                  _p(_c(inst.Wl, np.int64), _I64P), _p(lab, _U8P)))


def shifted_caps(inst: Instance, y, a, mu):
    """Eq. 8 unaries x1024: (unrounded double s, rne int64 C)."""
    y = _c(y, np.float64).reshape(-1)
    a = _c(a, np.float64).reshape(-1)
    s = np.empty(inst.n, np.float64)
    C = np.empty(inst.n, np.int64)
    rc = _load().orc_shifted_caps(*inst._geo(), _p(inst.U, _I64P), _p(inst.Wl, _I64P),
                                  _p(y, _F64P), _p(a, _F64P), float(mu), _p(s, _F64P), _p(C, _I64P))
    assert rc == 0
    return s, C


def block_cuts(inst: Instance, C):
    """Canonical exact minimiser of Eq. 8 in every block, given int64 unaries C."""
    C = _c(C, np.int64).reshape(-1)
    yhat = np.empty(inst.n, np.uint8)
    rc = _load().orc_block_cuts(*inst._geo(), _p(inst.Wl, _I64P), _p(C, _I64P), _p(yhat, _U8P))
    assert rc == 0
    return yhat


def update(inst: Instance, yhat, mu, y, a):
    """Eq. 10 / Eq. 11 (returns new y, a and per-block ||yhat_k - S_k y||^2)."""
    y = np.array(y, dtype=np.float64).reshape(-1)
    a = np.array(a, dtype=np.float64).reshape(-1)
    yh = _c(yhat, np.uint8).reshape(-1)
    r2 = np.empty(inst.nblocks, np.float64)
    rc = _load().orc_update(*inst._geo(), _p(inst.Wl, _I64P), _p(yh, _U8P), float(mu),
                            _p(y, _F64P), _p(a, _F64P), _p(r2, _F64P))
    assert rc == 0
    return y, a, r2


def admm_step(inst: Instance, mu, y, a):
    """One iteration of Algorithm 1 from state (y, a, mu): (yhat, y', a', r2)."""
    y = np.array(y, dtype=np.float64).reshape(-1)
    a = np.array(a, dtype=np.float64).reshape(-1)
    yhat = np.empty(inst.n, np.uint8)
    r2 = np.empty(inst.nblocks, np.float64)
    rc = _load().orc_admm_step(*inst._geo(), _p(inst.U, _I64P), _p(inst.Wl, _I64P), float(mu),
                               _p(y, _F64P), _p(a, _F64P), _p(yhat, _U8P), _p(r2, _F64P))
    assert rc == 0
    return yhat, y, a, r2


def admm(inst: Instance, mu0, mu_fact=1.05, eps=1e-3, max_iter=1000):
    """Algorithm 1 to convergence; returns a dict with labels, iterations, traces, state."""
    n = inst.n
    labels = np.empty(n, np.uint8)
    iters = ctypes.c_int(0)
    rmax = np.zeros(max_iter, np.float64)
    flips = np.zeros(max_iter, np.int64)
    y = np.empty(n, np.float64)
    a = np.empty(n, np.float64)
    mu = np.zeros(1, np.float64)
    rc = _load().orc_admm(*inst._geo(), _p(inst.U, _I64P), _p(inst.Wl, _I64P), float(mu0),
                          float(mu_fact), float(eps), int(max_iter), _p(labels, _U8P),
                          ctypes.byref(iters), _p(rmax, _F64P), _p(flips, _I64P),
                          _p(y, _F64P), _p(a, _F64P), _p(mu, _F64P))
    if rc < 0:
        raise RuntimeError(f"orc_admm failed: {rc}")
    t = iters.value
    return {"labels": labels, "iterations": t, "converged": rc == 0,
            "rmax": rmax[:t].copy(), "flips": flips[:t].copy(), "y": y, "a": a,
            "mu": float(mu[0]), "energy": energy(inst, labels)}


def global_mincut(inst: Instance):
    """sGC: canonical exact global minimiser of Eq. 1 by BK; (labels, E_int)."""
    labels = np.empty(inst.n, np.uint8)
    e = _load().orc_global_mincut(*inst._geo(), _p(inst.U, _I64P), _p(inst.Wl, _I64P), _p(labels, _U8P))
    if e == np.iinfo(np.int64).min:
        raise RuntimeError("orc_global_mincut failed")
    return labels, int(e)


def bk_mincut(n, c, eu, ev, cuv, cvu):
    """Canonical min-cut of sum c_i y_i + sum cuv (1-y_u) y_v + cvu y_u (1-y_v)."""
    c = _c(c, np.int64)
    eu, ev = _c(eu, np.int32), _c(ev, np.int32)
    cuv, cvu = _c(cuv, np.int64), _c(cvu, np.int64)
    lab = np.empty(n, np.uint8)
    rc = _load().orc_bk_mincut(int(n), _p(c, _I64P), len(eu), _p(eu, _I32P), _p(ev, _I32P),
                               _p(cuv, _I64P), _p(cvu, _I64P), _p(lab, _U8P))
    if rc != 0:
        raise ValueError(f"orc_bk_mincut failed: {rc}")
    return lab


def bruteforce(n, c, eu, ev, w):
    """min over y in {0,1}^n of sum c_i y_i + sum w_e |y_u - y_v| (any sign of w)."""
    c = _c(c, np.int64)
    eu, ev, w = _c(eu, np.int32), _c(ev, np.int32), _c(w, np.int64)
    emin = ctypes.c_int64(0)
    cnt = ctypes.c_int64(0)
    a = np.empty(n, np.uint8)
    o = np.empty(n, np.uint8)
    rc = _load().orc_bruteforce(int(n), _p(c, _I64P), len(eu), _p(eu, _I32P), _p(ev, _I32P),
                                _p(w, _I64P), ctypes.byref(emin), _p(a, _U8P), _p(o, _U8P),
                                ctypes.byref(cnt))
    if rc != 0:
        raise ValueError("bruteforce: n too large")
    return int(emin.value), a, o, int(cnt.value)


def grid_edges(inst: Instance, within_blocks: bool = False):
    """Edge list (u, v, Wl) of the grid (each undirected edge once), optionally
    only the edges whose two ends share a block.  Plain numpy, for tests."""
    D, H, W = inst.dims
    from .theorem1 import _OFFS
    offs = _OFFS[inst.conn]
    bd, bh, bw = inst.block
    eu, ev, ww = [], [], []
    for k, (dz, dy, dx) in enumerate(offs):
        for z in range(D):
            for y in range(H):
                for x in range(W):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if not (0 <= zz < D and 0 <= yy < H and 0 <= xx < W):
                        continue
                    if within_blocks and (z // bd, y // bh, x // bw) != (zz // bd, yy // bh, xx // bw):
                        continue
                    i = (z * H + y) * W + x
                    j = (zz * H + yy) * W + xx
                    eu.append(i); ev.append(j); ww.append(int(inst.Wl[k, i]))
    return np.array(eu, np.int32), np.array(ev, np.int32), np.array(ww, np.int64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# Overlapping blocks (Q != I): every tile of `block` grown by `grow` pixels per
# side (clipped to the grid).  Block state (a, yhat, Eq. 8 unaries) is stored
# per block as the full box of (block + 2 grow) pixels, box-major; box nodes
# outside the grid are phantoms (0).
# --------------------------------------------------------------------------

class Overlap:
    """Geometry of an overlapping partition: q (Proposition 1's q_ii per pixel,
    image order), box extent, M = qmax^2 (integer scale of every block's Eq. 8
    objective), K."""

    def __init__(self, inst: Instance, grow):
        self.inst = inst
        self.grow = _dims3(grow) if len(tuple(grow)) < 3 else tuple(int(g) for g in grow)
        self._g = _c(self.grow, np.int32)
        q = np.empty(inst.n, np.int32)
        box = np.empty(3, np.int32)
        M = ctypes.c_int(0)
        K = np.zeros(1, np.int64)
        rc = _load().orc_ov_geometry(*inst._geo(), _p(self._g, _I32P), _p(q, _I32P), _p(box, _I32P),
                                     ctypes.byref(M), _p(K, _I64P))
        if rc != 0:
            raise ValueError("invalid overlap (needs 2 grow <= block on every axis)")
        self.q, self.box, self.M, self.K = q, tuple(int(b) for b in box), int(M.value), int(K[0])
        self.eb = int(np.prod(self.box))

    def _args(self):
        return self.inst._geo() + [_p(self._g, _I32P)]

    def caps(self, y, a, mu):
        """Eq. 8 unaries of every box node: (s = x1024 double, C = rne(M s))."""
        y = _c(y, np.float64).reshape(-1)
        a = _c(a, np.float64).reshape(-1)
        s = np.empty(self.K * self.eb, np.float64)
        C = np.empty(self.K * self.eb, np.int64)
        rc = _load().orc_ov_caps(*self._args(), _p(self.inst.U, _I64P), _p(self.inst.Wl, _I64P),
                                 _p(y, _F64P), _p(a, _F64P), float(mu), _p(s, _F64P), _p(C, _I64P))
        assert rc == 0
        return s, C

    def block_cuts(self, C):
        C = _c(C, np.int64).reshape(-1)
        yh = np.empty(self.K * self.eb, np.uint8)
        rc = _load().orc_ov_block_cuts(*self._args(), _p(self.inst.Wl, _I64P), _p(C, _I64P), _p(yh, _U8P))
        assert rc == 0
        return yh

    def update(self, yhat, mu, y, a):
        """Eq. 10 / Eq. 11: (y, a, r2) from block labels (box-major)."""
        y = np.array(y, dtype=np.float64).reshape(-1)
        a = np.array(a, dtype=np.float64).reshape(-1)
        yh = _c(yhat, np.uint8).reshape(-1)
        r2 = np.empty(self.K, np.float64)
        rc = _load().orc_ov_update(*self._args(), _p(self.inst.Wl, _I64P), _p(yh, _U8P), float(mu),
                                   _p(y, _F64P), _p(a, _F64P), _p(r2, _F64P))
        assert rc == 0
        return y, a, r2

    def labels(self, yhat):
        """Proposition 1 output: strict majority of the block copies."""
        yh = _c(yhat, np.uint8).reshape(-1)
        lab = np.empty(self.inst.n, np.uint8)
        assert _load().orc_ov_labels(*self._args(), _p(yh, _U8P), _p(lab, _U8P)) == 0
        return lab

    def step(self, mu, y, a):
        """One Algorithm 1 iteration: (yhat, y', a', r2)."""
        s, C = self.caps(y, a, mu)
        yh = self.block_cuts(C)
        y2, a2, r2 = self.update(yh, mu, y, a)
        return yh, y2, a2, r2

    def admm(self, mu0, mu_fact=1.05, eps=1e-3, max_iter=1000):
        n = self.inst.n
        labels = np.empty(n, np.uint8)
        iters = ctypes.c_int(0)
        rmax = np.zeros(max_iter, np.float64)
        y = np.empty(n, np.float64)
        a = np.empty(self.K * self.eb, np.float64)
        yh = np.empty(self.K * self.eb, np.uint8)
        mu = np.zeros(1, np.float64)
        rc = _load().orc_ov_admm(*self._args(), _p(self.inst.U, _I64P), _p(self.inst.Wl, _I64P),
                                 float(mu0), float(mu_fact), float(eps), int(max_iter), _p(labels, _U8P),
                                 ctypes.byref(iters), _p(rmax, _F64P), _p(y, _F64P), _p(a, _F64P),
                                 _p(yh, _U8P), _p(mu, _F64P))
        if rc < 0:
            raise RuntimeError(f"orc_ov_admm failed: {rc}")
        t = iters.value
        return {"labels": labels, "iterations": t, "converged": rc == 0, "rmax": rmax[:t].copy(),
                "y": y, "a": a, "yhat": yh, "mu": float(mu[0]), "energy": energy(self.inst, labels)}

    def box_pixels(self):
        """Pixel index of every box node (box-major, -1 for phantoms), plain numpy."""
        D, H, W = self.inst.dims
        bd, bh, bw = self.inst.block
        gd, gh, gw = self.grow
        ed, eh, ew = self.box
        out = np.full(self.K * self.eb, -1, np.int64)
        nbz, nby, nbx = D // bd, H // bh, W // bw
        lz, ly, lx = np.meshgrid(np.arange(ed), np.arange(eh), np.arange(ew), indexing="ij")
        for k in range(self.K):
            kz, ky, kx = k // (nby * nbx), (k // nbx) % nby, k % nbx
            z, y, x = kz * bd - gd + lz, ky * bh - gh + ly, kx * bw - gw + lx
            ok = (z >= 0) & (z < D) & (y >= 0) & (y < H) & (x >= 0) & (x < W)
            idx = np.where(ok, (z * H + y) * W + x, -1).reshape(-1)
            out[k * self.eb:(k + 1) * self.eb] = idx
        return out


# --------------------------------------------------------------------------
# Non-submodular blocks: LSA-TR (trust-region local submodular approximation)
# --------------------------------------------------------------------------

LSA_STEPS = 16


def nsm_block_solve(inst: Instance, C, yhat, steps=LSA_STEPS):
    """Every block's Eq. 8 by LSA-TR from the labels yhat (image order)."""
    C = _c(C, np.int64).reshape(-1)
    yh = np.array(yhat, dtype=np.uint8).reshape(-1)
    assert _load().orc_nsm_block_solve(*inst._geo(), _p(inst.Wl, _I64P), _p(C, _I64P), _p(yh, _U8P),
                                       int(steps)) == 0
    return yh


def nsm_step(inst: Instance, mu, y, a, yhat, steps=LSA_STEPS):
    """One Algorithm 1 iteration with LSA-TR blocks: (yhat', y', a', r2)."""
    s, C = shifted_caps(inst, y, a, mu)
    yh = nsm_block_solve(inst, C, yhat, steps)
    y2, a2, r2 = update(inst, yh, mu, y, a)
    return yh, y2, a2, r2


def nsm_admm(inst: Instance, mu0, mu_fact=1.05, eps=1e-3, max_iter=1000, steps=LSA_STEPS):
    n = inst.n
    labels = np.empty(n, np.uint8)
    iters = ctypes.c_int(0)
    rmax = np.zeros(max_iter, np.float64)
    y = np.empty(n, np.float64)
    a = np.empty(n, np.float64)
    mu = np.zeros(1, np.float64)
    rc = _load().orc_nsm_admm(*inst._geo(), _p(inst.U, _I64P), _p(inst.Wl, _I64P), float(mu0), float(mu_fact),
                              float(eps), int(max_iter), int(steps), _p(labels, _U8P), ctypes.byref(iters),
                              _p(rmax, _F64P), _p(y, _F64P), _p(a, _F64P), _p(mu, _F64P))
    if rc < 0:
        raise RuntimeError(f"orc_nsm_admm failed: {rc}")
    t = iters.value
    return {"labels": labels, "iterations": t, "converged": rc == 0, "rmax": rmax[:t].copy(), "y": y,
            "a": a, "mu": float(mu[0]), "energy": energy(inst, labels)}


def lsa_tr_block_trace(inst: Instance, k, Cb, x0, steps=LSA_STEPS):
    """LSA-TR on block k alone from labels x0 (block-local order) with block
    unaries Cb, recording every step: a list of dicts with the expansion point
    x_in, the approximation's unaries `un` and constant `cst`, the trust-region
    weight `lam`, the minimiser x_out, E(x_in) `ecur`, the approximation at the
    minimiser `ap`, E(minimiser) `enew`, and `accepted`; plus the final labels."""
    B = int(np.prod(inst.block))
    Cb = _c(Cb, np.int64).reshape(-1)
    x = np.array(x0, dtype=np.uint8).reshape(-1)
    assert Cb.shape == (B,) and x.shape == (B,)
    cap = int(steps)
    xin = np.zeros((cap, B), np.uint8)
    xout = np.zeros((cap, B), np.uint8)
    un = np.zeros((cap, B), np.int64)
    v = {nm: np.zeros(cap, np.int64) for nm in ("cst", "lam", "ecur", "ap", "enew")}
    acc = np.zeros(cap, np.int32)
    geo = inst._geo()[:3]
    done = _load().orc_lsa_tr_block_trace(*geo, _p(inst.Wl, _I64P), int(k), _p(Cb, _I64P), _p(x, _U8P),
                                          int(steps), cap, _p(xin, _U8P), _p(xout, _U8P), _p(un, _I64P),
                                          _p(v["cst"], _I64P), _p(v["lam"], _I64P), _p(v["ecur"], _I64P),
                                          _p(v["ap"], _I64P), _p(v["enew"], _I64P),
                                          acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if done < 0:
        raise RuntimeError("orc_lsa_tr_block_trace failed")
    recs = [{"x_in": xin[s].copy(), "x_out": xout[s].copy(), "un": un[s].copy(), "cst": int(v["cst"][s]),
             "lam": int(v["lam"][s]), "ecur": int(v["ecur"][s]), "ap": int(v["ap"][s]),
             "enew": int(v["enew"][s]), "accepted": bool(acc[s])} for s in range(min(done, cap))]
    return recs, x


def lsa_tr_global(inst: Instance, steps=200):
    """Serial LSA-TR on the whole grid from 0: (labels, E_int)."""
    d = _c(inst.dims, np.int64)
    labels = np.empty(inst.n, np.uint8)
    e = _load().orc_lsa_tr_global(_p(d, _I64P), int(inst.conn), _p(inst.U, _I64P), _p(inst.Wl, _I64P),
                                  int(steps), _p(labels, _U8P))
    if e == np.iinfo(np.int64).min:
        raise RuntimeError("orc_lsa_tr_global failed")
    return labels, int(e)
