"""Literal matrix form of DOPE's block decomposition -- TEST INFRASTRUCTURE ONLY.

Dense numpy, small grids only (N up to a few hundred).  Every quantity is
built exactly as Section 2 of Dolz, Ben Ayed, Desrosiers (arXiv 1704.03116)
defines it, for any partition, overlapping or not:

  * S_k        selection matrix of block k (|Omega_k| x |Omega|)
  * Q          = sum_k S_k^T S_k, diagonal, q_ii = number of blocks holding i
               (Proposition 1, Eq. 4)
  * L = D - W  Laplacian of the pairwise matrix (Eq. 3)
  * u_hat_k    = S_k Q^-1 u                                   (Theorem 1)
  * W_hat_k    = S_k Q^-1 W Q^-1 S_k^T, D_hat_k, L_hat_k = D_hat_k - W_hat_k
  * C_k        = S_k Q^-1 L (I - Q^-1 S_k^T S_k)
  * R_k        = S_k Q^-1 D Q^-1 S_k^T - D_hat_k
  * Eq. 5      the reformulated objective
  * Eq. 8      block unary  u_hat_k + lam (C_k + R_k S_k) y + mu (a_k - S_k y + 1/2)
  * Eq. 10     y = (1/mu) Q^-1 sum_k ( mu S_k^T (yhat_k + a_k) - lam (C_k + R_k S_k)^T yhat_k )
  * Eq. 11     a_k = a_k + yhat_k - S_k y

Nothing here is shared with, or imported by, the CUDA library.
"""
from __future__ import annotations

import numpy as np

_OFFS = {4: [(0, 0, 1), (0, 1, 0)],
         8: [(0, 0, 1), (0, 1, 0), (0, 1, 1), (0, 1, -1)],
         6: [(0, 0, 1), (0, 1, 0), (1, 0, 0)]}
# larger kernels: every nonzero offset of the square (2-D) or ball (3-D) of
# radius r with a positive first nonzero coordinate, ordered by (dz, dy, dx)
for _r, _c3 in ((2, False), (3, False), (4, False), (2, True)):
    _l = sorted((dz, dy, dx) for dz in range(0, (_r if _c3 else 0) + 1)
                for dy in range(-_r, _r + 1) for dx in range(-_r, _r + 1)
                if (dz, dy, dx) > (0, 0, 0) and (not _c3 or dz * dz + dy * dy + dx * dx <= _r * _r))
    _OFFS[len(_l) * 2] = _l


def grid_pairwise(dims, conn, w_fwd):
    """Dense symmetric W (N x N) from per-pixel forward-edge weights
    w_fwd [conn/2, N] on a (D, H, W) grid (Eq. 1's w_ij on N(i))."""
    D, H, Wd = dims
    n = D * H * Wd
    Wm = np.zeros((n, n), np.float64)
    for k, (dz, dy, dx) in enumerate(_OFFS[conn]):
        for z in range(D):
            for y in range(H):
                for x in range(Wd):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < D and 0 <= yy < H and 0 <= xx < Wd:
                        i = (z * H + y) * Wd + x
                        j = (zz * H + yy) * Wd + xx
                        Wm[i, j] = Wm[j, i] = w_fwd[k, i]
    return Wm


def grid_blocks(dims, block, grow=(0, 0, 0)):
    """Pixel index sets Omega_k of a regular partition into `block`-shaped
    tiles, each grown by `grow` pixels on every side (clipped to the grid);
    grow = 0 gives the non-overlapping partition (Q = I)."""
    D, H, Wd = dims
    bd, bh, bw = block
    gd, gh, gw = grow
    blocks = []
    for kz in range(D // bd):
        for ky in range(H // bh):
            for kx in range(Wd // bw):
                zs = range(max(0, kz * bd - gd), min(D, (kz + 1) * bd + gd))
                ys = range(max(0, ky * bh - gh), min(H, (ky + 1) * bh + gh))
                xs = range(max(0, kx * bw - gw), min(Wd, (kx + 1) * bw + gw))
                blocks.append(np.array([(z * H + y) * Wd + x for z in zs for y in ys for x in xs],
                                       np.int64))
    return blocks


class Decomposition:
    """The matrices of Theorem 1 for one partition."""

    def __init__(self, u, Wm, blocks):
        n = len(u)
        self.n = n
        self.u = np.asarray(u, np.float64)
        self.W = np.asarray(Wm, np.float64)
        self.D = np.diag(self.W.sum(axis=1))
        self.L = self.D - self.W
        self.S = []
        for b in blocks:
            S = np.zeros((len(b), n))
            S[np.arange(len(b)), b] = 1.0
            self.S.append(S)
        self.Q = sum(S.T @ S for S in self.S)
        if np.any(np.diag(self.Q) == 0):
            raise ValueError("blocks do not cover the domain (Proposition 1 needs a cover)")
        self.Qi = np.diag(1.0 / np.diag(self.Q))
        I = np.eye(n)
        self.uh, self.Wh, self.Dh, self.Lh, self.C, self.R = [], [], [], [], [], []
        for S in self.S:
            uh = S @ self.Qi @ self.u
            Wh = S @ self.Qi @ self.W @ self.Qi @ S.T
            Dh = np.diag(Wh.sum(axis=1))
            Lh = Dh - Wh
            C = S @ self.Qi @ self.L @ (I - self.Qi @ S.T @ S)
            R = S @ self.Qi @ self.D @ self.Qi @ S.T - Dh
            self.uh.append(uh); self.Wh.append(Wh); self.Dh.append(Dh)
            self.Lh.append(Lh); self.C.append(C); self.R.append(R)

    @property
    def K(self):
        return len(self.S)

    def energy_eq3(self, lam, y):
        """u^T y + lam y^T L y."""
        y = np.asarray(y, np.float64)
        return float(self.u @ y + lam * y @ self.L @ y)

    def objective_eq5(self, lam, y, yhats):
        y = np.asarray(y, np.float64)
        tot = 0.0
        for k in range(self.K):
            lin = self.uh[k] + lam * (self.C[k] + self.R[k] @ self.S[k]) @ y
            tot += float(lin @ yhats[k] + lam * yhats[k] @ self.Lh[k] @ yhats[k])
        return tot

    def prop1(self, yhats):
        """Q^-1 sum_k S_k^T yhat_k  (Eq. 4)."""
        return self.Qi @ sum(self.S[k].T @ yhats[k] for k in range(self.K))

    def block_unary_eq8(self, k, lam, mu, y, a_k):
        y = np.asarray(y, np.float64)
        return (self.uh[k] + lam * (self.C[k] + self.R[k] @ self.S[k]) @ y
                + mu * (a_k - self.S[k] @ y + 0.5))

    def block_energy_eq8(self, k, lam, mu, y, a_k, yh):
        """The Eq. 8 objective for a candidate block labelling yh."""
        c = self.block_unary_eq8(k, lam, mu, y, a_k)
        yh = np.asarray(yh, np.float64)
        return float(c @ yh + lam * yh @ self.Lh[k] @ yh)

    def update_y_eq10(self, lam, mu, yhats, a_list):
        acc = np.zeros(self.n)
        for k in range(self.K):
            acc += mu * self.S[k].T @ (yhats[k] + a_list[k])
            acc -= lam * (self.C[k] + self.R[k] @ self.S[k]).T @ yhats[k]
        return (1.0 / mu) * self.Qi @ acc

    def update_a_eq11(self, yhats, y, a_list):
        return [a_list[k] + yhats[k] - self.S[k] @ y for k in range(self.K)]

    def residuals(self, yhats, y):
        """||yhat_k - S_k y||_2 for every block (the stop test of Algorithm 1)."""
        return np.array([np.linalg.norm(yhats[k] - self.S[k] @ y) for k in range(self.K)])
