"""Oracle for the whole-image potentials -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s oracle legs may
import this module; it shares no code with the CUDA package.

Algorithm 1 starts by computing the unary and pairwise potentials of the whole
image; Section 4 notes that this step costs the same for every partition and
takes a large part of the paper's run times.  The potentials follow Section 2:

  * data term (Eq. 1): u_i = log p_bg(x_i) - log p_fg(x_i), the negative
    log-likelihood difference of the two colour models (u_i < 0 favours the
    foreground, Section 2); each model is a Gaussian mixture
    p(x) = sum_j pi_j N(x; m_j, S_j) over the pixel's feature vector (Section 4
    draws its colour models from clusters of seed pixels).  The weights pi_j
    are taken as given (no renormalisation) and the result is clipped to
    [-clip, clip].
  * pairwise term (Eq. 1, the contrast-sensitive Potts weights of Section 2):
    w_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)), optionally divided by the pixel
    distance |p_i - p_j|, for every forward offset of the neighbourhood; sigma
    is given or, by default, the mean of |x_i - x_j| over all neighbour pairs
    (floored at 1e-6); entries whose partner lies outside the grid are 0.

The oracle of the pairwise weights is ``contrast_weights``, the definition in
FP64 (with ``mean_contrast`` for the default sigma); parity tests compare the
GPU's quantised weights with rne(1024 w) of it outside a band around rounding
ties that the FP32 error bound fixes.  ``contrast_weights_q`` and
``sigma_fp32_path`` restate the same quantities with the decision taken in
FP32, one correctly rounded operation at a time; they only illustrate (in the
CPU tests) why FP32 and FP64 decisions differ near ties, and no parity test
uses them as the reference.
The data term is a float output (its quantisation happens later, in FP64, when
it is loaded into a solver), so ``gmm_unaries`` is FP64 throughout.

Pins: tests/test_oracle_potentials.py (closed forms, scipy's multivariate
normal, brute-force loops over every pair, a two-colour step image).
"""
from __future__ import annotations

import math

import numpy as np

from .theorem1 import _OFFS


def gmm_loglik(X, weights, means, covs):
    """log sum_j pi_j N(x; m_j, S_j) for every row x of X [n, C], in FP64.

    N(x; m, S) = (2 pi)^(-C/2) det(S)^(-1/2) exp(-(x-m)^T S^-1 (x-m) / 2); the
    sum over components uses the largest term as the shift (log-sum-exp)."""
    X = np.asarray(X, np.float64)
    n, C = X.shape
    terms = []
    for pi, m, S in zip(weights, means, covs):
        S = np.asarray(S, np.float64)
        d = X - np.asarray(m, np.float64)[None, :]
        Sinv = np.linalg.inv(S)
        sign, logdet = np.linalg.slogdet(S)
        if sign <= 0:
            raise ValueError("covariance is not positive definite")
        quad = np.einsum("ni,ij,nj->n", d, Sinv, d)
        terms.append(math.log(pi) - 0.5 * quad - 0.5 * logdet - 0.5 * C * math.log(2.0 * math.pi))
    T = np.stack(terms, axis=1)
    top = T.max(axis=1)
    return top + np.log(np.exp(T - top[:, None]).sum(axis=1))


def gmm_unaries(image, fg, bg, clip=1.0e5):
    """u_i = clip(log p_bg(x_i) - log p_fg(x_i)) for image [..., C] (or [...]
    for one channel); fg / bg are (weights, means, covs).  Returns (u, ll_fg,
    ll_bg) as flat FP64 arrays."""
    C = len(fg[1][0])
    X = np.asarray(image, np.float64).reshape(-1, C)
    lf = gmm_loglik(X, *fg)
    lb = gmm_loglik(X, *bg)
    return np.clip(lb - lf, -clip, clip), lf, lb


def _as_volume(image, dims):
    """(D, H, W, C) FP view of an image given in pixel-major order."""
    D, H, W = dims
    a = np.asarray(image)
    return a.reshape(D, H, W, -1)


def _pairs(vol, off):
    """(valid mask [D,H,W], neighbour features [D,H,W,C]) for forward offset
    off = (dz, dy, dx): the neighbour of (z, y, x) is (z+dz, y+dy, x+dx)."""
    D, H, W, C = vol.shape
    dz, dy, dx = off
    nb = np.zeros_like(vol)
    valid = np.zeros((D, H, W), bool)
    for z in range(D):
        zz = z + dz
        if not 0 <= zz < D:
            continue
        y0, y1 = max(0, -dy), min(H, H - dy)
        x0, x1 = max(0, -dx), min(W, W - dx)
        if y0 >= y1 or x0 >= x1:
            continue
        nb[z, y0:y1, x0:x1] = vol[zz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        valid[z, y0:y1, x0:x1] = True
    return valid, nb


def mean_contrast(image, dims, conn):
    """Mean of |x_i - x_j| over every neighbour pair (each once), in FP64 from
    the FP64 features; the default sigma before its 1e-6 floor."""
    vol = _as_volume(np.asarray(image, np.float64), dims)
    tot, cnt = 0.0, 0
    for off in _OFFS[conn]:
        valid, nb = _pairs(vol, off)
        d = vol - nb
        tot += float(np.sqrt((d * d).sum(axis=-1))[valid].sum())
        cnt += int(valid.sum())
    return tot / cnt if cnt else 0.0


def contrast_weights(image, dims, conn, sigma=None, inv_dist=False):
    """FP64 definition: w [conn/2, N] and the sigma used."""
    vol = _as_volume(np.asarray(image, np.float64), dims)
    sig = float(sigma) if sigma is not None else max(mean_contrast(image, dims, conn), 1e-6)
    out = []
    for (dz, dy, dx) in _OFFS[conn]:
        valid, nb = _pairs(vol, (dz, dy, dx))
        d = vol - nb
        w = np.exp(-(d * d).sum(axis=-1) / (2.0 * sig * sig))
        if inv_dist:
            w = w / math.sqrt(dz * dz + dy * dy + dx * dx)
        out.append(np.where(valid, w, 0.0).reshape(-1))
    return np.stack(out), sig


def sigma_fp32_path(image, dims, conn):
    """The default sigma as the FP32 path forms it: per pair
    d2 = (((x0-y0)^2 + (x1-y1)^2) + ...) in FP32 and sqrt(d2) in FP32; per
    pixel the sum of its pairs' roots in FP32, in offset order; the pixels'
    sums added in FP64 and divided by the number of pairs; floored at 1e-6."""
    vol = _as_volume(np.asarray(image, np.float32), dims)
    per_pixel = np.zeros(vol.shape[:3], np.float32)
    cnt = 0
    for off in _OFFS[conn]:
        valid, nb = _pairs(vol, off)
        r = np.where(valid, np.sqrt(_d2_fp32(vol, nb)), np.float32(0.0)).astype(np.float32)
        per_pixel = (per_pixel + r).astype(np.float32)
        cnt += int(valid.sum())
    tot = float(per_pixel.astype(np.float64).sum())
    return max(tot / cnt, 1e-6) if cnt else 1e-6


def _d2_fp32(vol, nb):
    d = (vol - nb).astype(np.float32)
    s = d[..., 0] * d[..., 0]
    for c in range(1, vol.shape[-1]):
        s = (s + d[..., c] * d[..., c]).astype(np.float32)
    return s


def contrast_weights_q(image, dims, conn, sigma=None, inv_dist=False):
    """Quantised weights wq = rne(1024 w) [conn/2, N] int32 with the decision
    in FP32: d2 as in ``sigma_fp32_path``; s = sigma (given, else that
    function's); k = fp32(1 / (2 s^2)) formed in FP64; e = exp(-(d2 * k)) in
    FP32; w = e * fp32(1 / |p_i - p_j|) (or e); wq = rne(1024 w).  Returns
    (wq, sigma, margin) where margin = | |1024 w - floor(1024 w)| - 1/2 |, the
    distance of each decision from a rounding tie."""
    vol = _as_volume(np.asarray(image, np.float32), dims)
    sig = float(sigma) if sigma is not None else sigma_fp32_path(image, dims, conn)
    k = np.float32(1.0 / (2.0 * sig * sig))
    out, marg = [], []
    for (dz, dy, dx) in _OFFS[conn]:
        valid, nb = _pairs(vol, (dz, dy, dx))
        d2 = _d2_fp32(vol, nb)
        e = np.exp(-(d2 * k)).astype(np.float32)
        if inv_dist:
            e = (e * np.float32(1.0 / math.sqrt(dz * dz + dy * dy + dx * dx))).astype(np.float32)
        v = (np.float32(1024.0) * e).astype(np.float32)
        q = np.rint(v).astype(np.int32)
        m = np.abs(np.abs(v.astype(np.float64) - np.floor(v.astype(np.float64))) - 0.5)
        out.append(np.where(valid, q, 0).reshape(-1))
        marg.append(np.where(valid, m, 1.0).reshape(-1))
    return np.stack(out).astype(np.int32), sig, np.stack(marg)
