"""Seeded synthetic DOPE instances.

This module only draws images / volumes and turns them into the potentials of
Eq. 1 - 2 (unaries as log-posterior ratios, contrast-sensitive Potts weights).
It holds none of the ADMM arithmetic and imports neither the CUDA library nor
the oracle, so both sides can be fed from it.

Every instance is a dict:
    grid   (H, W) or (D, H, W)
    conn   4 or 8 (2-D), 6 (3-D)
    block  sub-region shape, same rank as grid
    lam    lambda of Eq. 1
    mu0    initial ADMM penalty (100 in 2-D, 500 in 3-D: Section 3 settings)
    u      float32 [N]  unary  u_i = log p(y_i=0|x_i) - log p(y_i=1|x_i)   (Eq. 2)
    wq     int32 [conn/2, N]  rne(1024 w_ij) of the edge from pixel i to its
           forward neighbour along offset k (0 where the neighbour is outside)

Forward offsets (same order everywhere in this project): 2-D (dy, dx):
4-conn (0,+1), (+1,0); 8-conn adds (+1,+1), (+1,-1).  3-D (dz, dy, dx):
(0,0,+1), (0,+1,0), (+1,0,0).

The paper's own images, MRI volume and CNN unaries are not available; these
generators are synthetic stand-ins with the same kinds of structure.
"""
from __future__ import annotations

import numpy as np

FWD_OFFSETS = {
    4: [(0, 0, 1), (0, 1, 0)],
    8: [(0, 0, 1), (0, 1, 0), (0, 1, 1), (0, 1, -1)],
    6: [(0, 0, 1), (0, 1, 0), (1, 0, 0)],
}


def _kernel_offsets(r, is3d):
    """Forward offsets of a square (2-D) or spherical (3-D) kernel of radius r:
    dz = 0..r, dy = -r..r, dx = -r..r, lexicographically positive ones inside
    the kernel, in that order."""
    out = []
    for dz in range(0, (r if is3d else 0) + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if not (dz > 0 or (dz == 0 and dy > 0) or (dz == 0 and dy == 0 and dx > 0)):
                    continue
                if is3d and dz * dz + dy * dy + dx * dx > r * r:
                    continue
                out.append((dz, dy, dx))
    return out


# Section 3's larger kernels: 5x5, 7x7, 9x9 squares (24, 48, 80 neighbours) and
# the radius-2 sphere in 3-D (32 neighbours)
for _r in (2, 3, 4):
    FWD_OFFSETS[(2 * _r + 1) ** 2 - 1] = _kernel_offsets(_r, False)
FWD_OFFSETS[32] = _kernel_offsets(2, True)
KERNEL_CONN = {(2, 3): 8, (2, 5): 24, (2, 7): 48, (2, 9): 80, (3, 3): 6, (3, 5): 32}


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _shifted(vol, dz, dy, dx):
    """(valid mask, neighbour values) for the forward offset on a (D,H,W[,C]) array."""
    D, H, W = vol.shape[:3]
    nb = np.zeros_like(vol)
    valid = np.zeros((D, H, W), bool)
    zs = slice(0, D - dz) if dz >= 0 else slice(-dz, D)
    ys = slice(0, H - dy) if dy >= 0 else slice(-dy, H)
    xs = slice(0, W - dx) if dx >= 0 else slice(-dx, W)
    zt = slice(dz, D) if dz >= 0 else slice(0, D + dz)
    yt = slice(dy, H) if dy >= 0 else slice(0, H + dy)
    xt = slice(dx, W) if dx >= 0 else slice(0, W + dx)
    nb[zs, ys, xs] = vol[zt, yt, xt]
    valid[zs, ys, xs] = True
    return valid, nb


def contrast_weights(vol, conn, sigma=None, fixed_sigma=None, inv_dist=False):
    """Contrast-sensitive Potts weights w_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)) [/ |p_i - p_j|]
    for every forward offset.  vol is (D, H, W) or (D, H, W, C).  sigma defaults
    to the mean feature difference over all neighbour pairs.  Returns float64
    [conn/2, N] and the sigma used."""
    offs = FWD_OFFSETS[conn]
    diffs, valids = [], []
    for (dz, dy, dx) in offs:
        valid, nb = _shifted(vol, dz, dy, dx)
        d = vol - nb
        d2 = (d * d).sum(axis=-1) if vol.ndim == 4 else d * d
        diffs.append(d2)
        valids.append(valid)
    if fixed_sigma is not None:
        sig = float(fixed_sigma)
    elif sigma is None:
        tot = sum(np.sqrt(d2[v]).sum() for d2, v in zip(diffs, valids))
        cnt = sum(int(v.sum()) for v in valids)
        sig = float(tot / max(cnt, 1))
        sig = max(sig, 1e-6)
    else:
        sig = float(sigma)
    out = np.zeros((len(offs),) + vol.shape[:3], np.float64)
    for k, ((dz, dy, dx), d2, v) in enumerate(zip(offs, diffs, valids)):
        w = np.exp(-d2 / (2.0 * sig * sig))
        if inv_dist:
            w = w / np.sqrt(dz * dz + dy * dy + dx * dx)
        out[k] = np.where(v, w, 0.0)
    return out.reshape(len(offs), -1), sig


def quantise_weights(w):
    """wq = rne(1024 w) as int32 (numpy rint rounds half to even)."""
    return np.rint(1024.0 * np.asarray(w, np.float64)).astype(np.int32)


def _gauss_logpdf(x, m, s):
    return -0.5 * ((x - m) / s) ** 2 - np.log(s) - 0.5 * np.log(2 * np.pi)


# --------------------------------------------------------------------------
# 64x64 single-channel disk (4-conn Potts, lambda = 2, 16x16 sub-regions)
# --------------------------------------------------------------------------

def disk64(seed=0, size=64, radius=20.0, lam=2.0, block=(16, 16), sigma=0.1):
    """Two-region disk on background: intensities N(0.7, 0.1) inside, N(0.3, 0.1)
    outside (fp32); u = log N(x; 0.3, 0.1) - log N(x; 0.7, 0.1); 4-connected
    w = exp(-(x_i - x_j)^2 / (2 * 0.1^2))."""
    rng = _rng(seed)
    yy, xx = np.mgrid[0:size, 0:size]
    c = size / 2.0
    inside = (yy - c) ** 2 + (xx - c) ** 2 <= radius * radius
    img = np.where(inside, rng.normal(0.7, 0.1, (size, size)),
                   rng.normal(0.3, 0.1, (size, size))).astype(np.float32)
    x = img.astype(np.float64)
    u = (_gauss_logpdf(x, 0.3, 0.1) - _gauss_logpdf(x, 0.7, 0.1)).astype(np.float32)
    w, _ = contrast_weights(x[None], 4, fixed_sigma=sigma)
    return {"name": f"disk{size}", "grid": (size, size), "conn": 4, "block": tuple(block),
            "lam": float(lam), "mu0": 100.0, "u": u.reshape(-1), "wq": quantise_weights(w),
            "truth": inside.reshape(-1).astype(np.uint8), "image": img}


# --------------------------------------------------------------------------
# 512x512 RGB ellipses, GMM unaries (8-conn contrast Potts, 32x32 sub-regions)
# --------------------------------------------------------------------------

def _kmeanspp(X, k, rng):
    cent = [X[rng.integers(len(X))]]
    for _ in range(1, k):
        d2 = np.min(((X[:, None, :] - np.array(cent)[None]) ** 2).sum(-1), axis=1)
        p = d2 / d2.sum() if d2.sum() > 0 else np.full(len(X), 1.0 / len(X))
        cent.append(X[rng.choice(len(X), p=p)])
    return np.array(cent)


def fit_gmm(X, k, rng, iters=50, reg=1e-4):
    """Full-covariance EM from a k-means++ start; returns (weights, means, covs)."""
    X = np.asarray(X, np.float64)
    n, dim = X.shape
    mu = _kmeanspp(X, k, rng)
    lab = np.argmin(((X[:, None, :] - mu[None]) ** 2).sum(-1), axis=1)
    pi = np.array([max((lab == j).mean(), 1e-3) for j in range(k)])
    pi /= pi.sum()
    cov = np.array([np.cov(X[lab == j].T) + reg * np.eye(dim) if (lab == j).sum() > dim
                    else np.cov(X.T) + reg * np.eye(dim) for j in range(k)])
    for _ in range(iters):
        logr = np.stack([np.log(pi[j]) + _mvn_logpdf(X, mu[j], cov[j]) for j in range(k)], 1)
        m = logr.max(1, keepdims=True)
        r = np.exp(logr - m)
        r /= r.sum(1, keepdims=True)
        nk = r.sum(0) + 1e-12
        pi = nk / n
        mu = (r.T @ X) / nk[:, None]
        for j in range(k):
            d = X - mu[j]
            cov[j] = (r[:, j, None] * d).T @ d / nk[j] + reg * np.eye(dim)
    return pi, mu, cov


def _mvn_logpdf(X, m, C):
    dim = X.shape[1]
    L = np.linalg.cholesky(C)
    z = np.linalg.solve(L, (X - m).T)
    return -0.5 * (z * z).sum(0) - np.log(np.diag(L)).sum() - 0.5 * dim * np.log(2 * np.pi)


def gmm_loglik(X, gmm):
    pi, mu, cov = gmm
    logs = np.stack([np.log(pi[j]) + _mvn_logpdf(X, mu[j], cov[j]) for j in range(len(pi))], 1)
    m = logs.max(1, keepdims=True)
    return (m[:, 0] + np.log(np.exp(logs - m).sum(1)))


def ellipses_rgb(seed=0, size=512, lam=4.0, block=(32, 32), conn=8, n_ellipses=12,
                 noise=0.08, box=24):
    """12 random ellipses (centres U[0,size)^2, semi-axes U[16,128], angle U[0,pi),
    colours U[0,1]^3) painted in order over a U[0,1]^3 background, plus N(0, 0.08^2)
    noise; two 3-component GMMs fit on a 24x24 foreground box (centre of the largest
    ellipse) and a 24x24 background box (a corner away from the ellipses);
    u = log p_bg(x) - log p_fg(x); contrast weights with sigma = mean colour
    difference over neighbour pairs, divided by the pixel distance."""
    rng = _rng(seed)
    H = W = size
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.empty((H, W, 3), np.float64)
    img[:] = rng.uniform(0, 1, 3)
    masks, areas, centres = [], [], []
    scale = size / 512.0
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(16, 128) * scale, rng.uniform(16, 128) * scale
        th = rng.uniform(0, np.pi)
        col = rng.uniform(0, 1, 3)
        dy, dx = yy - cy, xx - cx
        xr = dx * np.cos(th) + dy * np.sin(th)
        yr = -dx * np.sin(th) + dy * np.cos(th)
        m = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
        img[m] = col
        masks.append(m); areas.append(np.pi * a * b); centres.append((cy, cx))
    img = img + rng.normal(0, noise, img.shape)
    img32 = img.astype(np.float32)
    X = img32.reshape(-1, 3).astype(np.float64)
    anym = np.zeros((H, W), bool)
    for m in masks:
        anym |= m
    big = int(np.argmax(areas))
    cy, cx = centres[big]
    fy = int(np.clip(round(cy) - box // 2, 0, H - box))
    fx = int(np.clip(round(cx) - box // 2, 0, W - box))
    corners = [(0, 0), (0, W - box), (H - box, 0), (H - box, W - box)]
    cover = [anym[y:y + box, x:x + box].sum() for (y, x) in corners]
    by, bx = corners[int(np.argmin(cover))]
    fg = img32[fy:fy + box, fx:fx + box].reshape(-1, 3).astype(np.float64)
    bg = img32[by:by + box, bx:bx + box].reshape(-1, 3).astype(np.float64)
    g_fg = fit_gmm(fg, 3, rng)
    g_bg = fit_gmm(bg, 3, rng)
    u = (gmm_loglik(X, g_bg) - gmm_loglik(X, g_fg))
    u = np.clip(u, -1.0e5, 1.0e5).astype(np.float32)
    w, sig = contrast_weights(img32.astype(np.float64)[None], conn, inv_dist=True)
    return {"name": f"ellipses{size}", "grid": (H, W), "conn": conn, "block": tuple(block),
            "lam": float(lam), "mu0": 100.0, "u": u, "wq": quantise_weights(w),
            "sigma": sig, "image": img32, "gmm_fg": g_fg, "gmm_bg": g_bg, "inv_dist": True}


# --------------------------------------------------------------------------
# 256x256x128 volume, nested ellipsoids (6-conn, 16x16x8 sub-regions)
# --------------------------------------------------------------------------

def ellipsoids3d(seed=0, shape=(128, 256, 256), lam=3.0, block=(8, 16, 16), noise=0.05):
    """3 nested random ellipsoids (levels 0.2 background, 0.45, 0.7, 0.9), smooth
    multiplicative bias 1 + 0.2 * (random 2nd-order polynomial), Rician-like noise
    sqrt((v + n1)^2 + n2^2) with n ~ N(0, 0.05^2).  Foreground = inside the middle
    ellipsoid; u = log-ratio of Gaussians fit to the two classes; 6-connected
    contrast weights, sigma = mean |dx| over neighbour pairs."""
    rng = _rng(seed)
    D, H, W = shape
    z, y, x = np.meshgrid(np.linspace(-1, 1, D), np.linspace(-1, 1, H), np.linspace(-1, 1, W),
                          indexing="ij")
    vol = np.full(shape, 0.2)
    c0 = rng.uniform(-0.15, 0.15, 3)
    ax0 = rng.uniform(0.6, 0.85, 3)
    levels = [0.45, 0.7, 0.9]
    fg = None
    for lvl, f in zip(levels, [1.0, 0.7, 0.4]):
        c = c0 + rng.uniform(-0.05, 0.05, 3) * f
        ax = ax0 * f * rng.uniform(0.9, 1.0, 3)
        m = ((z - c[0]) / ax[0]) ** 2 + ((y - c[1]) / ax[1]) ** 2 + ((x - c[2]) / ax[2]) ** 2 <= 1
        vol[m] = lvl
        if lvl == 0.7:
            fg = m
    coef = rng.normal(0, 1, 10)
    terms = [np.ones_like(z), z, y, x, z * z, y * y, x * x, z * y, z * x, y * x]
    poly = sum(cf * t for cf, t in zip(coef, terms))
    poly = poly / max(np.abs(poly).max(), 1e-9)
    vol = vol * (1.0 + 0.2 * poly)
    n1 = rng.normal(0, noise, shape)
    n2 = rng.normal(0, noise, shape)
    vol = np.sqrt((vol + n1) ** 2 + n2 ** 2).astype(np.float32)
    v64 = vol.astype(np.float64)
    m1, s1 = v64[fg].mean(), v64[fg].std() + 1e-6
    m0, s0 = v64[~fg].mean(), v64[~fg].std() + 1e-6
    u = (_gauss_logpdf(v64, m0, s0) - _gauss_logpdf(v64, m1, s1)).astype(np.float32)
    w, sig = contrast_weights(v64, 6)
    return {"name": "ellipsoids%dx%dx%d" % (W, H, D), "grid": tuple(shape), "conn": 6,
            "block": tuple(block), "lam": float(lam), "mu0": 500.0, "u": u.reshape(-1),
            "wq": quantise_weights(w), "sigma": sig, "truth": fg.reshape(-1).astype(np.uint8),
            "image": vol.reshape(-1), "inv_dist": False,
            # the two classes' Gaussians as one-component, one-channel mixtures
            "gmm_fg": (np.array([1.0]), np.array([[m1]]), np.array([[[s1 * s1]]])),
            "gmm_bg": (np.array([1.0]), np.array([[m0]]), np.array([[[s0 * s0]]]))}


def crop_instance(d, lo, shape):
    """The sub-grid of instance d starting at `lo` with extent `shape` (same
    connectivity, block shape, lambda, mu0): unaries cropped, weights cropped
    with every n-link that leaves the crop set to 0."""
    grid = tuple(d["grid"])
    nd = len(grid)
    assert nd == len(lo) == len(shape)
    sl = tuple(slice(a, a + n) for a, n in zip(lo, shape))
    u = np.ascontiguousarray(d["u"].reshape(grid)[sl]).reshape(-1)
    nh = d["conn"] // 2
    w = np.array(d["wq"].reshape((nh,) + grid)[(slice(None),) + sl])
    offs = FWD_OFFSETS[d["conn"]]
    sh3 = (1,) * (3 - nd) + tuple(shape)
    w3 = w.reshape((nh,) + sh3)
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in sh3], indexing="ij")
    for k, (dz, dy, dx) in enumerate(offs):
        z2, y2, x2 = zz + dz, yy + dy, xx + dx
        out = (z2 < 0) | (z2 >= sh3[0]) | (y2 < 0) | (y2 >= sh3[1]) | (x2 < 0) | (x2 >= sh3[2])
        w3[k][out] = 0
    r = dict(d, grid=tuple(shape), u=u, wq=np.ascontiguousarray(w3.reshape(nh, -1)))
    n = int(np.prod(grid))
    for key in ("image", "truth"):
        if key in d:
            a = np.asarray(d[key])
            extra = a.size // n
            b = a.reshape(grid + ((extra,) if extra > 1 else ()))[sl]
            if a.ndim == 1:
                b = b.reshape(-1)
            elif a.ndim == 2:
                b = b.reshape(-1, extra)
            r[key] = np.ascontiguousarray(b)
    return r


# --------------------------------------------------------------------------
# Small random instances for tests
# --------------------------------------------------------------------------

def random_instance(grid, conn, block, lam=1.0, seed=0, u_scale=4.0, w_max=1.0, mu0=None,
                    smooth=True, w_int_max=None):
    """A random instance: a smooth random field plus noise for u (so that
    labels form regions and blocks have boundaries), uniform random weights.
    If w_int_max is given, weights are integers in [0, w_int_max] (x1024 not
    applied) -- useful for exact hand checks."""
    rng = _rng(seed)
    grid = tuple(int(g) for g in grid)
    dims = grid if len(grid) == 3 else (1,) + grid
    n = int(np.prod(dims))
    if smooth:
        f = rng.normal(0, 1, dims)
        for ax in range(3):
            if dims[ax] > 2:
                f = (f + np.roll(f, 1, ax) + np.roll(f, -1, ax)) / 3.0
        f = f / (f.std() + 1e-9)
        u = u_scale * f + rng.normal(0, u_scale * 0.5, dims)
    else:
        u = rng.normal(0, u_scale, dims)
    vol = np.zeros(dims)
    offs = FWD_OFFSETS[conn]
    wq = np.zeros((len(offs), n), np.int32)
    for k, (dz, dy, dx) in enumerate(offs):
        valid, _ = _shifted(vol, dz, dy, dx)
        if w_int_max is not None:
            w = rng.integers(0, w_int_max + 1, dims)
            wq[k] = np.where(valid, w, 0).reshape(-1).astype(np.int32)
        else:
            w = rng.uniform(0, w_max, dims)
            wq[k] = np.where(valid, np.rint(1024.0 * w), 0).reshape(-1).astype(np.int32)
    if mu0 is None:
        mu0 = 500.0 if len(grid) == 3 else 100.0
    return {"name": "random", "grid": grid, "conn": conn, "block": tuple(block), "lam": float(lam),
            "mu0": float(mu0), "u": u.reshape(-1).astype(np.float32), "wq": wq}


CONFIGS = {
    "disk64": disk64,
    "ellipses512": ellipses_rgb,
    "ellipsoids256": ellipsoids3d,
}


def pad_to_blocks(d):
    """Copy of instance d with its grid rounded up to whole blocks: the extra
    pixels get unary 0 and no n-links (isolated zero-cost pixels), which is the
    padding the request server applies to ragged grids."""
    grid = tuple(int(g) for g in d["grid"])
    block = tuple(int(b) for b in d["block"])
    pg = tuple(-(-g // b) * b for g, b in zip(grid, block))
    if pg == grid:
        return dict(d)
    nh = len(FWD_OFFSETS[d["conn"]])
    u = np.zeros(pg, np.float32)
    u[tuple(slice(0, g) for g in grid)] = np.asarray(d["u"], np.float32).reshape(grid)
    wq = np.zeros((nh,) + pg, np.int32)
    wq[(slice(None),) + tuple(slice(0, g) for g in grid)] = np.asarray(d["wq"], np.int32).reshape((nh,) + grid)
    out = dict(d)
    out.update(grid=pg, u=u.reshape(-1), wq=wq.reshape(nh, -1), unpadded_grid=grid)
    return out


def crop_padded(labels, d_padded):
    """The caller's pixels of labels computed on pad_to_blocks(d)."""
    grid = d_padded.get("unpadded_grid", d_padded["grid"])
    full = np.asarray(labels).reshape(d_padded["grid"])
    return full[tuple(slice(0, g) for g in grid)].reshape(-1)


# --------------------------------------------------------------------------
# Serving stream: Poisson arrivals of RGB contrast-Potts segmentations of
# random side in [128, 2048], 4- or 8-connected, lambda in [1, 16]
# --------------------------------------------------------------------------

def serving_base(seed=0, size=2048, noise=0.08, box=24):
    """A size x size RGB image with the statistics of ellipses_rgb: 12 ellipses
    per 512x512 of area (centres uniform, semi-axes U[16,128], angle U[0,pi),
    colours U[0,1]^3) over a U[0,1]^3 background, N(0, 0.08^2) noise; 3-component
    GMMs fit on a 24x24 box inside the largest ellipse and on the 24x24 box (of
    64 seeded candidates) least covered by ellipses; unaries and 8-connected
    contrast weights (sigma = mean colour difference, divided by the pixel
    distance) over the whole image.  Requests are crops of it."""
    rng = _rng(1000 + seed)
    H = W = size
    n_ell = 12 * max(1, (size * size) // (512 * 512))
    img = np.empty((H, W, 3), np.float32)
    img[:] = rng.uniform(0, 1, 3)
    anym = np.zeros((H, W), bool)
    areas, centres = [], []
    for _ in range(n_ell):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(16, 128), rng.uniform(16, 128)
        th = rng.uniform(0, np.pi)
        col = rng.uniform(0, 1, 3).astype(np.float32)
        r = max(a, b)
        y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        dy, dx = yy - cy, xx - cx
        xr = dx * np.cos(th) + dy * np.sin(th)
        yr = -dx * np.sin(th) + dy * np.cos(th)
        m = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
        img[y0:y1, x0:x1][m] = col
        anym[y0:y1, x0:x1] |= m
        areas.append(np.pi * a * b)
        centres.append((cy, cx))
    img += rng.normal(0, noise, img.shape).astype(np.float32)
    cy, cx = centres[int(np.argmax(areas))]
    fy = int(np.clip(round(cy) - box // 2, 0, H - box))
    fx = int(np.clip(round(cx) - box // 2, 0, W - box))
    cand = rng.integers(0, H - box, (64, 2))
    cover = [anym[y:y + box, x:x + box].sum() for (y, x) in cand]
    by, bx = (int(v) for v in cand[int(np.argmin(cover))])
    g_fg = fit_gmm(img[fy:fy + box, fx:fx + box].reshape(-1, 3).astype(np.float64), 3, rng)
    g_bg = fit_gmm(img[by:by + box, bx:bx + box].reshape(-1, 3).astype(np.float64), 3, rng)
    X = img.reshape(-1, 3).astype(np.float64)
    u = np.clip(gmm_loglik(X, g_bg) - gmm_loglik(X, g_fg), -1.0e5, 1.0e5).astype(np.float32)
    del X
    w, sig = contrast_weights(img.astype(np.float64)[None], 8, inv_dist=True)
    return {"size": size, "u": u.reshape(H, W), "wq": quantise_weights(w).reshape(4, H, W), "sigma": sig,
            "image": img, "gmm_fg": g_fg, "gmm_bg": g_bg}


def serving_requests(n=1000, rate=200.0, seed=0, side=(128, 2048), n_bases=2, base_size=2048,
                     block=(32, 32), lam=(1.0, 16.0)):
    """The request stream: Poisson arrivals (exponential gaps of mean 1/rate),
    side uniform in [side0, side1], 4- or 8-connectivity 50/50, lambda uniform
    in [lam0, lam1], a base image and a uniform crop position."""
    rng = _rng(2000 + seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t -= t[0]
    out = []
    for i in range(n):
        s = int(rng.integers(side[0], side[1] + 1))
        conn = 4 if rng.random() < 0.5 else 8
        out.append({"arrival": float(t[i]), "base": int(rng.integers(n_bases)), "side": s,
                    "y0": int(rng.integers(0, base_size - s + 1)), "x0": int(rng.integers(0, base_size - s + 1)),
                    "conn": conn, "lam": float(rng.uniform(lam[0], lam[1])), "block": tuple(block),
                    "grid": (s, s), "mu0": 100.0})
    return out


def crop_request(base, req):
    """(u [s*s] float32, wq [conn/2, s*s] int32) of a request: the crop of the
    base image's potentials, with the n-links that leave the crop set to 0."""
    s, y0, x0 = req["side"], req["y0"], req["x0"]
    nh = req["conn"] // 2
    u = np.ascontiguousarray(base["u"][y0:y0 + s, x0:x0 + s]).reshape(-1)
    w = np.array(base["wq"][:nh, y0:y0 + s, x0:x0 + s])
    w[0, :, -1] = 0
    w[1, -1, :] = 0
    if nh == 4:
        w[2, -1, :] = 0
        w[2, :, -1] = 0
        w[3, -1, :] = 0
        w[3, :, 0] = 0
    return u, w.reshape(nh, -1)


def nonsubmodular_instance(seed=0, size=1024, block=(16, 16), lam=1.0, neg_frac=0.2, u_sd=2.0):
    """A 4-connected grid with non-submodular pairwise terms: unaries N(0, 2^2);
    |w_ij| ~ |N(0, 1)|, and a random neg_frac of the edges negative (for
    w |y_i - y_j| that is f(1,0) + f(0,1) < f(0,0) + f(1,1), the footnote's
    non-submodular case); wq = rne(1024 w), 0 toward the outside."""
    rng = _rng(3000 + seed)
    H = W = size
    u = rng.normal(0.0, u_sd, (H, W)).astype(np.float32)
    wq = np.zeros((2, H * W), np.int32)
    vol = np.zeros((1, H, W))
    for k, (dz, dy, dx) in enumerate(FWD_OFFSETS[4]):
        valid, _ = _shifted(vol, dz, dy, dx)
        mag = np.abs(rng.normal(0.0, 1.0, (1, H, W)))
        sign = np.where(rng.random((1, H, W)) < neg_frac, -1.0, 1.0)
        wq[k] = np.where(valid, np.rint(1024.0 * mag * sign), 0).reshape(-1).astype(np.int32)
    return {"name": f"nonsubmodular{size}", "grid": (H, W), "conn": 4, "block": tuple(block),
            "lam": float(lam), "mu0": 100.0, "u": u.reshape(-1), "wq": wq}


def signed_instance(d, neg_frac=0.2, seed=0):
    """Copy of instance d with a random neg_frac of its edges made negative
    (non-submodular pairwise terms)."""
    rng = _rng(4000 + seed)
    wq = np.array(d["wq"], np.int32)
    flip = rng.random(wq.shape) < neg_frac
    out = dict(d)
    out["wq"] = np.where(flip, -wq, wq).astype(np.int32)
    out["name"] = d.get("name", "instance") + "_signed"
    return out
