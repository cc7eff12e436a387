"""Pins of the potentials oracle (oracle/potentials.py) against closed forms,
scipy's multivariate normal, brute-force loops over every neighbour pair and
images whose weights follow by hand.  CPU only."""
import math

import numpy as np
import pytest

from oracle import potentials as P
from paper_1704_03116_gb300 import inputs


def _spd(rng, C, scale=0.05):
    A = rng.normal(0, scale, (C, C))
    return A @ A.T + scale * scale * np.eye(C)


def _gmm(rng, K, C):
    w = rng.uniform(0.2, 1.0, K)
    w /= w.sum()
    return w, rng.uniform(0, 1, (K, C)), np.stack([_spd(rng, C) for _ in range(K)])


def test_single_component_identity_closed_form():
    rng = np.random.default_rng(1)
    for C in (1, 2, 3, 4):
        X = rng.normal(0, 2, (50, C))
        m = rng.normal(0, 1, C)
        ll = P.gmm_loglik(X, [1.0], [m], [np.eye(C)])
        ref = -0.5 * ((X - m) ** 2).sum(1) - 0.5 * C * math.log(2 * math.pi)
        np.testing.assert_allclose(ll, ref, rtol=0, atol=1e-12)


def test_univariate_gaussian_closed_form():
    x = np.linspace(-3, 3, 41)
    m, s = 0.4, 0.7
    ll = P.gmm_loglik(x[:, None], [1.0], [[m]], [[[s * s]]])
    ref = -0.5 * ((x - m) / s) ** 2 - math.log(s) - 0.5 * math.log(2 * math.pi)
    np.testing.assert_allclose(ll, ref, rtol=0, atol=1e-12)


def test_mixture_matches_scipy_density_sum():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(2)
    for K, C in ((3, 3), (5, 3), (2, 1), (8, 4)):
        w, mu, cov = _gmm(rng, K, C)
        X = mu[rng.integers(K, size=200)] + rng.normal(0, 0.05, (200, C))
        dens = sum(w[j] * stats.multivariate_normal(mu[j], cov[j]).pdf(X) for j in range(K))
        np.testing.assert_allclose(P.gmm_loglik(X, w, mu, cov), np.log(dens), rtol=1e-10, atol=1e-10)


def test_duplicate_components_merge():
    rng = np.random.default_rng(3)
    m, S = rng.uniform(0, 1, 3), _spd(rng, 3)
    X = rng.uniform(0, 1, (100, 3))
    a = P.gmm_loglik(X, [0.3, 0.7], [m, m], [S, S])
    b = P.gmm_loglik(X, [1.0], [m], [S])
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_far_points_no_underflow():
    # every density underflows in FP64 at this distance; the shifted sum does not
    X = np.array([[50.0, 50.0, 50.0]])
    ll = P.gmm_loglik(X, [0.5, 0.5], [[0, 0, 0], [1, 1, 1]], [1e-3 * np.eye(3)] * 2)
    assert np.isfinite(ll).all() and ll[0] < -1e6


def test_unaries_antisymmetric_clipped_and_signed():
    rng = np.random.default_rng(4)
    fg, bg = _gmm(rng, 3, 3), _gmm(rng, 2, 3)
    img = rng.uniform(0, 1, (7, 9, 3))
    u, lf, lb = P.gmm_unaries(img, fg, bg, clip=1e9)
    u2, _, _ = P.gmm_unaries(img, bg, fg, clip=1e9)
    np.testing.assert_array_equal(u, -u2)
    np.testing.assert_allclose(u, lb - lf, rtol=0, atol=0)
    uc, _, _ = P.gmm_unaries(img, fg, bg, clip=1.5)
    assert np.abs(uc).max() <= 1.5
    # a pixel at the foreground mean of a tight foreground model favours the
    # foreground: u < 0 (Section 2's sign convention)
    fg1 = ([1.0], [[0.2, 0.4, 0.6]], [1e-3 * np.eye(3)])
    bg1 = ([1.0], [[0.8, 0.1, 0.1]], [1e-3 * np.eye(3)])
    u3, _, _ = P.gmm_unaries(np.array([[0.2, 0.4, 0.6]]), fg1, bg1)
    assert u3[0] < 0


def test_empty_image():
    fg = ([1.0], [[0.0]], [[[1.0]]])
    u, lf, lb = P.gmm_unaries(np.zeros((0,)), fg, fg)
    assert u.shape == (0,)


def _brute_weights(img, dims, radius, is3d, norm, sigma, inv_dist):
    """Every unordered neighbour pair by a loop over all offsets within
    `radius` in the given norm (1: the 4- / 6-neighbour cross, 2: the ball,
    'inf': the square); returns {(i, j): w} with i < j and the mean contrast."""
    D, H, W = dims
    vol = np.asarray(img, np.float64).reshape(D, H, W, -1)
    pairs = {}
    for z in range(D):
        for y in range(H):
            for x in range(W):
                for dz in range(-radius if is3d else 0, (radius if is3d else 0) + 1):
                    for dy in range(-radius, radius + 1):
                        for dx in range(-radius, radius + 1):
                            if (dz, dy, dx) == (0, 0, 0):
                                continue
                            if norm == 1 and abs(dz) + abs(dy) + abs(dx) > radius:
                                continue
                            if norm == 2 and dz * dz + dy * dy + dx * dx > radius * radius:
                                continue
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if not (0 <= zz < D and 0 <= yy < H and 0 <= xx < W):
                                continue
                            i, j = (z * H + y) * W + x, (zz * H + yy) * W + xx
                            if i < j:
                                diff = vol[z, y, x] - vol[zz, yy, xx]
                                pairs[(i, j)] = (float(diff @ diff), math.sqrt(dz * dz + dy * dy + dx * dx))
    mean = sum(math.sqrt(d2) for d2, _ in pairs.values()) / len(pairs)
    s = sigma if sigma is not None else max(mean, 1e-6)
    out = {k: math.exp(-d2 / (2 * s * s)) / (dist if inv_dist else 1.0) for k, (d2, dist) in pairs.items()}
    return out, mean


@pytest.mark.parametrize("conn,dims,radius,is3d,norm", [
    (4, (1, 5, 6), 1, False, 1), (8, (1, 5, 6), 1, False, "inf"), (24, (1, 6, 7), 2, False, "inf"),
    (48, (1, 8, 8), 3, False, "inf"), (6, (3, 4, 5), 1, True, 1), (32, (4, 5, 5), 2, True, 2)])
@pytest.mark.parametrize("inv_dist", [False, True])
def test_contrast_weights_brute_force(conn, dims, radius, is3d, norm, inv_dist):
    rng = np.random.default_rng(conn)
    n = int(np.prod(dims))
    img = rng.uniform(0, 1, (n, 3))
    ref, mean = _brute_weights(img, dims, radius, is3d, norm, None, inv_dist)
    w, sig = P.contrast_weights(img, dims, conn, inv_dist=inv_dist)
    assert sig == pytest.approx(mean, rel=1e-13)
    D, H, W = dims
    got = {}
    from oracle.theorem1 import _OFFS
    for k, (dz, dy, dx) in enumerate(_OFFS[conn]):
        for i in range(n):
            z, y, x = i // (H * W), (i // W) % H, i % W
            zz, yy, xx = z + dz, y + dy, x + dx
            if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W:
                j = (zz * H + yy) * W + xx
                got[(min(i, j), max(i, j))] = w[k, i]
            else:
                assert w[k, i] == 0.0
    assert set(got) == set(ref)          # every pair exactly once, no other
    for key, v in ref.items():
        assert got[key] == pytest.approx(v, rel=1e-13)


def test_constant_image_weights():
    img = np.full((6 * 7, 3), 0.3)
    w, sig = P.contrast_weights(img, (1, 6, 7), 8, inv_dist=True)
    assert sig == 1e-6                  # no contrast: the floor
    valid = w > 0
    np.testing.assert_allclose(w[0][valid[0]], 1.0)
    np.testing.assert_allclose(w[2][valid[2]], 1.0 / math.sqrt(2.0))
    wq, _, _ = P.contrast_weights_q(img, (1, 6, 7), 8, inv_dist=True)
    assert set(np.unique(wq[0])) == {0, 1024} and set(np.unique(wq[2])) == {0, 724}
    assert (wq[0].reshape(6, 7)[:, -1] == 0).all() and (wq[1].reshape(6, 7)[-1] == 0).all()


def test_step_image_closed_form():
    # left half colour a, right half colour b: 4-connected pairs crossing the
    # step have |dx| = |a - b|, all others 0; sigma = H |a-b| / #pairs
    H, W = 4, 6
    a, b = np.array([0.1, 0.2, 0.3]), np.array([0.5, 0.2, 0.0])
    img = np.broadcast_to(np.where((np.arange(W) < 3)[None, :, None], a, b), (H, W, 3)).reshape(-1, 3)
    gap = float(np.linalg.norm(a - b))
    npairs = H * (W - 1) + (H - 1) * W
    w, sig = P.contrast_weights(img, (1, H, W), 4)
    assert sig == pytest.approx(H * gap / npairs, rel=1e-14)
    cross = w[0].reshape(H, W)[:, 2]
    np.testing.assert_allclose(cross, math.exp(-gap * gap / (2 * sig * sig)), rtol=1e-14)
    others = np.delete(w[0].reshape(H, W)[:, :-1], 2, axis=1)
    np.testing.assert_allclose(others, 1.0)
    np.testing.assert_allclose(w[1].reshape(H, W)[:-1], 1.0)


def test_fp32_decision_within_one_of_fp64_definition():
    d = inputs.ellipses_rgb(size=128)
    dims = (1, 128, 128)
    w64, s64 = P.contrast_weights(d["image"], dims, 8, inv_dist=True)
    wq32, s32, margin = P.contrast_weights_q(d["image"], dims, 8, inv_dist=True)
    assert s32 == pytest.approx(s64, rel=1e-6)
    ref = np.rint(1024.0 * w64).astype(np.int32)
    diff = np.abs(wq32.astype(np.int64) - ref)
    assert diff.max() <= 1
    # they differ only where the decision sits on a rounding tie
    assert (diff[margin > 1e-3] == 0).all()


def test_generators_agree_with_oracle():
    # the input generators compute the same potentials with a Cholesky-based
    # density and their own pair loop; the oracle uses the inverse/determinant
    d = inputs.ellipses_rgb(size=128)
    u, lf, lb = P.gmm_unaries(d["image"], d["gmm_fg"], d["gmm_bg"])
    np.testing.assert_allclose(d["u"], u.astype(np.float32), rtol=1e-6, atol=1e-5)
    w64, sig = P.contrast_weights(d["image"], (1, 128, 128), 8, inv_dist=True)
    assert sig == pytest.approx(d["sigma"], rel=1e-12)
    np.testing.assert_array_equal(np.rint(1024.0 * w64).astype(np.int32), d["wq"])
