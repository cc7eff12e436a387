"""GPU parity of the whole-image potentials (Algorithm 1's first step) against
the oracle (oracle/potentials.py).

  * data term: FP32 on the device vs the FP64 definition.  Tolerance from the
    arithmetic: every component term c_j - q_j / 2 is formed from FP32-rounded
    constants and ~C^2 fused operations, so its error is a small multiple of
    the FP32 unit roundoff (6e-8) times the magnitude of the terms, which the
    two log-likelihoods bound; 4e-6 (|ll_fg| + |ll_bg| + 1) leaves a margin of
    about 60 roundoffs.
  * weights: against the FP64 definition, w = exp(-|x_i - x_j|^2 / (2 s^2))
    (divided by the pixel distance where asked) at the kernel's sigma s,
    quantised rne(1024 w).  The kernel decides in FP32: |x_i - x_j|^2 carries
    at most (C + 2) roundings, k = 1 / (2 s^2) one, their product one, exp a
    few ulp, so the argument a = d2 k is off by at most (C + 4) 2^-24 a and
    1024 w by at most 1024 (a e^-a (C + 4) + 4) 2^-24 <= 1024 (0.37 (C + 4) + 4)
    6e-8 < 5e-4 (C <= 4).  So the quantised weights equal the definition's
    wherever 1024 w lies farther than 1e-3 from a rounding tie, and are within
    one of it everywhere.
  * sigma (the mean contrast): each pair's root in FP32 (at most C + 3
    roundings) and each pixel's sum of up to conn/2 roots in FP32, then FP64:
    relative error below (C + 3 + conn/2) 2^-24 <= 1e-5 of the FP64 definition.
"""
import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    from paper_1704_03116_gb300 import _build
    _build.build()
    from paper_1704_03116_gb300 import dope
    return dope


@pytest.fixture(scope="module")
def P():
    from oracle import potentials
    return potentials


@pytest.fixture(scope="module")
def ell():
    return inputs.ellipses_rgb()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _spd(rng, C, scale):
    A = rng.normal(0, scale, (C, C))
    return A @ A.T + scale * scale * np.eye(C)


def _mix(rng, K, C, scale=0.08):
    w = rng.uniform(0.2, 1.0, K)
    return w / w.sum(), rng.uniform(0, 1, (K, C)), np.stack([_spd(rng, C, scale) for _ in range(K)])


def _check_u(P, img, fg, bg, got, clip=1.0e5):
    img = np.asarray(img, np.float32)          # the values the device sees
    u, lf, lb = P.gmm_unaries(img, fg, bg, clip=clip)
    err = np.abs(got.astype(np.float64) - u)
    tol = 4e-6 * (np.abs(lf) + np.abs(lb) + 1.0)
    bad = err > tol
    assert not bad.any(), (int(bad.sum()), float((err / tol).max()))
    return float((err / tol).max())


def test_unaries_ellipses512(dp, P, ell):
    img = _cuda(ell["image"])
    got = dp.dope_gmm_unaries(img, ell["gmm_fg"], ell["gmm_bg"]).cpu().numpy()
    _check_u(P, ell["image"], ell["gmm_fg"], ell["gmm_bg"], got)


@pytest.mark.parametrize("C,K,n", [(1, 1, 4097), (2, 5, 70001), (3, 3, 1000), (3, 8, 65536), (4, 7, 12345),
                                   (4, 1, 1), (3, 2, 255)])
def test_unaries_random_mixtures(dp, P, C, K, n):
    rng = np.random.default_rng(100 * C + K)
    fg, bg = _mix(rng, K, C), _mix(rng, max(1, K - 1), C, 0.2)
    img = rng.uniform(-0.2, 1.2, (n, C))
    got = dp.dope_gmm_unaries(_cuda(img), fg, bg).cpu().numpy()
    _check_u(P, img, fg, bg, got)


def test_unaries_clip_and_empty(dp, P):
    import torch
    rng = np.random.default_rng(7)
    fg = ([1.0], [[0.1, 0.1, 0.1]], [1e-4 * np.eye(3)])
    bg = ([1.0], [[0.9, 0.9, 0.9]], [1e-4 * np.eye(3)])
    img = rng.uniform(0, 1, (5000, 3))
    got = dp.dope_gmm_unaries(_cuda(img), fg, bg, clip=50.0).cpu().numpy()
    assert np.abs(got).max() <= 50.0 and (np.abs(got) == 50.0).mean() > 0.5
    _check_u(P, img, fg, bg, got, clip=50.0)
    empty = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    assert dp.dope_gmm_unaries(empty, fg, bg).numel() == 0


def _check_w(P, img, dims, conn, got, sig_got, sigma=None, inv_dist=False):
    """The kernel's quantised weights against the FP64 definition (see the
    module docstring for the tie band and the sigma bound)."""
    img = np.asarray(img, np.float32)
    if sigma is None:
        sig64 = max(P.mean_contrast(img, dims, conn), 1e-6)
        assert abs(sig_got - sig64) <= 1e-5 * sig64, (sig_got, sig64)
    else:
        assert sig_got == sigma
    w64, _ = P.contrast_weights(img, dims, conn, sigma=sig_got, inv_dist=inv_dist)
    v = 1024.0 * w64
    ref = np.rint(v).astype(np.int64)
    margin = np.abs(np.abs(v - np.floor(v)) - 0.5)
    diff = np.abs(got.astype(np.int64) - ref)
    assert diff.max() <= 1
    assert (diff[margin > 1e-3] == 0).all(), int((diff[margin > 1e-3] != 0).sum())
    return int((diff != 0).sum())


def test_weights_ellipses512(dp, P, ell):
    img = _cuda(ell["image"])
    got, sig = dp.dope_contrast_weights(img, (512, 512), 8, channels=3, inv_dist=True)
    _check_w(P, ell["image"], (1, 512, 512), 8, got.cpu().numpy(), sig, inv_dist=True)
    # the generator's FP64 weights agree to within one as well
    assert np.abs(got.cpu().numpy().astype(np.int64) - ell["wq"]).max() <= 1


@pytest.mark.parametrize("conn,grid,C,sigma,inv_dist", [
    (4, (37, 53), 3, None, False), (8, (64, 33), 2, 0.3, True), (24, (40, 45), 3, None, True),
    (48, (29, 31), 1, None, True), (80, (33, 40), 4, 0.5, False), (6, (9, 17, 23), 1, None, False),
    (32, (7, 12, 11), 3, None, True), (8, (1, 300), 3, None, True), (4, (300, 1), 1, None, False)])
def test_weights_random_images(dp, P, conn, grid, C, sigma, inv_dist):
    rng = np.random.default_rng(conn + C)
    dims = grid if len(grid) == 3 else (1,) + grid
    n = int(np.prod(dims))
    img = np.round(rng.uniform(0, 1, (n, C)) * 8) / 8 + rng.normal(0, 0.02, (n, C))   # regions plus noise
    got, sig = dp.dope_contrast_weights(_cuda(img), grid, conn, channels=C,
                                        sigma=0.0 if sigma is None else sigma, inv_dist=inv_dist)
    _check_w(P, img, dims, conn, got.cpu().numpy(), sig, sigma=sigma, inv_dist=inv_dist)


def test_weights_single_pixel_and_constant(dp, P):
    got, sig = dp.dope_contrast_weights(_cuda(np.zeros((1, 3))), (1, 1), 8, channels=3)
    assert sig == 1e-6 and (got.cpu().numpy() == 0).all()
    got, sig = dp.dope_contrast_weights(_cuda(np.full((6 * 7, 3), 0.25)), (6, 7), 8, channels=3, inv_dist=True)
    wq = got.cpu().numpy().reshape(4, 6, 7)
    assert sig == 1e-6
    assert (wq[0][:, :-1] == 1024).all() and (wq[0][:, -1] == 0).all()
    assert (wq[2][:-1, :-1] == 724).all() and (wq[3][:-1, 1:] == 724).all() and (wq[3][:, 0] == 0).all()


def test_ellipsoids_volume(dp, P):
    d = inputs.ellipsoids3d(shape=(16, 48, 40), block=(8, 16, 8))
    img = d["image"]
    got_u = dp.dope_gmm_unaries(_cuda(img), d["gmm_fg"], d["gmm_bg"]).cpu().numpy()
    _check_u(P, img, d["gmm_fg"], d["gmm_bg"], got_u)
    got, sig = dp.dope_contrast_weights(_cuda(img), (16, 48, 40), 6, channels=1)
    _check_w(P, img, (16, 48, 40), 6, got.cpu().numpy(), sig)


@pytest.mark.parametrize("conn,grid,block,grow", [(8, (128, 96), (32, 32), None), (4, (64, 64), (16, 16), None),
                                                  (24, (48, 64), (16, 16), (2, 2)), (8, (64, 64), (16, 16), (2, 2))])
@pytest.mark.parametrize("where", ["device", "host"])
def test_set_image_equals_two_step(dp, conn, grid, block, grow, where):
    """set_image then solve == the two potentials calls, set_unaries /
    set_weights, then solve: the same labels, energy and iterations."""
    rng = np.random.default_rng(conn)
    n = grid[0] * grid[1]
    img = (np.round(rng.uniform(0, 1, (n, 3)) * 3) / 3 + rng.normal(0, 0.05, (n, 3))).astype(np.float32)
    fg, bg = _mix(rng, 3, 3, 0.1), _mix(rng, 2, 3, 0.1)
    kw = dict(max_iter=200) if grow is None else dict(grow=grow, max_iter=4)
    a = dp.Dope(grid, conn, block, 2.0, **kw)
    u = dp.dope_gmm_unaries(_cuda(img), fg, bg, clip=50.0)
    wq, sig = dp.dope_contrast_weights(_cuda(img), grid, conn, channels=3, inv_dist=True)
    a.set_unaries(u)
    a.set_weights(wq)
    la, ea, ia = a.solve(allow_notconv=True)
    b = dp.Dope(grid, conn, block, 2.0, **kw)
    sig_b = b.set_image(_cuda(img) if where == "device" else img, fg, bg, clip=50.0, inv_dist=True)
    lb, eb, ib = b.solve(allow_notconv=True)
    assert sig_b == pytest.approx(sig, rel=1e-12)
    assert ia == ib and ea == eb and np.array_equal(la, lb)
    a.close()
    b.close()


def test_serving_base_2048_sampled(dp, P):
    """The 2048 x 2048 image the serving stream crops from: every weight
    against the FP32 restatement, the data term on a sample of pixels."""
    d = inputs.serving_base(0)
    img = d["image"].reshape(-1, 3)
    img_d = _cuda(img)
    u = dp.dope_gmm_unaries(img_d, d["gmm_fg"], d["gmm_bg"]).cpu().numpy()
    idx = np.random.default_rng(0).choice(img.shape[0], 20000, replace=False)
    _check_u(P, img[idx], d["gmm_fg"], d["gmm_bg"], u[idx])
    got, sig = dp.dope_contrast_weights(img_d, (2048, 2048), 8, channels=3, inv_dist=True)
    _check_w(P, img, (1, 2048, 2048), 8, got.cpu().numpy(), sig, inv_dist=True)
