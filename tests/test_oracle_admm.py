"""Pins of the oracle's ADMM arithmetic (Eq. 5, 8, 10, 11, Algorithm 1) against
the literal matrix form of Theorem 1, Proposition 1, closed forms and the
special cases the method reduces to."""
import itertools

import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs
from oracle import theorem1 as T1


def _inst(orc, d):
    return orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])


def _decomp(inst, grow=(0, 0, 0)):
    """Theorem 1 matrices with lambda * w_ij = Wl_ij / 1024 and u = U / 1024."""
    Wm = T1.grid_pairwise(inst.dims, inst.conn, inst.Wl.astype(np.float64) / 1024.0)
    blocks = T1.grid_blocks(inst.dims, inst.block, grow)
    return T1.Decomposition(inst.U.astype(np.float64) / 1024.0, Wm, blocks), blocks


CASES = [((4, 6), 4, (2, 3)), ((6, 6), 8, (3, 3)), ((2, 4, 4), 6, (1, 2, 2)), ((4, 8), 8, (4, 4))]


@pytest.mark.parametrize("grid,conn,block", CASES)
@pytest.mark.parametrize("grow", [(0, 0, 0), (0, 1, 1)])
def test_theorem1_reformulation_equals_energy(orc, grid, conn, block, grow):
    """Theorem 1: with yhat_k = S_k y (y binary) the objective of Eq. 5 equals
    u^T y + lambda y^T L y (Eq. 3), for non-overlapping and overlapping blocks."""
    d = inputs.random_instance(grid, conn, block, lam=1.3, seed=3)
    inst = _inst(orc, d)
    dec, blocks = _decomp(inst, grow if len(grid) == 2 else (0, 0, 0))
    rng = np.random.default_rng(0)
    for _ in range(20):
        y = (rng.random(inst.n) < 0.5).astype(np.float64)
        yh = [S @ y for S in dec.S]
        assert dec.objective_eq5(1.0, y, yh) == pytest.approx(dec.energy_eq3(1.0, y), rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("grid,conn,block", CASES)
def test_eq3_matches_integer_energy(orc, grid, conn, block):
    """Eq. 3 (y^T L y) counts each undirected edge once: it equals the oracle's
    integer E_int / 1024 for binary y."""
    d = inputs.random_instance(grid, conn, block, lam=2.0, seed=5)
    inst = _inst(orc, d)
    dec, _ = _decomp(inst)
    rng = np.random.default_rng(1)
    for _ in range(10):
        y = (rng.random(inst.n) < 0.5).astype(np.uint8)
        assert orc.energy(inst, y) / 1024.0 == pytest.approx(dec.energy_eq3(1.0, y.astype(float)), abs=1e-9)


def test_prop1_overlapping(orc):
    """Proposition 1: consistent block labels give back y = Q^-1 sum S_k^T yhat_k."""
    d = inputs.random_instance((6, 8), 4, (3, 4), seed=1)
    inst = _inst(orc, d)
    dec, _ = _decomp(inst, (0, 1, 1))
    assert np.max(np.diag(dec.Q)) > 1
    y = (np.random.default_rng(2).random(inst.n) < 0.5).astype(float)
    assert np.array_equal(dec.prop1([S @ y for S in dec.S]), y)


@pytest.mark.parametrize("grid,conn,block", CASES)
def test_stencil_caps_equal_matrix_eq8(orc, grid, conn, block):
    """The oracle's per-pixel Eq. 8 unary (stencil form, x1024) equals the literal
    u_hat_k + lambda (C_k + R_k S_k) y + mu (a_k - S_k y + 1/2) of Theorem 1
    for arbitrary real (y, a, mu)."""
    d = inputs.random_instance(grid, conn, block, lam=1.7, seed=11)
    inst = _inst(orc, d)
    dec, blocks = _decomp(inst)
    rng = np.random.default_rng(4)
    for _ in range(5):
        y = rng.random(inst.n)
        a = rng.normal(0, 0.3, inst.n)
        mu = float(rng.uniform(1, 300))
        s, C = orc.shifted_caps(inst, y, a, mu)
        ref = np.zeros(inst.n)
        for k, b in enumerate(blocks):
            ref[b] = dec.block_unary_eq8(k, 1.0, mu, y, a[b])
        np.testing.assert_allclose(s / 1024.0, ref, rtol=1e-11, atol=1e-9)
        assert np.array_equal(C, np.rint(s).astype(np.int64))


@pytest.mark.parametrize("grid,conn,block", CASES)
def test_stencil_update_equals_matrix_eq10_eq11(orc, grid, conn, block):
    """The oracle's y / a updates equal Eq. 10 and Eq. 11 in matrix form, and the
    per-block residuals equal ||yhat_k - S_k y||^2."""
    d = inputs.random_instance(grid, conn, block, lam=0.9, seed=12)
    inst = _inst(orc, d)
    dec, blocks = _decomp(inst)
    rng = np.random.default_rng(5)
    for _ in range(5):
        yhat = (rng.random(inst.n) < 0.5).astype(np.uint8)
        a = rng.normal(0, 0.05, inst.n)
        y0 = rng.random(inst.n)
        mu = float(rng.uniform(50, 500))
        y1, a1, r2 = orc.update(inst, yhat, mu, y0, a)
        yh = [yhat[b].astype(float) for b in blocks]
        al = [a[b] for b in blocks]
        y_ref = dec.update_y_eq10(1.0, mu, yh, al)
        a_ref = dec.update_a_eq11(yh, y_ref, al)
        np.testing.assert_allclose(y1, y_ref, rtol=0, atol=1e-12)
        for k, b in enumerate(blocks):
            np.testing.assert_allclose(a1[b], a_ref[k], rtol=0, atol=1e-12)
        np.testing.assert_allclose(np.sqrt(r2), dec.residuals(yh, y_ref), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("grid,conn,block", [((4, 6), 4, (2, 3)), ((4, 4), 8, (2, 2)), ((2, 4, 4), 6, (1, 2, 2))])
@pytest.mark.parametrize("seed", range(3))
def test_block_cut_minimises_eq8(orc, grid, conn, block, seed):
    """At the first iteration (y = 1/2, a = 0) the Eq. 8 unary is exactly u, so
    the oracle's block labels must be the pointwise-minimal minimiser of the
    literal Eq. 8 objective of each block (enumerated)."""
    d = inputs.random_instance(grid, conn, block, lam=1.0, seed=seed, u_scale=1.5)
    inst = _inst(orc, d)
    dec, blocks = _decomp(inst)
    y = np.full(inst.n, 0.5)
    a = np.zeros(inst.n)
    s, C = orc.shifted_caps(inst, y, a, 100.0)
    assert np.array_equal(C, inst.U)
    yhat = orc.block_cuts(inst, C)
    for k, b in enumerate(blocks):
        nb = len(b)
        best, mins = None, []
        for bits in itertools.product([0, 1], repeat=nb):
            e = dec.block_energy_eq8(k, 1.0, 100.0, y, a[b], np.array(bits, float))
            if best is None or e < best - 1e-9:
                best, mins = e, [bits]
            elif abs(e - best) <= 1e-9:
                mins.append(bits)
        assert yhat[b].tolist() == np.min(np.array(mins), axis=0).tolist()


@pytest.mark.parametrize("seed", range(4))
def test_block_cut_vs_bruteforce_any_caps(orc, seed):
    """Given arbitrary integer unaries (later iterations), each block's cut is the
    AND of all minimisers of C.y + sum_{intra edges} Wl |y_i - y_j|."""
    d = inputs.random_instance((8, 8), 4, (4, 4), lam=1.0, seed=seed)
    inst = _inst(orc, d)
    rng = np.random.default_rng(seed)
    C = rng.integers(-3000, 3000, inst.n)
    yhat = orc.block_cuts(inst, C)
    eu, ev, w = orc.grid_edges(inst, within_blocks=True)
    blocks = T1.grid_blocks(inst.dims, inst.block)
    for b in blocks:
        loc = {int(g): i for i, g in enumerate(b)}
        sel = [e for e in range(len(eu)) if int(eu[e]) in loc and int(ev[e]) in loc]
        bu = np.array([loc[int(eu[e])] for e in sel], np.int32)
        bv = np.array([loc[int(ev[e])] for e in sel], np.int32)
        emin, and_lab, _, _ = orc.bruteforce(len(b), C[b], bu, bv, w[sel])
        assert yhat[b].tolist() == and_lab.tolist()


def test_single_block_is_global_mincut(orc):
    """K = 1: C_k = R_k = 0, so one iteration is the exact global min-cut and the
    residual is 0 (Algorithm 1 stops after one iteration)."""
    d = inputs.random_instance((24, 24), 8, (24, 24), lam=2.0, seed=2)
    inst = _inst(orc, d)
    res = orc.admm(inst, 100.0)
    lab, e = orc.global_mincut(inst)
    assert res["iterations"] == 1
    assert res["labels"].tolist() == lab.tolist()
    assert res["energy"] == e


def test_lambda_zero_is_thresholding(orc):
    """lambda = 0: every sub-problem is separable, yhat_i = [U_i < 0] (ties -> 0),
    y = yhat, one iteration."""
    d = inputs.random_instance((16, 16), 4, (4, 4), lam=0.0, seed=4)
    d["u"][:5] = 0.0
    inst = _inst(orc, d)
    res = orc.admm(inst, 100.0)
    assert res["iterations"] == 1
    assert res["labels"].tolist() == (inst.U < 0).astype(np.uint8).tolist()


def test_first_iteration_is_independent_block_cuts(orc):
    """y = 1/2, a = 0 makes every shift vanish: iteration 1 = global min-cut of
    each block with the cross-block edges dropped (checked by enumeration)."""
    d = inputs.random_instance((4, 5), 4, (2, 5), lam=1.2, seed=9)
    inst = _inst(orc, d)
    yhat, y, a, r2 = orc.admm_step(inst, 100.0, np.full(inst.n, 0.5), np.zeros(inst.n))
    eu, ev, w = orc.grid_edges(inst, within_blocks=True)
    emin, and_lab, _, _ = orc.bruteforce(inst.n, inst.U, eu, ev, w)
    assert yhat.tolist() == and_lab.tolist()


def test_multiplier_closed_form(orc):
    """For Q = I, Eq. 10 + Eq. 11 give a = g(yhat) / mu with
    g_i = sum_{j in X(i)} lambda w_ij (yhat_i - yhat_j), starting from a = 0."""
    d = inputs.random_instance((16, 16), 8, (4, 4), lam=3.0, seed=6)
    inst = _inst(orc, d)
    mu = 100.0
    yhat, y, a, r2 = orc.admm_step(inst, mu, np.full(inst.n, 0.5), np.zeros(inst.n))
    blocks = T1.grid_blocks(inst.dims, inst.block)
    # g from the definition with the dense W: sum over cross-block neighbours
    W = T1.grid_pairwise(inst.dims, inst.conn, inst.Wl.astype(float) / 1024.0)
    bid = np.zeros(inst.n, int)
    for k, b in enumerate(blocks):
        bid[b] = k
    cross = (bid[:, None] != bid[None, :]) * W
    yh = yhat.astype(float)
    g = cross.sum(1) * yh - cross @ yh
    np.testing.assert_allclose(a, g / mu, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(y, yh - g / mu, rtol=0, atol=1e-12)


def test_residual_decay_after_labels_freeze(orc):
    """Once yhat stops changing, yhat - y = (1/mu_t - 1/mu_{t-1}) g, so each block
    residual shrinks by exactly 1/mu_fact per iteration (up to rounding)."""
    d = inputs.disk64()
    inst = _inst(orc, d)
    res = orc.admm(inst, 100.0, 1.05, 1e-3, 1000)
    flips, r = res["flips"], res["rmax"]
    t_freeze = max(i for i in range(len(flips)) if flips[i] > 0) + 1
    assert res["converged"]
    for t in range(t_freeze + 1, len(r)):
        assert r[t] / r[t - 1] == pytest.approx(1 / 1.05, rel=1e-9)


@pytest.mark.parametrize("name", ["disk64", "random"])
def test_admm_energy_not_below_global_minimum(orc, name):
    d = inputs.disk64() if name == "disk64" else inputs.random_instance((64, 64), 8, (16, 16), lam=2.0, seed=1)
    inst = _inst(orc, d)
    res = orc.admm(inst, d["mu0"])
    lab, e = orc.global_mincut(inst)
    assert res["converged"]
    assert res["energy"] >= e
    # and the energy equals E_int of the returned labels
    assert res["energy"] == orc.energy(inst, res["labels"])


def test_admm_step_matches_admm_loop(orc):
    """orc_admm is orc_admm_step repeated with mu <- mu * mu_fact."""
    d = inputs.random_instance((32, 32), 4, (8, 8), lam=2.0, seed=3)
    inst = _inst(orc, d)
    res = orc.admm(inst, 100.0, 1.05, 1e-3, 6)
    y, a, mu = np.full(inst.n, 0.5), np.zeros(inst.n), 100.0
    for t in range(res["iterations"]):
        yhat, y, a, r2 = orc.admm_step(inst, mu, y, a)
        assert np.sqrt(r2.max()) == res["rmax"][t]
        mu = mu * 1.05
    assert yhat.tolist() == res["labels"].tolist()
    assert np.array_equal(y, res["y"]) and np.array_equal(a, res["a"])


@pytest.mark.parametrize("grid,conn,block", [((37, 50), 4, (16, 16)), ((45, 29), 8, (8, 8)),
                                             ((9, 13, 11), 6, (4, 4, 4))])
def test_padding_pixels_change_nothing(orc, grid, conn, block):
    """Isolated zero-cost pixels (the request server's padding of ragged grids)
    leave Algorithm 1 unchanged on the caller's pixels: same labels, same
    iteration count, same energy, and the global minimum is unchanged.  Pinned
    against the unpadded instance on a grid that the blocks tile, padded by
    one more row of blocks."""
    from paper_1704_03116_gb300 import inputs
    tiled = tuple(g // b * b for g, b in zip(grid, block))
    d = inputs.random_instance(tiled, conn, block, lam=2.0, seed=sum(grid))
    base = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
    ref = orc.admm(base, d["mu0"])
    # pad: one more block along the first axis, and the padded instance of a
    # ragged crop that pad_to_blocks rounds back up to `tiled`
    big = dict(d)
    big["grid"] = (tiled[0] + block[0],) + tiled[1:]
    big["unpadded_grid"] = tiled
    nh = d["wq"].shape[0]
    u = np.zeros(big["grid"], np.float32)
    u[:tiled[0]] = d["u"].reshape(tiled)
    w = np.zeros((nh,) + big["grid"], np.int32)
    w[:, :tiled[0]] = d["wq"].reshape((nh,) + tiled)
    big["u"], big["wq"] = u.reshape(-1), w.reshape(nh, -1)
    inst = orc.quantise(big["grid"], conn, block, big["u"], big["wq"], 2.0)
    got = orc.admm(inst, d["mu0"])
    assert got["iterations"] == ref["iterations"]
    assert np.array_equal(inputs.crop_padded(got["labels"], big), ref["labels"])
    assert got["energy"] == ref["energy"]
    assert orc.global_mincut(inst)[1] == orc.global_mincut(base)[1]
    # pad_to_blocks itself: a ragged grid is rounded up with zero pixels
    r = inputs.random_instance(grid, conn, block, lam=1.0, seed=1)
    p = inputs.pad_to_blocks(r)
    assert all(g % b == 0 for g, b in zip(p["grid"], block))
    assert np.array_equal(inputs.crop_padded(p["u"], p), r["u"])
    assert p["u"].size - r["u"].size == np.count_nonzero(p["u"] == 0) - np.count_nonzero(r["u"] == 0)
