"""The oracle's overlapping-block Algorithm 1 (Q != I) pinned against the
literal matrices of Theorem 1 (oracle/theorem1.py), enumeration, the Q = I
oracle and the structure of the first iteration."""
import itertools

import numpy as np
import pytest

from oracle import theorem1 as T
from paper_1704_03116_gb300 import inputs

CASES = [((8, 12), 4, (4, 4), (1, 1)), ((8, 12), 8, (4, 4), (2, 1)), ((9, 8), 4, (3, 4), (1, 2)),
         ((4, 6, 6), 6, (2, 3, 3), (1, 1, 1)), ((6, 8), 8, (6, 4), (0, 2))]


def _setup(orc, grid, conn, block, grow, seed=0, lam=2.0):
    d = inputs.random_instance(grid, conn, block, lam=lam, seed=seed)
    inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
    g3 = grow if len(grow) == 3 else (0,) + tuple(grow)
    ov = orc.Overlap(inst, g3)
    # dense Theorem 1 on the quantised instance (lambda folded into Wl / 1024)
    Wm = T.grid_pairwise(inst.dims, conn, inst.Wl / 1024.0)
    blocks = T.grid_blocks(inst.dims, inst.block, g3)
    dec = T.Decomposition(inst.U / 1024.0, Wm, blocks)
    return d, inst, ov, dec, blocks


def _to_lists(ov, blocks, box_arr):
    bp = ov.box_pixels()
    out = []
    for k, blk in enumerate(blocks):
        pos = {int(p): i for i, p in enumerate(blk)}
        v = np.zeros(len(blk))
        idx = bp[k * ov.eb:(k + 1) * ov.eb]
        for l in np.nonzero(idx >= 0)[0]:
            v[pos[int(idx[l])]] = box_arr[k * ov.eb + l]
        out.append(v)
    return out


@pytest.mark.parametrize("grid,conn,block,grow", CASES)
def test_overlap_stencils_equal_theorem1(orc, grid, conn, block, grow):
    d, inst, ov, dec, blocks = _setup(orc, grid, conn, block, grow)
    assert np.array_equal(np.diag(dec.Q).astype(int), ov.q)          # Proposition 1's q_ii
    rng = np.random.default_rng(1)
    bp = ov.box_pixels()
    real = bp >= 0
    y = rng.uniform(-0.5, 1.5, inst.n)
    a = np.zeros(ov.K * ov.eb)
    a[real] = rng.normal(0, 0.4, real.sum())
    mu = 123.0
    s, C = ov.caps(y, a, mu)
    a_l = _to_lists(ov, blocks, a)
    s_l = _to_lists(ov, blocks, s)
    for k in range(ov.K):
        ref = dec.block_unary_eq8(k, 1.0, mu, y, a_l[k])                # Eq. 8 unary, literal
        assert np.allclose(s_l[k] / 1024.0, ref, rtol=0, atol=1e-9)
    assert np.array_equal(C[real], np.rint(ov.M * s[real]).astype(np.int64))
    yh = np.zeros(ov.K * ov.eb, np.uint8)
    yh[real] = rng.integers(0, 2, real.sum())
    y2, a2, r2 = ov.update(yh, mu, y, a)
    yh_l = _to_lists(ov, blocks, yh)
    y_ref = dec.update_y_eq10(1.0, mu, yh_l, a_l)                          # Eq. 10, literal
    assert np.allclose(y2, y_ref, rtol=0, atol=1e-12)
    a_ref = dec.update_a_eq11(yh_l, y2, a_l)                               # Eq. 11, literal
    for k, v in enumerate(_to_lists(ov, blocks, a2)):
        assert np.allclose(v, a_ref[k], rtol=0, atol=1e-12)
    assert np.allclose(np.sqrt(r2), dec.residuals(yh_l, y2), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_overlap_block_cut_minimises_scaled_eq8(orc, seed):
    """Each block's cut is a minimiser of the literal Eq. 8 objective (n-links
    W_hat_k, scaled by M), checked by enumeration over the block's pixels."""
    d, inst, ov, dec, blocks = _setup(orc, (6, 6), 4, (3, 3), (1, 1), seed=seed)
    rng = np.random.default_rng(seed)
    bp = ov.box_pixels()
    C = np.zeros(ov.K * ov.eb, np.int64)
    C[bp >= 0] = rng.integers(-3000, 3000, (bp >= 0).sum())
    yh = ov.block_cuts(C)
    for k, blk in enumerate(blocks):
        n = len(blk)
        if n > 16:
            continue
        c = _to_lists(ov, blocks, C)[k]
        Wh = dec.Wh[k] * 1024.0 * ov.M
        assert np.allclose(Wh, np.rint(Wh))                             # integer n-links
        best = None
        for bits in itertools.product((0, 1), repeat=n):
            v = np.array(bits, float)
            e = c @ v + 0.5 * np.sum(Wh * np.abs(v[:, None] - v[None, :]))
            best = e if best is None else min(best, e)
        got = _to_lists(ov, blocks, yh)[k]
        e_got = c @ got + 0.5 * np.sum(Wh * np.abs(got[:, None] - got[None, :]))
        assert e_got == pytest.approx(best, abs=1e-6)


@pytest.mark.parametrize("grid,conn,block", [((24, 32), 4, (8, 8)), ((16, 16), 8, (8, 8)),
                                             ((8, 8, 8), 6, (4, 4, 4))])
def test_overlap_zero_growth_is_the_q_identity_path(orc, grid, conn, block):
    d = inputs.random_instance(grid, conn, block, lam=2.0, seed=5)
    inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
    ref = orc.admm(inst, d["mu0"])
    got = orc.Overlap(inst, (0, 0, 0)).admm(d["mu0"])
    assert got["iterations"] == ref["iterations"]
    assert np.array_equal(got["labels"], ref["labels"])
    assert np.array_equal(got["y"], ref["y"])
    assert got["energy"] == ref["energy"]


def test_overlap_first_iteration_is_independent_block_cuts(orc):
    """At y = 1/2, a = 0 the Eq. 8 unary is U_i / q_i and the n-links W_hat_k:
    iteration 1 solves every block's own subgraph (exact BK on it)."""
    d, inst, ov, dec, blocks = _setup(orc, (16, 20), 8, (8, 10), (2, 2), seed=3)
    y = np.full(inst.n, 0.5)
    a = np.zeros(ov.K * ov.eb)
    yh, y1, a1, r2 = ov.step(100.0, y, a)
    bp = ov.box_pixels()
    for k, blk in enumerate(blocks):
        pos = {int(p): i for i, p in enumerate(blk)}
        q = ov.q[blk]
        c = inst.U[blk] * (ov.M // q)                                   # M U / q
        eu, ev, w = [], [], []
        Wh = np.rint(dec.Wh[k] * 1024.0 * ov.M).astype(np.int64)
        for i in range(len(blk)):
            for j in range(i + 1, len(blk)):
                if Wh[i, j] > 0:
                    eu.append(i); ev.append(j); w.append(Wh[i, j])
        lab = orc.bk_mincut(len(blk), c, eu, ev, w, w)
        got = _to_lists(ov, blocks, yh)[k]
        assert np.array_equal(got, lab)


def test_overlap_energy_not_below_global_minimum_and_prop1(orc):
    d = inputs.ellipses_rgb(size=128, lam=4.0, block=(32, 32))
    inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
    e_gc = orc.global_mincut(inst)[1]
    for grow in ((0, 2, 2), (0, 4, 4)):
        ov = orc.Overlap(inst, grow)
        r = ov.admm(d["mu0"], max_iter=100)
        assert r["energy"] >= e_gc
        if r["converged"]:
            # consistent copies: Proposition 1 gives y = the common labels (up to eps)
            assert np.max(np.abs(r["y"] - r["labels"])) < 1e-2
            bp = ov.box_pixels()
            m = bp >= 0
            assert np.array_equal(r["yhat"][m], r["labels"][bp[m]])
