"""Larger kernels (Section 3: 5x5, 7x7, 9x9 squares in 2-D, the radius-2 ball
in 3-D) in the oracle, pinned like the 3x3 case: stencils against the literal
Theorem 1 matrices, the global cut against enumeration, the overlap form at
zero growth against the Q = I loop, one block against the global minimum."""
import numpy as np
import pytest

from oracle import theorem1 as T
from paper_1704_03116_gb300 import inputs


def test_offset_tables_agree():
    assert inputs.FWD_OFFSETS[24] == T._OFFS[24]
    assert [len(inputs.FWD_OFFSETS[c]) for c in (24, 48, 80, 32)] == [12, 24, 40, 16]
    assert inputs.KERNEL_CONN[(2, 5)] == 24 and inputs.KERNEL_CONN[(3, 5)] == 32


@pytest.mark.parametrize("conn,grid,block", [(24, (4, 5), (4, 5)), (48, (4, 4), (4, 4)), (32, (2, 3, 3), (2, 3, 3))])
def test_big_kernel_global_cut_vs_enumeration(orc, conn, grid, block):
    d = inputs.random_instance(grid, conn, block, lam=1.5, seed=conn)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    eu, ev, w = orc.grid_edges(inst)
    assert len(eu) > inst.n               # more than a 4-neighbourhood
    emin, a_lab, o_lab, cnt = orc.bruteforce(inst.n, inst.U, eu, ev, w)
    lab, e = orc.global_mincut(inst)
    assert e == emin and np.array_equal(lab, a_lab)      # canonical = AND of minimisers


@pytest.mark.parametrize("conn,grid,block,grow", [(24, (8, 12), (4, 4), (1, 1)), (48, (12, 12), (6, 6), (0, 0)),
                                                  (32, (4, 6, 6), (2, 3, 3), (0, 1, 1))])
def test_big_kernel_stencils_equal_theorem1(orc, conn, grid, block, grow):
    d = inputs.random_instance(grid, conn, block, lam=2.0, seed=1)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    g3 = grow if len(grow) == 3 else (0,) + tuple(grow)
    ov = orc.Overlap(inst, g3)
    Wm = T.grid_pairwise(inst.dims, conn, inst.Wl / 1024.0)
    blocks = T.grid_blocks(inst.dims, inst.block, g3)
    dec = T.Decomposition(inst.U / 1024.0, Wm, blocks)
    assert np.array_equal(np.diag(dec.Q).astype(int), ov.q)
    rng = np.random.default_rng(2)
    bp = ov.box_pixels()
    real = bp >= 0
    y = rng.uniform(-0.5, 1.5, inst.n)
    a = np.zeros(ov.K * ov.eb)
    a[real] = rng.normal(0, 0.4, real.sum())
    s, C = ov.caps(y, a, 77.0)
    for k, blk in enumerate(blocks):
        pos = {int(p): i for i, p in enumerate(blk)}
        ak = np.zeros(len(blk))
        sk = np.zeros(len(blk))
        idx = bp[k * ov.eb:(k + 1) * ov.eb]
        for l in np.nonzero(idx >= 0)[0]:
            ak[pos[int(idx[l])]] = a[k * ov.eb + l]
            sk[pos[int(idx[l])]] = s[k * ov.eb + l]
        assert np.allclose(sk / 1024.0, dec.block_unary_eq8(k, 1.0, 77.0, y, ak), rtol=0, atol=1e-9)
    if grow == (0, 0) or g3 == (0, 0, 0):
        # Q = I: the plain stencil functions agree with the overlap form
        a_img = np.zeros(inst.n)
        a_img[bp[real]] = a[real]
        s0, C0 = orc.shifted_caps(inst, y, a_img, 77.0)
        assert np.allclose(s0[bp[real]], s[real], rtol=0, atol=0)


@pytest.mark.parametrize("conn,grid,block", [(24, (24, 32), (8, 8)), (48, (24, 24), (12, 12)), (80, (18, 18), (9, 9)),
                                             (32, (8, 8, 8), (4, 4, 4))])
def test_big_kernel_overlap_form_at_zero_growth_is_q_identity(orc, conn, grid, block):
    d = inputs.random_instance(grid, conn, block, lam=1.0, seed=2)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    ref = orc.admm(inst, d["mu0"])
    got = orc.Overlap(inst, (0, 0, 0)).admm(d["mu0"])
    assert got["iterations"] == ref["iterations"]
    assert np.array_equal(got["labels"], ref["labels"]) and np.array_equal(got["y"], ref["y"])
    assert ref["energy"] >= orc.global_mincut(inst)[1]


def test_big_kernel_one_block_is_global_minimum(orc):
    d = inputs.random_instance((16, 16), 48, (16, 16), lam=1.0, seed=3)
    inst = orc.quantise(d["grid"], 48, d["block"], d["u"], d["wq"], d["lam"])
    r = orc.admm(inst, d["mu0"])
    lab, e = orc.global_mincut(inst)
    assert r["iterations"] == 1 and np.array_equal(r["labels"], lab) and r["energy"] == e
