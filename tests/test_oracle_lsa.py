"""The oracle's LSA-TR block solver (non-submodular Eq. 8) pinned against
exact references: with no negative weight the local approximation is exact,
so LSA-TR must reach the global minimum cut and the whole Algorithm 1 must
equal the submodular oracle; on tiny crops brute force bounds every result."""
import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs


def _crop(d, H, W, y0=0, x0=0):
    G = d["grid"]
    u = d["u"].reshape(G)[y0:y0 + H, x0:x0 + W].reshape(-1)
    w = d["wq"].reshape((2,) + G)[:, y0:y0 + H, x0:x0 + W].copy()
    w[0, :, -1] = 0
    w[1, -1, :] = 0
    return dict(d, grid=(H, W), u=np.ascontiguousarray(u), wq=w.reshape(2, -1))


@pytest.mark.parametrize("seed", range(6))
def test_lsa_on_submodular_reaches_global_minimum(orc, seed):
    d = inputs.random_instance((12, 14), 4, (12, 14), lam=2.0, seed=seed)
    inst = orc.quantise(d["grid"], 4, d["block"], d["u"], d["wq"], d["lam"])
    lab_gc, e_gc = orc.global_mincut(inst)
    lab, e = orc.lsa_tr_global(inst)
    assert e == e_gc and np.array_equal(lab, lab_gc)


@pytest.mark.parametrize("grid,block", [((48, 48), (16, 16)), ((40, 56), (8, 8))])
def test_nsm_admm_on_submodular_equals_oracle(orc, grid, block):
    d = inputs.random_instance(grid, 4, block, lam=2.0, seed=7)
    inst = orc.quantise(d["grid"], 4, d["block"], d["u"], d["wq"], d["lam"])
    ref = orc.admm(inst, d["mu0"])
    got = orc.nsm_admm(inst, d["mu0"])
    assert got["iterations"] == ref["iterations"]
    assert np.array_equal(got["labels"], ref["labels"])
    assert np.array_equal(got["y"], ref["y"]) and got["energy"] == ref["energy"]


def test_lsa_bounded_by_bruteforce_on_crops(orc):
    """4x5 crops of the non-submodular workload: global LSA-TR and DOPE with
    LSA-TR blocks are never below the exact minimum; report how often they hit it."""
    d = inputs.nonsubmodular_instance(size=64)
    hits_g = hits_d = 0
    for c in range(12):
        dc = _crop(d, 4, 5, 4 * c, 3 * c)
        dc["block"] = (2, 5)
        inst = orc.quantise(dc["grid"], 4, dc["block"], dc["u"], dc["wq"], dc["lam"], signed=True)
        eu, ev, w = orc.grid_edges(inst)
        emin, a, o, cnt = orc.bruteforce(inst.n, inst.U, eu, ev, w)
        lab, e = orc.lsa_tr_global(inst)
        assert e >= emin and e == orc.energy(inst, lab)
        r = orc.nsm_admm(inst, 100.0, max_iter=200)
        assert r["energy"] >= emin
        hits_g += e == emin
        hits_d += r["energy"] == emin
    assert hits_g >= 6 and hits_d >= 4


def test_lsa_steps_never_raise_the_energy(orc):
    d = inputs.nonsubmodular_instance(size=32)
    inst = orc.quantise(d["grid"], 4, (32, 32), d["u"], d["wq"], d["lam"], signed=True)
    prev = orc.energy(inst, np.zeros(inst.n, np.uint8))
    for steps in (1, 2, 4, 8, 16, 64):
        lab, e = orc.lsa_tr_global(inst, steps=steps)
        assert e <= prev
        prev = e


# --------------------------------------------------------------------------
# Every LSA-TR step pinned to its definition (the trust-region local
# submodular approximation: Gorelick et al. 2014, as Section 3.4 uses it).
# --------------------------------------------------------------------------

def _block_pixels_edges(inst, k):
    """Image indices of block k's pixels (block-local order) and its own edges
    (local l, local lj, signed weight), enumerated from the grid geometry."""
    D, H, W = (int(x) for x in inst.dims)
    bd, bh, bw = (int(x) for x in inst.block)
    nbz, nby, nbx = D // bd, H // bh, W // bw
    kz, ky, kx = k // (nby * nbx), (k // nbx) % nby, k % nbx
    pix = []
    for lz in range(bd):
        for ly in range(bh):
            for lx in range(bw):
                pix.append(((kz * bd + lz) * H + ky * bh + ly) * W + kx * bw + lx)
    offs = inputs.FWD_OFFSETS[inst.conn]
    edges = []
    for l, i in enumerate(pix):
        lz, ly, lx = l // (bh * bw), (l // bw) % bh, l % bw
        for o, (dz, dy, dx) in enumerate(offs):
            z2, y2, x2 = lz + dz, ly + dy, lx + dx
            if 0 <= z2 < bd and 0 <= y2 < bh and 0 <= x2 < bw:
                w = int(inst.Wl[o, i])
                if w:
                    edges.append((l, (z2 * bh + y2) * bw + x2, w))
    return np.array(pix), edges


def _all_labellings(B):
    return ((np.arange(1 << B)[:, None] >> np.arange(B)[None, :]) & 1).astype(np.int64)


def _energy_all(X, C, edges):
    """Eq. 8's block objective, sum_l C_l x_l + sum_edges w |x_l - x_lj|
    (any sign of w), for every row of X."""
    e = X @ np.asarray(C, np.int64)
    for (l, lj, w) in edges:
        e = e + w * (X[:, l] != X[:, lj])
    return e


def _approx_all(X, r, edges):
    """The recorded approximation: cst + sum un_l x_l + positive n-links."""
    e = r["cst"] + X @ r["un"]
    for (l, lj, w) in edges:
        if w > 0:
            e = e + w * (X[:, l] != X[:, lj])
    return e


def _signed_blocks():
    """Small signed blocks (<= 12 nodes) cut from the non-submodular workload
    and a random signed instance with larger weights."""
    out = []
    d = inputs.nonsubmodular_instance(size=64)
    for c in range(5):
        dc = _crop(d, 4, 6, 5 * c, 4 * c + 1)
        dc["block"] = (2, 6)
        out.append(dc)
    d2 = inputs.nonsubmodular_instance(size=32, seed=3)
    dc = _crop(d2, 3, 4, 7, 9)
    dc["block"] = (3, 4)
    out.append(dc)
    return out


@pytest.mark.parametrize("case", range(6))
def test_lsa_steps_follow_their_definition(orc, case):
    """For every recorded step of every block, exhaustively over all labellings:
    (a) the approximation differs from the block energy by exactly
        sum over negative edges of 2 m (x_l - x^s_l)(x_lj - x^s_lj) (the product
        replaced by its tangent at x^s), so it is exact at x^s and E(x^s) is
        the recorded current energy;
    (b) the step's minimiser is the pointwise-minimal minimiser (AND of all
        minimisers) of approx(x) + lam * Hamming(x, x^s);
    (c) the step's predicted and actual values are approx and E at the
        minimiser, and the minimiser is kept iff E decreases."""
    dc = _signed_blocks()[case]
    inst = orc.quantise(dc["grid"], 4, dc["block"], dc["u"], dc["wq"], dc["lam"], signed=True)
    K = (dc["grid"][0] // dc["block"][0]) * (dc["grid"][1] // dc["block"][1])
    rng = np.random.default_rng(case)
    nsteps = 0
    for k in range(K):
        pix, edges = _block_pixels_edges(inst, k)
        B = len(pix)
        X = _all_labellings(B)
        C = inst.U[pix].astype(np.int64) + rng.integers(-3000, 3000, B)
        x0 = (rng.random(B) < 0.5).astype(np.uint8)
        recs, xf = orc.lsa_tr_block_trace(inst, k, C, x0, steps=16)
        E = _energy_all(X, C, edges)
        assert recs and np.array_equal(recs[0]["x_in"], x0)
        for r in recs:
            xs = r["x_in"].astype(np.int64)
            corr = np.zeros(len(X), np.int64)
            for (l, lj, w) in edges:
                if w < 0:
                    corr += 2 * (-w) * (X[:, l] - xs[l]) * (X[:, lj] - xs[lj])
            A = _approx_all(X, r, edges)
            assert np.array_equal(E - A, corr)                                      # (a)
            idx_s = int((xs << np.arange(B)).sum())
            assert r["ecur"] == E[idx_s] == A[idx_s]
            obj = A + r["lam"] * (X != xs[None, :]).sum(axis=1)                      # (b)
            mins = X[obj == obj.min()]
            assert np.array_equal(r["x_out"], mins.min(axis=0).astype(np.uint8))
            assert obj[int((r["x_out"].astype(np.int64) << np.arange(B)).sum())] == obj.min()
            if not np.array_equal(r["x_out"], r["x_in"]):                            # (c)
                idx = int((r["x_out"].astype(np.int64) << np.arange(B)).sum())
                assert r["ap"] == A[idx] and r["enew"] == E[idx]
                assert r["accepted"] == (r["enew"] < r["ecur"])
            nsteps += 1
        assert _energy_all(X, C, edges)[int((xf.astype(np.int64) << np.arange(B)).sum())] <= E[
            int((x0.astype(np.int64) << np.arange(B)).sum())]
    assert nsteps > 3 * K


@pytest.mark.parametrize("case", range(6))
def test_lsa_trust_region_schedule(orc, case):
    """The trust-region weight and the expansion point evolve as stated: a step
    that does not move divides lam by 4 (and ends the run at lam = 0); an
    accepted step moves x^s to the minimiser and divides lam by 4 when the
    actual decrease is at least 3/4 of the predicted one, else keeps it; a
    rejected step keeps x^s and sets lam = max(4 lam, 1), at most 2^50."""
    dc = _signed_blocks()[case]
    inst = orc.quantise(dc["grid"], 4, dc["block"], dc["u"], dc["wq"], dc["lam"], signed=True)
    K = (dc["grid"][0] // dc["block"][0]) * (dc["grid"][1] // dc["block"][1])
    rng = np.random.default_rng(100 + case)
    for k in range(K):
        pix, edges = _block_pixels_edges(inst, k)
        C = inst.U[pix].astype(np.int64) + rng.integers(-3000, 3000, len(pix))
        recs, xf = orc.lsa_tr_block_trace(inst, k, C, np.zeros(len(pix), np.uint8), steps=16)
        assert recs[0]["lam"] == 1024
        for a, b in zip(recs, recs[1:]):
            moved = not np.array_equal(a["x_out"], a["x_in"])
            if not moved:
                assert a["lam"] > 0 and b["lam"] == a["lam"] // 4
                assert np.array_equal(b["x_in"], a["x_in"])
            elif a["accepted"]:
                R, P = a["ecur"] - a["enew"], a["ecur"] - a["ap"]
                assert b["lam"] == (a["lam"] // 4 if 4 * R >= 3 * P else a["lam"])
                assert np.array_equal(b["x_in"], a["x_out"]) and b["ecur"] == a["enew"]
            else:
                assert b["lam"] == min(max(4 * a["lam"], 1), 1 << 50)
                assert np.array_equal(b["x_in"], a["x_in"]) and b["ecur"] == a["ecur"]
        last = recs[-1]
        if len(recs) < 16:     # stopped early: a step at lam = 0 that did not move
            assert last["lam"] == 0 and np.array_equal(last["x_out"], last["x_in"])


def test_lsa_hand_derived_block(orc):
    """A 1x3 block worked by hand.  C = (3, -1, 2), edge (0,1) weight -4, edge
    (1,2) weight +2: E(x) = 3x0 - x1 + 2x2 - 4|x0 - x1| + 2|x1 - x2|, minimum -3
    at 010 and 011.  From x = 000 the tangent gives un = (3-4, -1-4, 2) =
    (-1, -5, 2), cst 0.  With lam = 1024, 256, 64, 16, 4 every flip costs more
    than it gains, so x stays and lam /= 4.  At lam = 1, approx + Hamming is -2
    at 010 and 110; their AND is 010: predicted -3, actual E(010) = -3, so
    R = P = 3 and the step is kept with lam = 1 // 4 = 0.  Around 010 the tangent
    gives un = (3 - 4 + 8, -5, 2) = (7, -5, 2); the minimisers are 010 and 011,
    AND 010: no move at lam = 0, so the run ends after 7 steps at 010."""
    grid = (1, 3)
    wq = np.zeros((2, 3), np.int32)
    wq[0, 0], wq[0, 1] = -4, 2
    inst = orc.quantise(grid, 4, (1, 3), np.zeros(3, np.float32), wq, 1.0, signed=True)
    recs, xf = orc.lsa_tr_block_trace(inst, 0, np.array([3, -1, 2]), np.zeros(3, np.uint8), steps=16)
    assert [r["lam"] for r in recs] == [1024, 256, 64, 16, 4, 1, 0]
    assert [r["accepted"] for r in recs] == [False] * 5 + [True, False]
    assert list(recs[0]["un"]) == [-1, -5, 2] and recs[0]["cst"] == 0
    assert list(recs[5]["x_out"]) == [0, 1, 0] and recs[5]["ap"] == -3 and recs[5]["enew"] == -3
    assert list(recs[6]["un"]) == [7, -5, 2] and recs[6]["cst"] == 0 and recs[6]["ecur"] == -3
    assert [r["ecur"] for r in recs] == [0] * 6 + [-3]
    assert list(xf) == [0, 1, 0]
