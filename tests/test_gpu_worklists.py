"""Block worklists of the persistent kernel (k_admm_persistent).

After a launch's first iteration the kernel solves only the blocks on its
solve list and updates only those on its update list; the skipped blocks are
quiet (their Eq. 8 problem provably keeps its labels and their Eq. 10 / 11
update provably leaves the state unchanged).  These tests check that the
skipping is exact: the iterates after any number of iterations, in one launch
or several, equal the oracle's Algorithm 1 and the per-iteration launches
(launch_mode 1, which run every block), bit for bit.  A CTA width given by the
caller (threads) selects the persistent kernel even where the resident one
would fit.  Small mu0 keeps labels moving for many iterations, so blocks
leave and re-enter the lists.
"""
import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    # grid, conn, block, lam, mu0
    ((96, 128), 4, (16, 16), 2.0, 0.5),
    ((128, 96), 8, (16, 32), 4.0, 1.0),
    ((64, 64), 8, (8, 8), 8.0, 3.0),
    ((24, 48, 40), 6, (8, 8, 8), 2.5, 2.0),
    ((16, 64, 64), 6, (8, 16, 16), 3.0, 500.0),
    ((64, 80), 4, (8, 16), 1.0, 100.0),
]


@pytest.fixture(scope="module")
def dp():
    from paper_1704_03116_gb300 import _build
    _build.build()
    from paper_1704_03116_gb300 import dope
    return dope


def _inst(orc, d):
    return orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])


def _oracle_states(orc, inst, mu0, t_max):
    y, a, mu = np.full(inst.n, 0.5), np.zeros(inst.n), mu0
    out = {}
    for t in range(1, t_max + 1):
        yhat, y, a, r2 = orc.admm_step(inst, mu, y, a)
        mu = mu * 1.05
        out[t] = (yhat.copy(), y.copy(), a.copy(), mu)
    return out


@pytest.mark.parametrize("grid,conn,block,lam,mu0", CASES)
def test_worklist_iterates_equal_oracle(orc, dp, grid, conn, block, lam, mu0):
    """Iterate in launches of 1, 2, 5 and 9 iterations; after each launch the
    state (labels, y, a, mu) equals the oracle's after the same iterations."""
    d = inputs.random_instance(grid, conn, block, lam=lam, seed=len(grid) * 7 + conn)
    inst = _inst(orc, d)
    ref = _oracle_states(orc, inst, mu0, 17)
    g = dp.Dope.from_instance(d, mu0=mu0, threads=256 if np.prod(block) <= 2048 else 512)
    g.reset()
    t = 0
    for n in (1, 2, 5, 9):
        done, conv = g.iterate(n)
        if conv:
            break
        t += n
        assert done == t
        st = g.get_state()
        yh, y, a, mu = ref[t]
        assert np.array_equal(st["yhat"], yh), f"t={t}"
        assert np.array_equal(st["y"], y) and np.array_equal(st["a"], a), f"t={t}"
        assert st["mu"] == mu
    assert g.stats()["solver_kernel"] == 1


@pytest.mark.parametrize("grid,conn,block,lam,mu0", CASES)
def test_worklist_solve_equals_oracle_and_mode1(orc, dp, grid, conn, block, lam, mu0):
    """Whole solves: labels, energy, iteration count and residual trace equal
    the oracle's and the per-iteration launches'; the lists skip work."""
    d = inputs.random_instance(grid, conn, block, lam=lam, seed=len(grid) * 5 + conn)
    inst = _inst(orc, d)
    ref = orc.admm(inst, mu0, 1.05, 1e-3, 1000)
    thr = 256 if np.prod(block) <= 2048 else 512
    a = dp.Dope.from_instance(d, mu0=mu0, threads=thr)
    la, Ea, ita = a.solve()
    b = dp.Dope.from_instance(d, mu0=mu0, threads=thr, launch_mode=1)
    lb, Eb, itb = b.solve()
    assert ita == itb and np.array_equal(la, lb) and Ea == Eb
    assert np.array_equal(a.trace(), b.trace())
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["y"], sb["y"]) and np.array_equal(sa["a"], sb["a"])
    if ita == ref["iterations"]:
        assert np.array_equal(la, ref["labels"]) and Ea * 1024 == ref["energy"]
    else:   # the deciding residual sits on eps within rounding (sum order)
        assert abs(ref["rmax"][min(ita, ref["iterations"]) - 1] - 1e-3) <= 1e-12
    st = a.stats()
    assert st["solver_kernel"] == 1
    if ita > 2:
        # later iterations run from the lists, which hold at most every block
        assert st["blocks_solved"] <= a.nblocks * (ita - 1)
        assert st["blocks_updated"] <= a.nblocks * (ita - 1)


def test_worklists_skip_on_volume(orc, dp):
    """On a 3-D volume whose labels freeze after the first iteration most
    blocks leave both lists, and the solve still equals the oracle's."""
    d = inputs.ellipsoids3d(shape=(32, 128, 128))
    inst = _inst(orc, d)
    ref = orc.admm(inst, d["mu0"], 1.05, 1e-3, 1000)
    g = dp.Dope.from_instance(d, threads=512)
    lab, E, it = g.solve()
    assert it == ref["iterations"] and np.array_equal(lab, ref["labels"]) and E * 1024 == ref["energy"]
    st = g.stats()
    assert it > 3 and st["blocks_solved"] < 0.5 * g.nblocks * (it - 1), st


def test_worklists_after_set_state(orc, dp):
    """A state set from outside (checkpoint / resume) is never trusted by the
    lists: the next launch's first iteration does every block."""
    d = inputs.random_instance((96, 96), 8, (16, 16), lam=3.0, seed=8)
    inst = _inst(orc, d)
    ref = _oracle_states(orc, inst, 2.0, 12)
    g = dp.Dope.from_instance(d, mu0=2.0, threads=256)
    yh, y, a, mu = ref[4]
    g.set_state(y, a, yh, mu, 4)
    done, conv = g.iterate(8)
    st = g.get_state()
    yh, y, a, mu = ref[12]
    assert done == 12 and np.array_equal(st["yhat"], yh)
    assert np.array_equal(st["y"], y) and np.array_equal(st["a"], a)


def test_batched_worklists_equal_oracle(orc, dp):
    """The batched launch keeps per-problem worklists too: problems of several
    shapes with small mu0 (labels move for many iterations), advanced in
    launches of 1, 4 and 7 iterations, equal the oracle's states after the same
    iterations, and skip blocks after their first iteration in a launch."""
    cases = [inputs.random_instance(gr, cn, bl, lam=lam, seed=s) for (gr, cn, bl, lam, s) in (
        ((96, 128), 4, (16, 16), 2.0, 1), ((64, 96), 8, (16, 32), 4.0, 2), ((24, 48, 40), 6, (8, 8, 8), 2.5, 3),
        ((128, 128), 8, (32, 32), 8.0, 4))]
    mu0s = [0.5, 1.0, 2.0, 3.0]
    refs = []
    for d, mu0 in zip(cases, mu0s):
        refs.append(_oracle_states(orc, _inst(orc, d), mu0, 12))
    gs = [dp.Dope.from_instance(d, mu0=mu0) for d, mu0 in zip(cases, mu0s)]
    for g in gs:
        g.reset()
    t = 0
    for n in (1, 4, 7):
        res = dp.iterate_batch(gs, n)
        t += n
        for g, ref, (it, conv, st) in zip(gs, refs, res):
            assert st == 0 and it == t and not conv
            s = g.get_state()
            yh, y, a, mu = ref[t]
            assert np.array_equal(s["yhat"], yh), t
            assert np.array_equal(s["y"], y) and np.array_equal(s["a"], a), t


def test_batched_worklists_skip_and_match_oracle(orc, dp):
    """At the paper's mu0 labels freeze after a few iterations: a batch solved to
    convergence in one launch matches the oracle's solves and, after each
    problem's first iteration, solves fewer blocks than it has."""
    cases = [inputs.ellipses_rgb(size=256, lam=lam) for lam in (1.0, 8.0)] + \
        [inputs.ellipsoids3d(shape=(32, 96, 96)), inputs.random_instance((192, 160), 4, (16, 16), lam=2.0, seed=9)]
    gs = [dp.Dope.from_instance(d) for d in cases]
    res = dp.iterate_batch(gs, 1000)
    for j, (d, g, (it, conv, st)) in enumerate(zip(cases, gs, res)):
        ref = orc.admm(_inst(orc, d), d["mu0"], 1.05, 1e-3, 1000)
        assert st == 0 and conv and it == ref["iterations"]
        lab, e = g.labels()
        assert np.array_equal(lab, ref["labels"]) and e == ref["energy"]
        s = g.stats()
        assert s["solver_kernel"] == 3 and s["blocks_solved"] > 0
        if j < 3:       # the noisy random field keeps label boundaries on most block faces
            assert s["blocks_solved"] < g.nblocks * (it - 1), (s, g.nblocks, it)


def test_worklists_dropped_when_inputs_change(orc, dp):
    """Lists left by a launch are reused by the next launch only while nothing
    changed: new unaries between two launches must be seen by every block."""
    d = inputs.random_instance((96, 96), 8, (16, 16), lam=2.0, seed=12)
    d2 = dict(d, u=np.ascontiguousarray(d["u"][::-1]))      # other unaries, same weights
    i1, i2 = _inst(orc, d), _inst(orc, d2)
    g = dp.Dope.from_instance(d, mu0=100.0, threads=256)
    g.reset()
    done, conv = g.iterate(6)
    assert done == 6 and not conv
    g.set_unaries(d2["u"])
    done, conv = g.iterate(5)
    st = g.get_state()
    y, a, mu = np.full(i1.n, 0.5), np.zeros(i1.n), 100.0
    for t in range(done):
        yh, y, a, r2 = orc.admm_step(i1 if t < 6 else i2, mu, y, a)
        mu *= 1.05
    assert np.array_equal(st["yhat"], yh) and np.array_equal(st["y"], y) and np.array_equal(st["a"], a)
