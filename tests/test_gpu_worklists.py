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
