"""Run-ahead windows of the persistent kernel (k_admm_persistent, launch_mode 0).

Once an iteration solves no block by a cut, the kernel advances several
iterations at once over the blocks on its solve list: the moving face slots'
states are stepped through the window, every window iteration's Eq. 8 forced
tests are certified (interval certificates; at the window's first iteration the
exact unary where those are too weak), and the first iteration whose stop test
holds is committed.  These tests
check that a solve with windows equals, bit for bit, the same solve without
them (launch_mode 2) and the oracle's Algorithm 1: labels, energy, iteration
count, residual trace and the final state (y, a, labels), in one launch or in
launches cut short by the iteration limit.  The grids have more blocks than the
persistent launch has CTAs, which is where windows run.
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


def _inst(orc, d):
    return orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])


def _solve_pair(dp, d, **kw):
    out = []
    for mode in (0, 2):
        g = dp.Dope.from_instance(d, launch_mode=mode, **kw)
        lab, E, it = g.solve(allow_notconv=True)
        out.append((g, lab, E, it, g.trace(), g.get_state(), g.stats()))
    return out


def _assert_same(w, p):
    gw, lw, Ew, itw, tw, sw, stw = w
    gp, lp, Ep, itp, tp, sp, stp = p
    assert itw == itp and Ew == Ep and np.array_equal(lw, lp)
    assert np.array_equal(tw, tp)
    for key in ("y", "a", "yhat"):
        assert np.array_equal(sw[key].view(np.uint8), sp[key].view(np.uint8)), key
    assert sw["mu"] == sp["mu"] and sw["t"] == sp["t"]
    assert stp["windows"] == 0


@pytest.fixture(scope="module")
def volume():
    # 8 x 8 x 8 blocks of 8 x 16 x 16: more blocks than the launch's CTAs
    return inputs.ellipsoids3d(shape=(64, 128, 128))


def test_windows_on_volume_equal_plain_and_oracle(orc, dp, volume):
    d = volume
    w, p = _solve_pair(dp, d, threads=512)
    _assert_same(w, p)
    st = w[6]
    assert st["windows"] >= 1 and st["window_iterations"] >= 2, st
    ref = orc.admm(_inst(orc, d), d["mu0"], 1.05, 1e-3, 1000)
    assert w[3] == ref["iterations"] and np.array_equal(w[1], ref["labels"]) and w[2] * 1024 == ref["energy"]
    assert np.array_equal(w[5]["y"], ref["y"]) and np.array_equal(w[5]["a"], ref["a"])


@pytest.mark.parametrize("max_iter", [4, 5, 9, 13])
def test_windows_cut_by_the_iteration_limit(orc, dp, volume, max_iter):
    """A window never runs past the launch's last iteration; the state after
    max_iter iterations equals the plain launch's and the oracle's."""
    d = volume
    w, p = _solve_pair(dp, d, threads=512, max_iter=max_iter)
    _assert_same(w, p)
    inst = _inst(orc, d)
    y, a, mu = np.full(inst.n, 0.5), np.zeros(inst.n), d["mu0"]
    for _ in range(max_iter):
        yh, y, a, r2 = orc.admm_step(inst, mu, y, a)
        mu *= 1.05
    s = w[5]
    assert np.array_equal(s["yhat"], yh) and np.array_equal(s["y"], y) and np.array_equal(s["a"], a)


def test_windows_across_launches(orc, dp, volume):
    """Iterating in launches of 2, 3, 4 and 6 iterations (each launch may open
    windows from its lists) gives the oracle's states after each launch."""
    d = volume
    inst = _inst(orc, d)
    g = dp.Dope.from_instance(d, threads=512)
    g.reset()
    y, a, mu = np.full(inst.n, 0.5), np.zeros(inst.n), d["mu0"]
    t = 0
    wins = 0
    for n in (2, 3, 4, 6):
        done, conv = g.iterate(n)
        for _ in range(done - t):
            yh, y, a, r2 = orc.admm_step(inst, mu, y, a)
            mu *= 1.05
        t = done
        s = g.get_state()
        assert np.array_equal(s["yhat"], yh) and np.array_equal(s["y"], y) and np.array_equal(s["a"], a), t
        wins += g.stats()["windows"]
        if conv:
            break
    assert wins >= 1


def test_windows_with_weak_certificates(orc, dp):
    """At mu0 = 100 with strong n-links the interval certificates fail for some
    slots: exact unaries decide at a window's first iteration, and windows end
    early; the solve still equals the plain one and the oracle's."""
    d = inputs.random_instance((512, 384), 8, (16, 16), lam=6.0, seed=21)
    w, p = _solve_pair(dp, d, threads=256, mu0=100.0)
    _assert_same(w, p)
    ref = orc.admm(_inst(orc, d), 100.0, 1.05, 1e-3, 1000)
    assert w[3] == ref["iterations"] and np.array_equal(w[1], ref["labels"])
