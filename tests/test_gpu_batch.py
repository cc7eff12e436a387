"""GPU: the batched launch (dope_iterate_batch) against the single-problem path
and the oracle.

Each problem in a batch runs its own Algorithm 1 with the per-block
arithmetic of the single-problem kernels, so its iterates must be
bit-identical to solving it alone: labels, iteration count, energy and the
y / a state are compared for exact equality.  Small members are also checked
against the oracle with the parity bars of test_gpu_parity.
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


def _mix():
    """Problems of different grids, connectivities, block shapes and lambdas."""
    out = [inputs.disk64()]
    for lam in (1.0, 4.0, 16.0):
        out.append(inputs.ellipses_rgb(lam=lam))
    out.append(inputs.random_instance((96, 80), 4, (16, 16), lam=2.0, seed=3))
    out.append(inputs.random_instance((40, 48), 8, (8, 8), lam=3.0, seed=4))
    out.append(inputs.random_instance((16, 16, 16), 6, (8, 8, 4), lam=2.5, seed=5))
    out.append(inputs.random_instance((32, 32), 4, (32, 32), lam=1.0, seed=6))      # one block
    out.append(inputs.random_instance((50, 80), 8, (25, 40), lam=2.0, seed=7))      # 1000-node blocks
    return out


def _alone(dp, d, **kw):
    g = dp.Dope.from_instance(d, **kw)
    lab, e, it = g.solve(allow_notconv=True)
    st = g.get_state()
    g.close()
    return lab, e, it, st["y"], st["a"]


@pytest.fixture(scope="module")
def mix_alone(dp):
    mix = _mix()
    return mix, [_alone(dp, d) for d in mix]


def test_batch_equals_alone(dp, mix_alone):
    mix, alone = mix_alone
    gs = [dp.Dope.from_instance(d) for d in mix]
    res = dp.iterate_batch(gs, 1000)
    for d, g, (it, conv, st), (lab0, e0, it0, y0, a0) in zip(mix, gs, res, alone):
        assert st == 0 and conv
        assert it == it0, d["name"]
        lab, e = g.labels()
        assert np.array_equal(lab, lab0), d["name"]
        assert e / 1024.0 == e0
        st = g.get_state()
        assert np.array_equal(st["y"], y0) and np.array_equal(st["a"], a0)
        assert st["t"] == it0
        g.close()


def test_batch_in_short_launches(dp, mix_alone):
    """Launches of 3 iterations at a time, resumed from the contexts' state."""
    mix, alone = mix_alone
    gs = [dp.Dope.from_instance(d) for d in mix]
    live = list(range(len(gs)))
    rounds = 0
    while live:
        res = dp.iterate_batch([gs[i] for i in live], 3)
        live = [i for i, (it, conv, st) in zip(live, res) if not conv]
        rounds += 1
        assert rounds < 400
    for d, g, (lab0, e0, it0, y0, a0) in zip(mix, gs, alone):
        lab, e = g.labels()
        assert g.stats()["iterations"] == it0
        assert np.array_equal(lab, lab0), d["name"]
        g.close()


def test_batch_subsets_and_order(dp, mix_alone):
    """A problem's result does not depend on its companions or its position."""
    mix, alone = mix_alone
    idx = [8, 2, 5, 0]
    gs = [dp.Dope.from_instance(mix[i]) for i in idx]
    dp.iterate_batch(gs, 1000)
    for i, g in zip(idx, gs):
        lab, e = g.labels()
        assert np.array_equal(lab, alone[i][0])
        g.close()
    g = dp.Dope.from_instance(mix[3])
    (it, conv, st), = dp.iterate_batch([g], 1000)
    assert it == alone[3][2] and np.array_equal(g.labels()[0], alone[3][0])
    g.close()


def test_batch_vs_oracle(orc, dp):
    ds = [inputs.random_instance((48, 40), 8, (8, 8), lam=3.0, seed=11),
          inputs.random_instance((30, 35), 4, (5, 7), lam=1.5, seed=12),
          inputs.random_instance((12, 18, 20), 6, (4, 6, 5), lam=1.0, seed=13),
          inputs.disk64()]
    gs = [dp.Dope.from_instance(d) for d in ds]
    res = dp.iterate_batch(gs, 1000)
    for d, g, (it, conv, st) in zip(ds, gs, res):
        inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
        ref = orc.admm(inst, d["mu0"])
        lab, e = g.labels()
        assert it == ref["iterations"]
        assert np.array_equal(lab, ref["labels"])
        assert e == ref["energy"]
        st = g.get_state()
        y, a = st["y"], st["a"]
        assert np.all(np.abs(y - ref["y"]) <= 1e-5 * np.maximum(np.abs(ref["y"]), 1.0))
        assert np.all(np.abs(a - ref["a"]) <= 1e-5 * np.maximum(np.abs(ref["a"]), 1.0))
        g.close()


def test_batch_max_iter_and_mixed_params(dp):
    """max_iter reached before convergence; per-problem mu0 / eps honoured."""
    d1 = inputs.ellipses_rgb(lam=4.0)
    d2 = inputs.disk64()
    alone1 = dp.Dope.from_instance(d1, max_iter=3)
    lab1, e1, it1 = alone1.solve(allow_notconv=True)
    alone1.close()
    alone2 = dp.Dope.from_instance(d2, eps=1e-6, mu0=50.0)
    lab2, e2, it2 = alone2.solve(allow_notconv=True)
    alone2.close()
    g1 = dp.Dope.from_instance(d1, max_iter=3)
    g2 = dp.Dope.from_instance(d2, eps=1e-6, mu0=50.0)
    (ia, ca, sa), (ib, cb, sb) = dp.iterate_batch([g1, g2], 1000)
    assert ia == 3 == it1 and not ca
    assert ib == it2
    assert np.array_equal(g1.labels()[0], lab1) and np.array_equal(g2.labels()[0], lab2)
    g1.close()
    g2.close()


def test_batch_argument_errors(dp):
    d = inputs.disk64()
    g = dp.Dope.from_instance(d)
    with pytest.raises(dp.DopeError) as e:
        dp.iterate_batch([g, g], 10)
    assert e.value.status == dp.DOPE_EINVAL
    h = dp.Dope(d["grid"], d["conn"], d["block"], d["lam"])
    with pytest.raises(dp.DopeError) as e:
        dp.iterate_batch([g, h], 10)          # h has no unaries / weights
    assert e.value.status == dp.DOPE_EINVAL
    with pytest.raises(dp.DopeError):
        dp.dope_iterate_batch([], 10)
    g.close()
    h.close()
