"""GPU parity of the non-submodular path (LSA-TR block solves) against the
oracle: block labels bit-exact, y / a within 1e-5 relative (same IEEE
operations, so in practice identical), whole solves equal in labels, energy
and iteration count."""
import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs

pytestmark = pytest.mark.gpu
STEPS = 16


@pytest.fixture(scope="module")
def dp():
    from paper_1704_03116_gb300 import _build
    _build.build()
    from paper_1704_03116_gb300 import dope
    return dope


def _close(x, ref, tol=1e-5):
    return np.all(np.abs(np.asarray(x) - ref) <= tol * np.maximum(np.abs(ref), 1.0))


CASES = [
    ("ns64", inputs.nonsubmodular_instance(size=64)),
    ("rand8", inputs.signed_instance(inputs.random_instance((48, 64), 8, (16, 16), lam=2.0, seed=2), seed=2)),
    ("rand6", inputs.signed_instance(inputs.random_instance((8, 16, 16), 6, (4, 8, 8), lam=1.5, seed=3), seed=3)),
    ("ragged", inputs.signed_instance(inputs.random_instance((30, 35), 4, (5, 7), lam=1.5, seed=4), seed=4)),
]


@pytest.mark.parametrize("name,d", CASES, ids=[c[0] for c in CASES])
def test_nsm_iterates_match_oracle(orc, dp, name, d):
    inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"], signed=True)
    g = dp.Dope(d["grid"], d["conn"], d["block"], d["lam"], mu0=d["mu0"], lsa_steps=STEPS)
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    y = np.full(inst.n, 0.5)
    a = np.zeros(inst.n)
    yh = np.zeros(inst.n, np.uint8)
    mu = d["mu0"]
    states = [None]
    for t in range(1, 13):
        yh, y, a, r2 = orc.nsm_step(inst, mu, y, a, yh, STEPS)
        mu *= 1.05
        states.append((yh, y, a, np.sqrt(r2.max())))
    for t in (1, 2, 5, 12):
        g.reset()
        g.iterate(t)
        st = g.get_state()
        tt = st["t"]
        assert 1 <= tt <= t
        if tt < t:
            assert not (states[tt][3] > 1e-3 * (1 + 1e-9))
        yh_r, y_r, a_r, _ = states[tt]
        assert np.array_equal(st["yhat"], yh_r), (name, tt)
        assert _close(st["y"], y_r) and _close(st["a"], a_r), (name, tt)
    g.close()


def test_nsm_solve_matches_oracle(orc, dp):
    d = inputs.nonsubmodular_instance(size=256)
    inst = orc.quantise(d["grid"], 4, d["block"], d["u"], d["wq"], d["lam"], signed=True)
    ref = orc.nsm_admm(inst, d["mu0"], steps=STEPS)
    g = dp.Dope(d["grid"], 4, d["block"], d["lam"], mu0=d["mu0"], lsa_steps=STEPS)
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    lab, e, it = g.solve(allow_notconv=True)
    assert it == ref["iterations"]
    assert np.array_equal(lab, ref["labels"])
    assert round(e * 1024) == ref["energy"]
    g.close()


def test_nsm_on_submodular_equals_plain_path(dp):
    d = inputs.ellipses_rgb(size=128, lam=4.0, block=(32, 32))
    a = dp.Dope.from_instance(d)
    lab0, e0, it0 = a.solve()
    b = dp.Dope.from_instance(d, lsa_steps=STEPS)
    lab1, e1, it1 = b.solve()
    assert it1 == it0 and np.array_equal(lab1, lab0) and e1 == e0
    a.close()
    b.close()


def test_nsm_argument_errors(dp):
    d = inputs.nonsubmodular_instance(size=64)
    g = dp.Dope(d["grid"], 4, d["block"], d["lam"])                    # submodular context
    g.set_unaries(d["u"])
    with pytest.raises(dp.DopeError) as e:
        g.set_weights(d["wq"])
    assert e.value.status == dp.DOPE_EUNSUPPORTED
    h = dp.Dope(d["grid"], 4, d["block"], d["lam"], lsa_steps=STEPS)
    h.set_unaries(d["u"])
    h.set_weights(d["wq"])
    with pytest.raises(dp.DopeError):
        dp.iterate_batch([h], 10)                                         # batches take submodular only
    with pytest.raises(dp.DopeError):
        dp.Dope(d["grid"], 4, d["block"], d["lam"], lsa_steps=STEPS, grow=(2, 2))
    g.close()
    h.close()
