"""GPU: bounded device waits and loops run out cleanly.

Every wait and loop in the kernels has a bound; when it is reached, the kernel
writes DOPE_ETIMEOUT into the context's status word and its CTAs leave. No
trap and no hang: the call returns the status, and the device and the
context stay usable. These tests make the bounds run out on purpose, without
faulting anything:
  * a grid-barrier wait limited to 1 us. The blocks' first cuts take
    different times (5 to 60 us on this image), so the CTAs that arrive first
    give up.
  * a push-relabel bound of one pulse on blocks that need more.
After each, a default context solves the same image and matches the oracle.
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
def ell():
    return inputs.ellipses_rgb(lam=16.0)


@pytest.fixture(scope="module")
def ref(ell):
    import oracle
    q = oracle.quantise(ell["grid"], ell["conn"], ell["block"], ell["u"], ell["wq"], 16.0)
    return oracle.admm(q, ell["mu0"])


def _check_default_solve(dp, ell, ref):
    g = dp.Dope(ell["grid"], ell["conn"], ell["block"], 16.0, mu0=ell["mu0"])
    g.set_inputs(ell["u"], ell["wq"])
    lab, E, it = g.solve()
    g.close()
    assert it == ref["iterations"] and E * 1024 == ref["energy"] and np.array_equal(lab, ref["labels"])


def test_barrier_wait_runs_out(dp, ell, ref):
    g = dp.Dope(ell["grid"], ell["conn"], ell["block"], 16.0, mu0=ell["mu0"], barrier_timeout_us=1)
    g.set_inputs(ell["u"], ell["wq"])
    for _ in range(2):                                   # the next solve starts from a clean control block
        with pytest.raises(dp.DopeError) as ei:
            g.solve()
        assert ei.value.status == dp.DOPE_ETIMEOUT
    g.close()
    _check_default_solve(dp, ell, ref)


def test_pulse_bound_runs_out(dp, ell, ref):
    g = dp.Dope(ell["grid"], ell["conn"], ell["block"], 16.0, mu0=ell["mu0"], max_pulses=1)
    g.set_inputs(ell["u"], ell["wq"])
    with pytest.raises(dp.DopeError) as ei:
        g.solve()
    assert ei.value.status == dp.DOPE_ETIMEOUT
    g.close()
    _check_default_solve(dp, ell, ref)
