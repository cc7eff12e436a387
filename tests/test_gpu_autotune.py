"""GPU: the autotuner.  Settings other than the block shape change speed
only, so every candidate with the starting block shape must reproduce the
default solve's labels energy and iteration count exactly; block-shape
candidates must tile the grid and their results must equal a plain solve
with that shape."""
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


def _solve(dp, d, block, **kw):
    g = dp.Dope(d["grid"], d["conn"], block, d["lam"], mu0=d["mu0"], **kw)
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    lab, e, it = g.solve(allow_notconv=True)
    g.close()
    return lab, e, it


def test_autotune_settings_keep_results(dp):
    d = inputs.ellipses_rgb(lam=4.0)
    best, tried = dp.dope_autotune(d["grid"], d["conn"], d["block"], d["lam"], d["u"], d["wq"], reps=1)
    lab0, e0, it0 = _solve(dp, d, d["block"])
    assert len(tried) >= 10
    for r in tried:
        assert r["status"] == 0 and r["ms"] > 0
        assert r["block"] == tuple(d["block"])
        assert r["energy_int"] == round(e0 * 1024) and r["iterations"] == it0
    assert best["ms"] == min(r["ms"] for r in tried)
    p = best["params"]
    lab, e, it = _solve(dp, d, best["block"], relabel_period=p.relabel_period, threads=p.threads,
                        fold_rounds=p.fold_rounds, launch_mode=p.launch_mode)
    assert np.array_equal(lab, lab0) and it == it0


def test_autotune_block_shapes(dp):
    d = inputs.random_instance((96, 128), 4, (16, 16), lam=2.0, seed=21)
    best, tried = dp.dope_autotune(d["grid"], d["conn"], d["block"], d["lam"], d["u"], d["wq"],
                                   flags=dp.DOPE_TUNE_BLOCK, reps=1)
    shapes = {r["block"] for r in tried}
    assert len(shapes) > 3
    for (by, bx) in shapes:
        assert 96 % by == 0 and 128 % bx == 0
    for r in tried[:6]:
        if r["params"].relabel_period or r["params"].threads:
            continue
        lab, e, it = _solve(dp, d, r["block"])
        assert r["energy_int"] == round(e * 1024) and r["iterations"] == it
    assert best["converged"] and best["ms"] == min(r["ms"] for r in tried if r["converged"])
