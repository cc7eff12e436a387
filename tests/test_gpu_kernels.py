"""GPU parity of the larger kernels (Section 3: 5x5, 7x7, 9x9 squares, the
radius-2 ball) against the oracle: the iterates after a fixed number of
iterations (block labels bit-exact, y / a within 1e-5 relative) and whole
solves (labels, energy, iteration count)."""
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


def _close(x, ref, tol=1e-5):
    return np.all(np.abs(np.asarray(x) - ref) <= tol * np.maximum(np.abs(ref), 1.0))


CASES = [
    ("k5", 24, (48, 64), (16, 16), (0, 0)),
    ("k5_grow", 24, (48, 64), (16, 16), (2, 2)),
    ("k7", 48, (40, 48), (8, 8), (0, 0)),
    ("k9", 80, (36, 36), (12, 12), (0, 0)),
    ("ball2", 32, (8, 16, 16), (4, 8, 8), (0, 0, 0)),
    ("k5_ragged", 24, (30, 35), (5, 7), (1, 2)),
]


@pytest.mark.parametrize("name,conn,grid,block,grow", CASES, ids=[c[0] for c in CASES])
def test_big_kernel_iterates_match_oracle(orc, dp, name, conn, grid, block, grow):
    d = inputs.random_instance(grid, conn, block, lam=1.0, seed=conn)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    g3 = grow if len(grow) == 3 else (0,) + tuple(grow)
    ov = orc.Overlap(inst, g3)
    g = dp.Dope(d["grid"], conn, d["block"], d["lam"], mu0=d["mu0"], grow=grow if any(grow) else None)
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    y = np.full(inst.n, 0.5)
    a = np.zeros(ov.K * ov.eb)
    mu = d["mu0"]
    states = [None]
    for t in range(1, 9):
        yh, y, a, r2 = ov.step(mu, y, a)
        mu *= 1.05
        states.append((yh, y, a, np.sqrt(r2.max())))
    for t in (1, 3, 8):
        g.reset()
        g.iterate(t)
        st = g.get_state()
        ga, gyh = g.block_state()
        tt = st["t"]
        assert 1 <= tt <= t
        if tt < t:
            assert not (states[tt][3] > 1e-3 * (1 + 1e-9))
        yh, y_r, a_r, _ = states[tt]
        assert np.array_equal(gyh, yh), (name, tt)
        assert _close(st["y"], y_r) and _close(ga, a_r), (name, tt)
    g.close()


@pytest.mark.parametrize("conn,block", [(24, (32, 32)), (48, (16, 16))])
def test_big_kernel_solve_matches_oracle(orc, dp, conn, block):
    d = inputs.ellipses_rgb(size=128, lam=1.0, block=block, conn=conn)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    ref = orc.admm(inst, d["mu0"])
    g = dp.Dope(d["grid"], conn, d["block"], d["lam"], mu0=d["mu0"])
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    lab, e, it = g.solve(allow_notconv=True)
    assert it == ref["iterations"]
    assert np.array_equal(lab, ref["labels"]) and round(e * 1024) == ref["energy"]
    g.close()


def test_big_kernel_argument_errors(dp):
    with pytest.raises(dp.DopeError):
        dp.Dope((8, 8, 8), 24, (4, 4, 4), 1.0)          # 24 is a 2-D kernel
    with pytest.raises(dp.DopeError):
        dp.Dope((64, 64), 80, (32, 32), 1.0)            # 81-node kernels on 1024-node blocks: too much shared memory
    with pytest.raises(dp.DopeError):
        dp.Dope((64, 64), 12, (16, 16), 1.0)            # no such kernel
