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
