"""Pins of the oracle's exact solvers (BK max-flow + canonical cut, brute force,
global min-cut) against things other than themselves: hand-computed values
(Eq. 1), exhaustive enumeration, and scipy's max-flow."""
import itertools
import os

import numpy as np
import pytest

from paper_1704_03116_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    d = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        d[k] = v
    return d


def test_energy_golden_2x2(orc):
    g = _read_golden("energy_2x2.txt")
    H, W = map(int, g["grid"])
    u = np.array(list(map(float, g["u"])), np.float32)
    wq = np.array([list(map(int, g["wq_right"])), list(map(int, g["wq_down"]))], np.int32)
    inst = orc.quantise((H, W), 4, (H, W), u, wq, float(g["lambda"][0]))
    lab = np.array(list(map(int, g["labels"])), np.uint8)
    assert orc.energy(inst, lab) == int(g["E_int"][0])
    labels, e = orc.global_mincut(inst)
    assert e == int(g["min_E_int"][0])
    assert labels.tolist() == list(map(int, g["min_labels"]))


def test_quantise_round_half_even(orc):
    # U = rne(1024 u): ties go to the even integer
    u = np.array([0.5, 1.5, 2.5, -0.5], np.float32) / 1024.0
    wq = np.zeros((2, 4), np.int32)
    inst = orc.quantise((2, 2), 4, (2, 2), u, wq, 1.0)
    assert inst.U.tolist() == [0, 2, 2, 0]
    # Wl = rne(lambda * wq)
    wq = np.array([[3, 0, 5, 0], [1, 7, 0, 0]], np.int32)
    inst = orc.quantise((2, 2), 4, (2, 2), np.zeros(4, np.float32), wq, 0.5)
    assert inst.Wl.tolist() == [[2, 0, 2, 0], [0, 4, 0, 0]]


def test_quantise_rejects_bad_weights(orc):
    wq = np.array([[-1, 0, 0, 0], [0, 0, 0, 0]], np.int32)
    with pytest.raises(ValueError):
        orc.quantise((2, 2), 4, (2, 2), np.zeros(4, np.float32), wq, 1.0)
    wq = np.array([[0, 5, 0, 0], [0, 0, 0, 0]], np.int32)  # pixel 1 has no right neighbour
    with pytest.raises(ValueError):
        orc.quantise((2, 2), 4, (2, 2), np.zeros(4, np.float32), wq, 1.0)


def _enum_energies(n, c, eu, ev, cuv, cvu):
    """All 2^n energies of sum c_i y_i + sum cuv (1-y_u) y_v + cvu y_u (1-y_v)."""
    Y = np.array(list(itertools.product([0, 1], repeat=n)), np.int64)[:, ::-1]
    E = Y @ np.asarray(c, np.int64)
    yu, yv = Y[:, eu], Y[:, ev]
    E += ((1 - yu) * yv) @ np.asarray(cuv, np.int64) + (yu * (1 - yv)) @ np.asarray(cvu, np.int64)
    return Y, E


@pytest.mark.parametrize("seed", range(40))
def test_bk_canonical_cut_vs_enumeration(orc, seed):
    """BK's residual-BFS cut is a minimiser and equals the AND of all minimisers
    (the pointwise-minimal one), on random graphs with asymmetric capacities."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 13))
    m = int(rng.integers(0, 3 * n))
    eu = rng.integers(0, n, m).astype(np.int32)
    ev = rng.integers(0, n, m).astype(np.int32)
    keep = eu != ev
    eu, ev = eu[keep], ev[keep]
    m = len(eu)
    cmax = int(rng.choice([1, 3, 50]))
    c = rng.integers(-cmax, cmax + 1, n)
    cuv = rng.integers(0, cmax + 1, m) * (rng.random(m) < 0.8)
    cvu = rng.integers(0, cmax + 1, m) * (rng.random(m) < 0.8)
    lab = orc.bk_mincut(n, c, eu, ev, cuv, cvu)
    Y, E = _enum_energies(n, c, eu, ev, cuv, cvu)
    emin = E.min()
    mins = Y[E == emin]
    e_lab = E[int((lab.astype(np.int64) << np.arange(n)).sum())]
    assert e_lab == emin
    assert lab.tolist() == mins.min(axis=0).tolist()


@pytest.mark.parametrize("seed", range(6))
def test_bk_flow_value_vs_scipy(orc, seed):
    """Min-cut value of the BK labels equals scipy's max-flow value (max-flow /
    min-cut theorem) on larger random graphs."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_flow
    rng = np.random.default_rng(100 + seed)
    n = 300
    m = 1200
    eu = rng.integers(0, n, m).astype(np.int32)
    ev = rng.integers(0, n, m).astype(np.int32)
    keep = eu != ev
    eu, ev = eu[keep], ev[keep]
    m = len(eu)
    c = rng.integers(-1000, 1001, n)
    cuv = rng.integers(0, 700, m)
    cvu = rng.integers(0, 700, m)
    lab = orc.bk_mincut(n, c, eu, ev, cuv, cvu).astype(np.int64)
    # cut value of the labelling in the s-t graph: s = n, t = n + 1
    cut = (np.where(c > 0, c, 0) * lab).sum() + (np.where(c < 0, -c, 0) * (1 - lab)).sum()
    cut += (cuv * (1 - lab[eu]) * lab[ev]).sum() + (cvu * lab[eu] * (1 - lab[ev])).sum()
    s, t = n, n + 1
    rows, cols, caps = [], [], []
    for i in range(n):
        if c[i] > 0:
            rows.append(s); cols.append(i); caps.append(c[i])
        elif c[i] < 0:
            rows.append(i); cols.append(t); caps.append(-c[i])
    rows += list(eu) + list(ev)
    cols += list(ev) + list(eu)
    caps += list(cuv) + list(cvu)
    A = csr_matrix((np.array(caps, np.int32), (rows, cols)), shape=(n + 2, n + 2))
    A.sum_duplicates()
    flow = maximum_flow(A, s, t).flow_value
    assert cut == flow


@pytest.mark.parametrize("shape,conn", [((4, 5), 4), ((4, 5), 8), ((2, 3, 3), 6), ((3, 6), 8)])
@pytest.mark.parametrize("seed", range(5))
def test_global_mincut_vs_bruteforce(orc, shape, conn, seed):
    """sGC on <= 20 pixels: BK energy == enumeration minimum, labels == AND of minimisers."""
    d = inputs.random_instance(shape, conn, shape, lam=1.5, seed=seed, u_scale=1.0)
    inst = orc.quantise(d["grid"], conn, d["block"], d["u"], d["wq"], d["lam"])
    labels, e = orc.global_mincut(inst)
    eu, ev, w = orc.grid_edges(inst)
    emin, and_lab, or_lab, cnt = orc.bruteforce(inst.n, inst.U, eu, ev, w)
    assert e == emin
    assert orc.energy(inst, labels) == e
    assert labels.tolist() == and_lab.tolist()


def test_bruteforce_handles_non_submodular(orc):
    """The enumeration itself: a 2-node frustrated pair (negative w) by hand:
    E = 0*y0 + 0*y1 - 5 |y0 - y1| has minimisers 01 and 10, E = -5."""
    emin, a, o, cnt = orc.bruteforce(2, np.array([0, 0]), np.array([0], np.int32),
                                     np.array([1], np.int32), np.array([-5]))
    assert (emin, cnt) == (-5, 2)
    assert a.tolist() == [0, 0] and o.tolist() == [1, 1]


def test_global_mincut_vs_scipy_grid(orc):
    """sGC energy on a 48x48 8-connected grid equals scipy's max-flow value + the
    constant of the terminal reparametrisation."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_flow
    d = inputs.random_instance((48, 48), 8, (16, 16), lam=2.0, seed=7)
    inst = orc.quantise(d["grid"], 8, d["block"], d["u"], d["wq"], d["lam"])
    labels, e = orc.global_mincut(inst)
    eu, ev, w = orc.grid_edges(inst)
    n = inst.n
    s, t = n, n + 1
    U = inst.U
    rows = [s if U[i] > 0 else i for i in range(n) if U[i] != 0]
    cols = [i if U[i] > 0 else t for i in range(n) if U[i] != 0]
    caps = [abs(int(U[i])) for i in range(n) if U[i] != 0]
    rows += list(eu) + list(ev)
    cols += list(ev) + list(eu)
    caps += list(w) + list(w)
    A = csr_matrix((np.array(caps, np.int32), (rows, cols)), shape=(n + 2, n + 2))
    A.sum_duplicates()
    flow = maximum_flow(A, s, t).flow_value
    # E_int(y) = sum U y + cut = (cut value) + sum_{U<0} U
    assert e == flow + int(U[U < 0].sum())
