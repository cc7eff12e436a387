"""GPU: dope_set_inputs (unaries and weights in one asynchronous call) and the
asynchronous dope_set_image.

They must give exactly what the synchronising calls give, on every kind of
context (resident, persistent, launch mode 1, overlapping partition, larger
kernel, non-submodular blocks). Their errors must surface at the next
synchronising call and leave both inputs unset until new ones arrive.
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


CASES = [
    ("resident_8", (128, 96), 8, (32, 32), {}),
    ("persistent_6", (32, 128, 128), 6, (4, 16, 16), {}),        # 512 blocks: not all co-resident
    ("mode1_4", (64, 64), 4, (16, 16), {"launch_mode": 1}),
    ("overlap_8", (64, 64), 8, (16, 16), {"grow": (2, 2), "max_iter": 6}),
    ("kernel5", (48, 64), 24, (16, 16), {}),
    ("nsm_4", (64, 64), 4, (16, 16), {"lsa_steps": 8}),
]


def _instance(name, grid, conn, block):
    if name.startswith("nsm"):
        d = inputs.nonsubmodular_instance(size=grid[0], block=block)
        return d["u"].reshape(-1), d["wq"]
    d = inputs.random_instance(grid, conn, block, lam=2.0, seed=len(name))
    return d["u"], d["wq"]


@pytest.mark.parametrize("name,grid,conn,block,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("where", ["host", "device"])
def test_set_inputs_equals_separate_calls(dp, name, grid, conn, block, kw, where):
    torch = pytest.importorskip("torch")
    u, wq = _instance(name, grid, conn, block)
    if where == "device":
        u, wq = torch.from_numpy(u).cuda(), torch.from_numpy(wq).cuda()
    notconv = "grow" in kw or "lsa_steps" in kw
    a = dp.Dope(grid, conn, block, 2.0, **kw)
    a.set_unaries(u)
    a.set_weights(wq)
    la, ea, ia = a.solve(allow_notconv=notconv)
    b = dp.Dope(grid, conn, block, 2.0, **kw)
    b.set_inputs(u, wq)
    lb, eb, ib = b.solve(allow_notconv=notconv)
    assert ia == ib and ea == eb and np.array_equal(la, lb)
    # twice on the same context, inputs replaced in between
    b.set_inputs(u, wq)
    lc, ec, ic = b.solve(allow_notconv=notconv)
    assert ic == ia and ec == ea and np.array_equal(lc, la)
    a.close()
    b.close()


def test_deferred_overflow_surfaces_at_solve(dp):
    d = inputs.random_instance((64, 64), 8, (32, 32), lam=1.0, seed=3)
    g = dp.Dope((64, 64), 8, (32, 32), 1.0)
    bad = d["wq"].copy()
    bad[0, 5] = 1 << 24                                    # lambda * wq >= 2^24
    g.set_inputs(d["u"], bad)                              # no error yet: not synchronised
    with pytest.raises(dp.DopeError) as ei:
        g.solve()
    assert ei.value.status == dp.DOPE_EOVERFLOW
    with pytest.raises(dp.DopeError) as ei:                # both inputs now count as unset
        g.solve()
    assert ei.value.status == dp.DOPE_EINVAL
    g.set_inputs(d["u"], d["wq"])
    l1, e1, i1 = g.solve()
    r = dp.Dope((64, 64), 8, (32, 32), 1.0)
    r.set_unaries(d["u"])
    r.set_weights(d["wq"])
    l2, e2, i2 = r.solve()
    assert i1 == i2 and e1 == e2 and np.array_equal(l1, l2)
    g.close()
    r.close()


def test_deferred_error_reaches_other_calls(dp):
    d = inputs.random_instance((64, 64), 4, (16, 16), lam=1.0, seed=4)
    neg = d["wq"].copy()
    neg[1, 10] = -5                                        # negative weight on the submodular path
    # the iterate path reports it
    g = dp.Dope((64, 64), 4, (16, 16), 1.0, launch_mode=1)
    g.set_inputs(d["u"], neg)
    with pytest.raises(dp.DopeError) as ei:
        g.iterate(3)
    assert ei.value.status == dp.DOPE_EUNSUPPORTED
    g.close()
    # replacing only the unaries leaves the weights unset
    g = dp.Dope((64, 64), 4, (16, 16), 1.0)
    g.set_inputs(d["u"], neg)
    g.set_unaries(d["u"])
    with pytest.raises(dp.DopeError) as ei:
        g.solve()
    assert ei.value.status == dp.DOPE_EINVAL
    g.set_weights(d["wq"])
    g.solve()
    g.close()


def test_set_image_async_equals_sync(dp):
    torch = pytest.importorskip("torch")
    d = inputs.ellipses_rgb(size=128)
    img = torch.from_numpy(d["image"].reshape(-1, 3)).cuda()
    a = dp.Dope((128, 128), 8, (32, 32), 2.0)
    sig = a.set_image(img, d["gmm_fg"], d["gmm_bg"], inv_dist=True)
    la, ea, ia = a.solve()
    b = dp.Dope((128, 128), 8, (32, 32), 2.0)
    assert b.set_image(d["image"], d["gmm_fg"], d["gmm_bg"], inv_dist=True, read_sigma=False) is None
    lb, eb, ib = b.solve()
    assert sig > 0 and ia == ib and ea == eb and np.array_equal(la, lb)
    a.close()
    b.close()


@pytest.mark.parametrize("name,grid,conn,block,kw", CASES, ids=[c[0] for c in CASES])
def test_solve_begin_end_equals_solve(dp, name, grid, conn, block, kw):
    u, wq = _instance(name, grid, conn, block)
    notconv = "grow" in kw or "lsa_steps" in kw
    a = dp.Dope(grid, conn, block, 2.0, **kw)
    a.set_inputs(u, wq)
    la, ea, ia = a.solve(allow_notconv=notconv)
    a.set_inputs(u, wq)
    lab = a.solve_begin()
    lb, eb, ib = a.solve_end(allow_notconv=notconv)
    assert lb is lab and ia == ib and ea == eb and np.array_equal(la, lb)
    a.close()


def test_solves_queued_on_several_contexts(dp):
    """Several contexts begun on one stream, then ended (in reverse order):
    each result equals its own dope_solve."""
    torch = pytest.importorskip("torch")
    ds = [inputs.random_instance((96, 128), 8, (32, 32), lam=float(l), seed=l) for l in (1, 3, 9)]
    ref = []
    for d in ds:
        g = dp.Dope(d["grid"], 8, d["block"], d["lam"])
        g.set_inputs(d["u"], d["wq"])
        ref.append(g.solve())
        g.close()
    gs = [dp.Dope(d["grid"], 8, d["block"], d["lam"]) for d in ds]
    labs = [torch.zeros(96 * 128, dtype=torch.uint8).pin_memory() for _ in ds]
    for g, d, lab in zip(gs, ds, labs):
        g.set_inputs(d["u"], d["wq"])
        g.solve_begin(lab.numpy())
    out = {}
    for i in (2, 0, 1):
        out[i] = gs[i].solve_end()
    for i, (l0, e0, i0) in enumerate(ref):
        l1, e1, i1 = out[i]
        assert i0 == i1 and e0 == e1 and np.array_equal(l0, l1) and np.array_equal(labs[i].numpy(), l0)
    for g in gs:
        g.close()


def test_solve_begin_end_misuse_and_deferred_error(dp):
    d = inputs.random_instance((64, 64), 8, (32, 32), lam=1.0, seed=5)
    g = dp.Dope((64, 64), 8, (32, 32), 1.0)
    with pytest.raises(dp.DopeError) as ei:                # end without begin
        g.solve_end()
    assert ei.value.status == dp.DOPE_EINVAL
    g.set_inputs(d["u"], d["wq"])
    g.solve_begin()
    with pytest.raises(dp.DopeError) as ei:                # a second begin
        g.solve_begin()
    assert ei.value.status == dp.DOPE_EINVAL
    with pytest.raises(dp.DopeError) as ei:                # dope_solve while begun
        g.solve()
    assert ei.value.status == dp.DOPE_EINVAL
    g.solve_end()
    bad = d["wq"].copy()
    bad[2, 7] = 1 << 24
    g.set_inputs(d["u"], bad)
    g.solve_begin()                                        # issued: the error is not known yet
    with pytest.raises(dp.DopeError) as ei:
        g.solve_end()
    assert ei.value.status == dp.DOPE_EOVERFLOW
    with pytest.raises(dp.DopeError) as ei:                # inputs now unset
        g.solve_begin()
    assert ei.value.status == dp.DOPE_EINVAL
    g.close()


def test_energy_trace_matches_oracle_steps(dp):
    """The per-iteration trace (energy of yhat_t, label flips, residual)
    against the oracle stepping Algorithm 1 itself; its last labels and
    energy are the solve's."""
    import oracle
    d = inputs.random_instance((64, 96), 8, (16, 16), lam=3.0, seed=21)
    g = dp.Dope(d["grid"], 8, d["block"], d["lam"])
    g.set_inputs(d["u"], d["wq"])
    tr = g.energy_trace()
    lab, E, it = g.solve()
    g.close()
    inst = oracle.quantise(d["grid"], 8, d["block"], d["u"], d["wq"], d["lam"])
    n = inst.n
    y, a, mu = np.full(n, 0.5), np.zeros(n), 100.0
    prev = np.zeros(n, np.uint8)
    for t, (e_gpu, f_gpu, r_gpu) in enumerate(zip(tr["energy_int"], tr["flips"], tr["rmax"]), start=1):
        yhat, y, a, r2 = oracle.admm_step(inst, mu, y, a)
        mu *= 1.05
        assert e_gpu == oracle.energy(inst, yhat), t
        assert f_gpu == int(np.count_nonzero(yhat != prev)), t
        assert r_gpu == pytest.approx(float(np.sqrt(r2.max())), rel=1e-9, abs=1e-12), t
        prev = yhat
    assert len(tr["energy_int"]) == it
    assert tr["energy_int"][-1] == E * 1024 and np.array_equal(tr["labels"], lab)
