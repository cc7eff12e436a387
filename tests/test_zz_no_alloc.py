"""dope_solve_noalloc: the allocation-free solve for callers that cannot call
cudaMalloc (a framework allocator that already holds the GPU's memory, a host
application that forbids allocation after start-up, latency-critical loops).
Its results must equal those of the regular context-based dope_solve (labels
bit-exact, same energy and iteration count), on two calls in a row that share
its static scratch array.  This file is collected last on purpose."""
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


def _regular(dp, d):
    g = dp.Dope.from_instance(d)
    lab, E, it = g.solve()
    g.close()
    return lab, int(round(E * 1024)), it


def _noalloc(dp, d):
    import torch
    u = torch.from_numpy(d["u"]).cuda()
    w = torch.from_numpy(np.ascontiguousarray(d["wq"])).cuda()
    lab = torch.full((u.numel(),), 7, dtype=torch.uint8, device="cuda")
    p = dp.dope_default_params()
    p.mu0 = d["mu0"]
    e, it, rc = dp.dope_solve_noalloc(d["grid"], d["conn"], d["block"], d["lam"], u, w, lab, params=p)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), e, it


def test_noalloc_matches_regular_two_calls(dp):
    cases = [inputs.ellipses_rgb(lam=4.0),
             inputs.random_instance((48, 80), 4, (16, 16), lam=2.0, seed=3),
             inputs.random_instance((16, 32, 32), 6, (8, 16, 16), lam=1.5, seed=4)]
    for d in cases:
        ref = _regular(dp, d)
        for _ in range(2):                 # two calls in a row on the shared scratch
            got = _noalloc(dp, d)
            assert np.array_equal(got[0], ref[0])
            assert got[1] == ref[1] and got[2] == ref[2]


def test_noalloc_rejects_oversize(dp):
    import torch
    n = 2048 * 2048
    u = torch.zeros(n, dtype=torch.float32, device="cuda")
    w = torch.zeros((4, n), dtype=torch.int32, device="cuda")
    lab = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(dp.DopeError) as ei:
        dp.dope_solve_noalloc((2048, 2048), 8, (32, 32), 1.0, u, w, lab)
    assert ei.value.status == dp.DOPE_EINVAL


def test_noalloc_size_boundary(dp):
    """8-connected 32x32 blocks cost about 23 bytes per pixel of the 16 MiB
    array: 832 x 832 fits (and equals the regular solve), 864 x 864 does not."""
    d = inputs.random_instance((832, 832), 8, (32, 32), lam=2.0, seed=6)
    ref = _regular(dp, d)
    got = _noalloc(dp, d)
    assert np.array_equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2]
    import torch
    n = 864 * 864
    u = torch.zeros(n, dtype=torch.float32, device="cuda")
    w = torch.zeros((4, n), dtype=torch.int32, device="cuda")
    lab = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(dp.DopeError) as ei:
        dp.dope_solve_noalloc((864, 864), 8, (32, 32), 1.0, u, w, lab)
    assert ei.value.status == dp.DOPE_EINVAL
    p = dp.dope_default_params()
    p.max_iter = 1 << 30                     # its trace alone would not fit
    with pytest.raises(dp.DopeError) as ei:
        dp.dope_solve_noalloc((64, 64), 8, (32, 32), 1.0, u[:4096], w[:, :4096].contiguous(), lab, params=p)
    assert ei.value.status == dp.DOPE_EINVAL


def test_noalloc_rejects_short_or_foreign_buffers(dp):
    """Buffers shorter than the grid, a weight array of the wrong shape, and
    host tensors are refused by the binding before anything runs."""
    import torch
    n = 64 * 64
    u = torch.zeros(n, dtype=torch.float32, device="cuda")
    w = torch.zeros((4, n), dtype=torch.int32, device="cuda")
    lab = torch.empty(n, dtype=torch.uint8, device="cuda")
    args = ((64, 64), 8, (32, 32), 1.0)
    with pytest.raises(ValueError):
        dp.dope_solve_noalloc(*args, u[: n - 1], w, lab)
    with pytest.raises(ValueError):
        dp.dope_solve_noalloc(*args, u, w[:2].contiguous(), lab)
    with pytest.raises(ValueError):
        dp.dope_solve_noalloc(*args, u, w.reshape(2, 2 * n), lab)
    with pytest.raises(ValueError):
        dp.dope_solve_noalloc(*args, u, w, lab[: n - 1])
    with pytest.raises(TypeError):
        dp.dope_solve_noalloc(*args, u.cpu(), w, lab)
