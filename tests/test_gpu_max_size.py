"""GPU: a solve at the top of the size range, checked by a property that holds
at any size (the oracle cannot run it).

A 23552 x 23552 grid with 8 neighbours: N = 554.7 M pixels, so the weight
array (conn/2 * N = 2.2 G entries) needs 64-bit offsets everywhere.  Every
unary dominates the pixel's n-links (|U_i| = 1024 > 8 * 64 = the sum of its
Wl), so flipping any pixel away from sign(u) raises the energy whatever its
neighbours: every minimiser of Eq. 1, and of every block sub-problem of Eq. 8
at iteration 1, is the threshold y_i = [u_i < 0], and the multipliers keep it
(their shift 1024 mu (a_i - y_i + 1/2) pushes each label towards its value).
The test checks those labels everywhere and the energy against its closed
form in int64.  The label pattern is 40 x 40 squares offset from the 32 x 32
blocks, so label boundaries cross block boundaries (the Eq. 10 cross terms
are not zero).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIDE = 23552          # 736 blocks of 32 per side
W_Q = 64              # wq; lambda 1 -> Wl = 64


@pytest.fixture(scope="module")
def dp():
    from paper_1704_03116_gb300 import _build
    _build.build()
    from paper_1704_03116_gb300 import dope
    return dope


def test_solve_at_maximum_size(dp):
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < 40 << 30:
        pytest.skip("needs 40 GB of free device memory")
    H = W = SIDE
    N = H * W
    # u = -1 on 40x40 squares (every other one, offset by 7 pixels), +1 elsewhere
    yy = ((np.arange(H) + 7) // 40) & 1
    xx = ((np.arange(W) + 7) // 40) & 1
    fg_rows = torch.from_numpy(yy.astype(np.bool_)).cuda()
    fg_cols = torch.from_numpy(xx.astype(np.bool_)).cuda()
    fg = (fg_rows[:, None] ^ fg_cols[None, :]).reshape(-1)          # device, N bools
    u = torch.where(fg, torch.tensor(-1.0, device="cuda"), torch.tensor(1.0, device="cuda"))
    wq = torch.full((4, H, W), W_Q, dtype=torch.int32, device="cuda")
    wq[0, :, -1] = 0                      # (0,+1)
    wq[1, -1, :] = 0                      # (+1,0)
    wq[2, -1, :] = 0
    wq[2, :, -1] = 0                      # (+1,+1)
    wq[3, -1, :] = 0
    wq[3, :, 0] = 0                       # (+1,-1)
    wq = wq.reshape(4, N)
    g = dp.Dope((H, W), 8, (32, 32), 1.0, max_iter=400)
    g.set_unaries(u)
    g.set_weights(wq)
    del wq
    lab = torch.empty(N, dtype=torch.uint8, device="cuda")
    _, E, it = g.solve(lab)
    st = g.stats()
    g.close()
    assert st["converged"] == 1 and it > 1
    want = fg.to(torch.uint8)
    assert torch.equal(lab, want)
    # E_int = sum U_i y_i + sum over undirected edges Wl |y_i - y_j|
    L = want.reshape(H, W).to(torch.int16)
    cut = (int((L[:, 1:] != L[:, :-1]).sum()) + int((L[1:, :] != L[:-1, :]).sum()) +
           int((L[1:, 1:] != L[:-1, :-1]).sum()) + int((L[1:, :-1] != L[:-1, 1:]).sum()))
    e_int = -1024 * int(want.sum()) + W_Q * cut
    assert E * 1024 == e_int
