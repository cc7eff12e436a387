"""GPU: the request server (continuous batching) -- each result is the same
alone and in the mix.

"Alone" is the same request solved by itself: through the single-problem path
(a server in one-at-a-time mode, which runs dope_solve's kernels), and for
small requests also by the oracle on the padded instance.  Labels, energies
and iteration counts must be identical.
"""
import time

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


def _requests(n, seed, max_side=200):
    """Mixed requests: ragged 2-D grids (not multiples of the block), 4- or
    8-connectivity, lambda in [1, 16], 16x16 or 32x32 blocks, a few 3-D."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if i % 7 == 6:
            g = tuple(int(x) for x in rng.integers(9, 20, 3))
            d = inputs.random_instance(g, 6, (4, 8, 8), lam=float(rng.uniform(1, 4)), seed=seed * 100 + i)
        else:
            g = (int(rng.integers(20, max_side)), int(rng.integers(20, max_side)))
            conn = 4 if rng.random() < 0.5 else 8
            blk = (16, 16) if rng.random() < 0.5 else (32, 32)
            d = inputs.random_instance(g, conn, blk, lam=float(rng.uniform(1, 16)), seed=seed * 100 + i)
        out.append(d)
    return out


def _run(dp, reqs, delays=None, **kw):
    srv = dp.Server(**kw)
    labels = [np.zeros(int(np.prod(d["grid"])), np.uint8) for d in reqs]
    ids = []
    for i, d in enumerate(reqs):
        if delays is not None:
            time.sleep(delays[i])
        ids.append(srv.submit(d["grid"], d["conn"], d["block"], d["lam"], d["u"], d["wq"], labels[i], tag=i))
    res = {}
    t0 = time.time()
    while len(res) < len(reqs):
        for r in srv.poll(timeout=1.0):
            res[r["tag"]] = r
        assert time.time() - t0 < 300, "server did not finish"
    st = srv.stats()
    srv.close()
    return labels, res, st


@pytest.fixture(scope="module")
def mix():
    return _requests(24, 1)


@pytest.fixture(scope="module")
def alone(dp, mix):
    labels, res, st = _run(dp, mix, mode=1)
    return labels, res


@pytest.mark.parametrize("mode", [0, 2])
def test_server_mix_equals_alone(dp, mix, alone, mode):
    lab1, res1 = alone
    labels, res, st = _run(dp, mix, mode=mode)
    for i in range(len(mix)):
        assert res[i]["status"] == 0 and res1[i]["status"] == 0
        assert res[i]["iterations"] == res1[i]["iterations"], i
        assert res[i]["energy_int"] == res1[i]["energy_int"], i
        assert np.array_equal(labels[i], lab1[i]), i
    assert st["completed"] == len(mix)
    assert st["max_in_flight"] > 1          # requests did run together


def test_server_matches_oracle(orc, dp, mix, alone):
    lab1, res1 = alone
    for i in (0, 1, 2, 6, 13):
        d = inputs.pad_to_blocks(mix[i])
        inst = orc.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
        ref = orc.admm(inst, d["mu0"])
        assert res1[i]["iterations"] == ref["iterations"]
        assert np.array_equal(lab1[i], inputs.crop_padded(ref["labels"], d))
        assert res1[i]["energy_int"] == ref["energy"]


def test_server_staggered_arrivals(dp, mix, alone):
    """Requests arriving while others run are admitted between iterations."""
    lab1, res1 = alone
    rng = np.random.default_rng(5)
    labels, res, st = _run(dp, mix, delays=rng.exponential(0.002, len(mix)), mode=0)
    for i in range(len(mix)):
        assert res[i]["status"] == 0
        assert res[i]["iterations"] == res1[i]["iterations"]
        assert np.array_equal(labels[i], lab1[i])
        assert res[i]["t_submit"] <= res[i]["t_admit"] <= res[i]["t_done"]


def test_server_admission_by_memory(dp, mix, alone):
    """A small arena admits a few requests at a time; all still finish, same results."""
    lab1, res1 = alone
    sub = mix[:16]
    labels, res, st = _run(dp, sub, mode=0, hbm_bytes=4 << 20)
    for i in range(len(sub)):
        assert res[i]["status"] == 0
        assert np.array_equal(labels[i], lab1[i])
    assert st["bytes_peak"] <= st["bytes_limit"] == 4 << 20
    assert st["max_in_flight"] < len(sub)


def test_server_request_too_large(dp):
    d = inputs.random_instance((512, 512), 8, (32, 32), lam=2.0, seed=9)
    small = inputs.random_instance((40, 40), 4, (16, 16), lam=2.0, seed=10)
    labels, res, st = _run(dp, [d, small], mode=0, hbm_bytes=4 << 20)
    assert res[0]["status"] == dp.DOPE_ENOMEM
    assert res[1]["status"] == 0


def test_server_device_buffers(dp, mix, alone):
    torch = pytest.importorskip("torch")
    lab1, res1 = alone
    srv = dp.Server(mode=0)
    outs = []
    for i, d in enumerate(mix[:6]):
        u = torch.from_numpy(d["u"]).cuda()
        w = torch.from_numpy(d["wq"]).cuda()
        lab = torch.zeros(int(np.prod(d["grid"])), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        srv.submit(d["grid"], d["conn"], d["block"], d["lam"], u, w, lab, tag=i)
        outs.append(lab)
    got = {}
    t0 = time.time()
    while len(got) < 6:
        for r in srv.poll(timeout=1.0):
            got[r["tag"]] = r
        assert time.time() - t0 < 120
    srv.close()
    for i in range(6):
        assert got[i]["status"] == 0
        assert np.array_equal(outs[i].cpu().numpy(), lab1[i])


def test_server_rejects_bad_requests(dp):
    srv = dp.Server()
    d = inputs.disk64()
    with pytest.raises(dp.DopeError):
        srv.submit(d["grid"], 6, d["block"], d["lam"], d["u"], d["wq"], np.zeros(4096, np.uint8))
    with pytest.raises(dp.DopeError):
        srv.submit(d["grid"], 4, d["block"], -1.0, d["u"], d["wq"], np.zeros(4096, np.uint8))
    srv.close()


def _mixture(rng, K, scale):
    w = rng.uniform(0.2, 1.0, K)
    A = rng.normal(0, scale, (K, 3, 3))
    cov = A @ A.transpose(0, 2, 1) + scale * scale * np.eye(3)
    return w / w.sum(), rng.uniform(0, 1, (K, 3)), cov


def _image_requests(n, seed):
    """Ragged RGB requests (regions plus noise) with their colour models."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = (int(v) for v in rng.integers(30, 150, 2))
        img = (np.round(rng.uniform(0, 1, (H * W, 3)) * 3) / 3 + rng.normal(0, 0.05, (H * W, 3))).astype(np.float32)
        out.append({"grid": (H, W), "conn": 4 if rng.random() < 0.5 else 8,
                    "block": (16, 16) if rng.random() < 0.5 else (32, 32), "lam": float(rng.uniform(1, 8)),
                    "image": img, "fg": _mixture(rng, 3, 0.1), "bg": _mixture(rng, 2, 0.1)})
    return out


def _collect(srv, n):
    got, t0 = {}, time.time()
    while len(got) < n:
        for r in srv.poll(timeout=1.0):
            got[r["tag"]] = r
        assert time.time() - t0 < 300, "server did not finish"
    return got


def test_server_image_requests(dp):
    """Requests given as images (potentials computed by the server on the GPU)
    equal the same requests given as the potentials the standalone calls
    compute: batched and one at a time, host and device images."""
    torch = pytest.importorskip("torch")
    reqs = _image_requests(10, 5)
    for d in reqs:
        img = torch.from_numpy(d["image"]).cuda()
        d["u"] = dp.dope_gmm_unaries(img, d["fg"], d["bg"], clip=50.0).cpu().numpy()
        d["wq"] = dp.dope_contrast_weights(img, d["grid"], d["conn"], channels=3, inv_dist=True)[0].cpu().numpy()
    ref_lab, ref_res, _ = _run(dp, reqs, mode=0)
    for mode, on_dev in ((0, False), (1, False), (0, True)):
        srv = dp.Server(mode=mode)
        labs = []
        for i, d in enumerate(reqs):
            n = int(np.prod(d["grid"]))
            if on_dev:
                lab = torch.zeros(n, dtype=torch.uint8, device="cuda")
                im = torch.from_numpy(d["image"]).cuda()
                torch.cuda.synchronize()
            else:
                lab, im = np.zeros(n, np.uint8), d["image"]
            srv.submit_image(d["grid"], d["conn"], d["block"], d["lam"], im, d["fg"], d["bg"], lab, clip=50.0,
                             inv_dist=True, tag=i)
            labs.append(lab)
        got = _collect(srv, len(reqs))
        srv.close()
        for i in range(len(reqs)):
            got_lab = labs[i].cpu().numpy() if on_dev else labs[i]
            assert got[i]["status"] == ref_res[i]["status"] == 0
            assert got[i]["energy_int"] == ref_res[i]["energy_int"]
            assert got[i]["iterations"] == ref_res[i]["iterations"]
            assert np.array_equal(got_lab, ref_lab[i]), (mode, on_dev, i)


def test_server_image_request_bad_model(dp):
    """A covariance that is not positive definite fails that request alone."""
    reqs = _image_requests(3, 9)
    srv = dp.Server(mode=0)
    bad = (np.array([1.0]), np.array([[0.5, 0.5, 0.5]]), np.array([np.diag([0.01, -0.01, 0.01])]))
    labs = [np.zeros(int(np.prod(d["grid"])), np.uint8) for d in reqs]
    for i, d in enumerate(reqs):
        srv.submit_image(d["grid"], d["conn"], d["block"], d["lam"], d["image"], bad if i == 1 else d["fg"], d["bg"],
                         labs[i], clip=50.0, inv_dist=True, tag=i)
    got = _collect(srv, 3)
    srv.close()
    assert got[1]["status"] == dp.DOPE_EINVAL
    assert got[0]["status"] == 0 and got[2]["status"] == 0


def test_server_cancel_queued_and_running(dp):
    """A queued request and one inside a running launch are both cancelled
    (status DOPE_ECANCELED); the request beside them finishes with the
    result it has alone; afterwards the arena holds only the cached tables."""
    big = inputs.random_instance((1536, 1536), 8, (32, 32), lam=6.0, seed=11)
    small = inputs.random_instance((256, 320), 4, (16, 16), lam=3.0, seed=12)
    # alone (one at a time)
    lab_small_alone = np.zeros(256 * 320, np.uint8)
    srv = dp.Server(mode=1)
    srv.submit(small["grid"], 4, small["block"], small["lam"], small["u"], small["wq"], lab_small_alone, tag=0)
    alone = _collect(srv, 1)[0]
    srv.close()
    # one batched iteration per launch, so the big request runs for many launches
    srv = dp.Server(mode=0, launch_iters=1)
    labs = [np.zeros(1536 * 1536, np.uint8), np.zeros(256 * 320, np.uint8), np.zeros(1536 * 1536, np.uint8)]
    id_big = srv.submit(big["grid"], 8, big["block"], big["lam"], big["u"], big["wq"], labs[0], tag=0)
    srv.submit(small["grid"], 4, small["block"], small["lam"], small["u"], small["wq"], labs[1], tag=1)
    t0 = time.time()
    while srv.stats()["in_flight"] < 2 and time.time() - t0 < 30:
        time.sleep(0.001)
    time.sleep(0.003)
    srv.cancel(id_big)                                   # running
    got = _collect(srv, 2)
    assert got[0]["status"] == dp.DOPE_ECANCELED
    assert got[1]["status"] == alone["status"] == 0
    assert got[1]["energy_int"] == alone["energy_int"] and got[1]["iterations"] == alone["iterations"]
    assert np.array_equal(labs[1], lab_small_alone)
    st = srv.stats()
    assert st["bytes_in_use"] < (1 << 20)                # only the shared face / halo tables stay
    srv.close()
    # queued: an arena that holds one big request at a time
    srv = dp.Server(mode=0, hbm_bytes=128 << 20, launch_iters=1)        # ~105 MB per request in set-up
    ids = [srv.submit(big["grid"], 8, big["block"], big["lam"], big["u"], big["wq"], labs[i % 2 * 2], tag=i)
           for i in range(2)]
    srv.cancel(ids[1])                                   # still waiting for memory
    with pytest.raises(dp.DopeError):
        srv.cancel(10 ** 9)                              # never issued
    got = _collect(srv, 2)
    assert got[1]["status"] == dp.DOPE_ECANCELED
    assert got[0]["status"] == 0
    srv.close()
