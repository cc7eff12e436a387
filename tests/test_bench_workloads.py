"""bench.py's workload table builds consistent instances (shapes, dtypes and
the keys its timed loops read), checked on CPU so that a GPU run cannot fail
on a malformed configuration."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("name", ["disk64", "ellipses512", "ellipses512_size10", "ellipses512_k5",
                                  "nonsubmodular1024"])
def test_workload_instances_are_consistent(name):
    import bench
    insts, cfg = bench.workload(name)
    assert insts and isinstance(cfg, dict) and "workload" in cfg
    for d in insts:
        n = int(np.prod(d["grid"]))
        nh = d["conn"] // 2
        assert np.asarray(d["u"]).reshape(-1).shape == (n,) and np.asarray(d["u"]).dtype == np.float32
        assert np.asarray(d["wq"]).reshape(nh, -1).shape == (nh, n) and np.asarray(d["wq"]).dtype == np.int32
        assert len(d["block"]) == len(d["grid"]) and d["lam"] > 0 and d["mu0"] > 0
        if "gmm_fg" in d:           # the end-to-end-from-image leg needs all three
            assert "image" in d and "inv_dist" in d and np.asarray(d["image"]).size % n == 0
            C = len(d["gmm_fg"][1][0])
            assert np.asarray(d["image"]).size == n * C


def test_replica_helpers_single_process():
    import bench
    assert bench.job_rate(100, 1, 4.0) == 25.0
    assert bench.max_over_ranks(1.25, 1) == 1.25


def test_reference_sample_is_a_slab_of_the_volume():
    """The reference arm's bounded sample of the 256x256x128 volume is its
    middle 16-slice slab: same unaries, weights inside the slab unchanged,
    n-links leaving it zero, whole blocks."""
    import bench
    from paper_1704_03116_gb300 import inputs
    full = inputs.ellipsoids3d()
    insts, sample = bench.reference_sample("ellipsoids256")
    d = insts[0]
    assert d["grid"] == (16, 256, 256) and "slab" in sample
    assert all(g % b == 0 for g, b in zip(d["grid"], d["block"]))
    u = full["u"].reshape(128, 256, 256)[56:72]
    assert np.array_equal(d["u"].reshape(16, 256, 256), u)
    w = full["wq"].reshape(3, 128, 256, 256)[:, 56:72]
    dw = d["wq"].reshape(3, 16, 256, 256)
    assert np.array_equal(dw[:, :-1], w[:, :-1]) and (dw[2, -1] == 0).all()
    assert np.array_equal(dw[:2, -1], w[:2, -1])


def test_dice():
    import bench
    a = np.array([1, 1, 0, 0], np.uint8)
    b = np.array([1, 0, 1, 0], np.uint8)
    assert bench.dice(a, a) == 1.0 and bench.dice(a, b) == 0.5 and bench.dice(a * 0, b * 0) == 1.0
