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
