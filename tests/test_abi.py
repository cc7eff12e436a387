"""The C-ABI library loads and exports every function include/dope.h declares,
and its host-side argument checks work without a GPU."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03116_gb300 import _build
    _build.build()
    from paper_1704_03116_gb300 import dope
    return dope


def test_every_declared_symbol_is_exported(lib):
    names = lib.declared_symbols()
    assert len(names) >= 15
    raw = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_strerror_and_defaults(lib):
    assert lib.dope_strerror(0) == "ok"
    assert "negative" in lib.dope_strerror(lib.DOPE_EUNSUPPORTED)
    p = lib.dope_default_params()
    assert (p.mu0, p.mu_fact, p.eps, p.max_iter) == (0.0, 1.05, 1e-3, 1000)


@pytest.mark.parametrize("grid,conn,block,lam", [
    ((64, 64), 6, (16, 16), 1.0),        # 6-conn needs 3-D
    ((8, 8, 8), 4, (4, 4, 4), 1.0),      # 4-conn needs 2-D
    ((64, 60), 4, (16, 16), 1.0),        # block does not tile the grid
    ((64, 64), 4, (0, 16), 1.0),         # empty block
    ((0, 64), 4, (16, 16), 1.0),         # empty grid
    ((128, 128), 4, (128, 64), 1.0),     # block volume above 4096
    ((64, 64), 4, (16, 16), -1.0),       # lambda < 0
])
def test_create_rejects_bad_arguments(lib, grid, conn, block, lam):
    with pytest.raises(lib.DopeError) as ei:
        lib.dope_create(grid, conn, block, lam)
    assert ei.value.status == lib.DOPE_EINVAL


def test_create_rejects_bad_thread_count(lib):
    p = lib.dope_default_params()
    p.threads = 48
    with pytest.raises(lib.DopeError) as ei:
        lib.dope_create((64, 64), 4, (16, 16), 1.0, p)
    assert ei.value.status == lib.DOPE_EINVAL


def test_no_gpu_fails_loudly(lib):
    """Without a device the library reports a CUDA error; it never falls back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.DopeError) as ei:
        lib.dope_create((64, 64), 4, (16, 16), 1.0)
    assert ei.value.status == lib.DOPE_ECUDA
