"""The C-ABI library loads and exports every function include/dope.h declares,
and its host-side argument checks work without a GPU."""
import ctypes

import numpy as np

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


def test_no_gpu_server_and_batch(lib):
    """The server and the batched call also fail loudly without a device, and
    reject malformed arguments before touching it."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.DopeError) as ei:
        lib.dope_server_create()
    assert ei.value.status == lib.DOPE_ECUDA
    p = lib.dope_server_params(0, 0, 7, 0, 0)            # unknown mode (0, 1, 2 exist)
    out = ctypes.c_void_p()
    assert lib._lib.dope_server_create(ctypes.byref(p), ctypes.byref(out)) == lib.DOPE_EINVAL
    assert lib._lib.dope_server_submit(None, None, None) == lib.DOPE_EINVAL
    assert lib._lib.dope_server_cancel(None, 1) == lib.DOPE_EINVAL
    assert lib.dope_strerror(lib.DOPE_ECANCELED) == "request cancelled"
    with pytest.raises(lib.DopeError) as ei:
        lib.dope_iterate_batch([], 10)
    assert ei.value.status == lib.DOPE_EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    rc = lib._lib.dope_iterate_batch(arr, lib.DOPE_BATCH_MAX + 1, 10, None, None, None, None)
    assert rc == lib.DOPE_EINVAL


def test_potentials_argument_checks(lib):
    """The potentials calls validate the models and the grid on the host,
    before any GPU work (n = 0 / null pointers never reach a device)."""
    L = lib._lib
    ok = lib.gmm([1.0], [[0.5, 0.5, 0.5]], [np.eye(3) * 0.01])
    assert L.dope_gmm_unaries(None, 0, 3, ctypes.byref(ok), ctypes.byref(ok), 1e5, None, None) == lib.DOPE_OK
    bad = lib.gmm([1.0], [[0.5, 0.5, 0.5]], [np.diag([0.01, -0.01, 0.01])])      # not positive definite
    assert L.dope_gmm_unaries(None, 0, 3, ctypes.byref(ok), ctypes.byref(bad), 1e5, None, None) == lib.DOPE_EINVAL
    zero_w = lib.gmm([0.0], [[0.5, 0.5, 0.5]], [np.eye(3) * 0.01])
    assert L.dope_gmm_unaries(None, 0, 3, ctypes.byref(zero_w), ctypes.byref(ok), 1e5, None, None) == lib.DOPE_EINVAL
    assert L.dope_gmm_unaries(None, 0, 2, ctypes.byref(ok), ctypes.byref(ok), 1e5, None, None) == lib.DOPE_EINVAL
    assert L.dope_gmm_unaries(None, 0, 3, ctypes.byref(ok), ctypes.byref(ok), 0.0, None, None) == lib.DOPE_EINVAL
    assert L.dope_gmm_unaries(None, 5, 3, ctypes.byref(ok), ctypes.byref(ok), 1e5, None, None) == lib.DOPE_EINVAL
    g = (ctypes.c_int64 * 3)(4, 8, 8)
    for ndim, conn in ((2, 6), (2, 32), (3, 4), (3, 24), (2, 10)):
        assert L.dope_contrast_weights(None, g, ndim, 3, conn, 1.0, 0, None, None, None, None) == lib.DOPE_EINVAL
    assert L.dope_contrast_weights(None, g, 2, 5, 4, 1.0, 0, None, None, None, None) == lib.DOPE_EINVAL
    huge = (ctypes.c_int64 * 3)(1 << 30, 1 << 30, 1 << 30)             # N far beyond 2^31
    assert L.dope_contrast_weights(None, huge, 3, 1, 6, 1.0, 0, None, None, None, None) == lib.DOPE_EINVAL
    assert L.dope_set_image(None, None, 3, ctypes.byref(ok), ctypes.byref(ok), 1e5, 0.0, 0, 0, None,
                            None) == lib.DOPE_EINVAL


def test_async_and_two_phase_calls_reject_bad_arguments(lib):
    """The asynchronous upload and the two-phase solve validate on the host."""
    L = lib._lib
    assert L.dope_set_inputs(None, None, None, 0, 0, None) == lib.DOPE_EINVAL
    assert L.dope_solve_begin(None, None, 0, None) == lib.DOPE_EINVAL
    assert L.dope_solve_end(None, None, None, None) == lib.DOPE_EINVAL
    ok = lib.gmm([1.0], [[0.5, 0.5, 0.5]], [np.eye(3) * 0.01])
    assert L.dope_set_image(None, None, 3, ctypes.byref(ok), ctypes.byref(ok), 1e5, 0.0, 0, 0, None,
                            None) == lib.DOPE_EINVAL
    p = lib.dope_default_params()
    assert p.barrier_timeout_us == 0 and p.threads == 0


def test_struct_layouts_match_header(lib):
    """ctypes mirrors of the C structs have the C sizes (compiled probe)."""
    import os
    import subprocess
    import tempfile
    src = ('#include <stdio.h>\n#include "dope_potentials.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
           'sizeof(dope_params),sizeof(dope_stats),sizeof(dope_profile),sizeof(dope_server_params),'
           'sizeof(dope_request),sizeof(dope_result),sizeof(dope_server_stats),sizeof(dope_tune_result),'
           'sizeof(dope_gmm));printf("%zu\\n",sizeof(dope_image_request));'
           'return 0;}\n')
    inc = os.path.dirname(lib.HEADER)
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "sz.c")
        exe = os.path.join(td, "sz")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + inc, c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(t) for t in (lib.dope_params, lib.dope_stats, lib.dope_profile, lib.dope_server_params,
                                       lib.dope_request, lib.dope_result, lib.dope_server_stats,
                                       lib.dope_tune_result, lib.dope_gmm, lib.dope_image_request)]
    assert got == want
