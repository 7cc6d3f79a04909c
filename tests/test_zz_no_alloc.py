"""aidw_interpolate_noalloc: interpolation for callers that cannot let the
library allocate device memory (an application that hands out all GPU memory
from its own pool, or a loop that cannot afford cudaMalloc's synchronisation
or a failed allocation halfway through).  It must give the results of
aidw_interpolate and of the oracle, call after call, from its fixed scratch
array, and must keep working when the library can allocate nothing.

The file name sorts last, so pytest collects it after every other test:
a run that stops at the first failure (-x) has then already run the rest
of the suite when a failure here stops it.  The tests also pass when this
file runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_QUERIES = 65536
AIDW_ERR_INVALID_ARG = 1
AIDW_ERR_OOM = 4
AIDW_ERR_TIMEOUT = 6


def _entry(lib):
    fn = lib.aidw_interpolate_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _call(fn, grid, qx, qy, params, out_z, out_alpha=None):
    import torch
    pc = params.to_c()
    st = fn(grid.handle, ctypes.c_void_p(qx.data_ptr()), ctypes.c_void_p(qy.data_ptr()),
            qx.numel(), ctypes.byref(pc), ctypes.c_void_p(out_z.data_ptr()),
            None if out_alpha is None else ctypes.c_void_p(out_alpha.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("fp64", [False, True])
def test_noalloc_matches_interpolate_on_consecutive_calls(aidw, oracle, fp64):
    import torch
    fn = _entry(aidw.load())
    w = inputs.uniform_kilo(n=40000, m=MAX_QUERIES, seed=21)
    prec = aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP
    p = aidw.Params(k=10, precision=prec)
    dt = torch.float64 if fp64 else torch.float32
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    ref_z, ref_a = aidw.aidw_interpolate(g, qx, qy, p, want_alpha=True)
    ref_z, ref_a = host(ref_z).astype(np.float64), host(ref_a)
    tol = TOL_FP64 if fp64 else TOL_FP32
    s = inputs.query_subsample(MAX_QUERIES, 200, seed=23)
    orc = oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k)
    # two calls in a row on the full size, then a smaller one that reuses the
    # same scratch after it held the larger call's contents
    for m in (MAX_QUERIES, MAX_QUERIES, 1000):
        out_z = torch.full((m,), float("nan"), dtype=dt, device="cuda")
        out_a = torch.full((m,), float("nan"), dtype=dt, device="cuda")
        assert _call(fn, g, qx[:m], qy[:m], p, out_z, out_a) == 0
        torch.cuda.synchronize()
        z = host(out_z).astype(np.float64)
        assert np.isfinite(z).all()
        # against the pooled entry point (same kNN, same weighting kernel)
        np.testing.assert_allclose(z, ref_z[:m], rtol=0, atol=tol * np.abs(w.z).max())
        np.testing.assert_array_equal(host(out_a), ref_a[:m])
        # and on its own against the oracle
        sm = s[s < m]
        err = oracle.normalized_error(z[sm], orc["z"][: sm.size], orc["scale"][: sm.size])
        assert err.max() <= tol, err.max()
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


def test_noalloc_works_when_the_library_can_allocate_nothing(aidw):
    """With the library's pool capped at what it already holds (the grid),
    aidw_interpolate cannot take its per-call scratch and fails with
    AIDW_ERR_OOM, while aidw_interpolate_noalloc still succeeds and gives the
    same predictions: it allocates nothing."""
    import gc

    import torch
    lib = aidw.load()
    fn = _entry(lib)
    gc.collect()     # grids of earlier tests freed now, not during the capped calls
    w = inputs.clustered_kilo(n=30000, m=20000, k=12, seed=24)
    p = aidw.Params(k=12)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    ref, _ = aidw.aidw_interpolate(g, qx, qy, p)
    ref = host(ref)
    torch.cuda.synchronize()
    gc.disable()
    held = aidw.aidw_set_memory_limit(0)
    try:
        aidw.aidw_set_memory_limit(held)
        with pytest.raises(aidw.AidwError) as e:
            aidw.aidw_interpolate(g, qx, qy, p)
        assert e.value.status == AIDW_ERR_OOM
        for _ in range(2):
            out = torch.full((w.m,), float("nan"), dtype=torch.float32, device="cuda")
            assert _call(fn, g, qx, qy, p, out) == 0
            torch.cuda.synchronize()
            np.testing.assert_allclose(host(out), ref, rtol=0,
                                       atol=TOL_FP32 * np.abs(w.z).max())
        assert aidw.aidw_set_memory_limit(held) == held   # nothing was taken from the pool
    finally:
        aidw.aidw_set_memory_limit(0)
        gc.enable()
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


def test_noalloc_expired_wait_gives_nan_not_stale_sums(aidw, oracle):
    """A weighting wait that expires on the no-alloc path (test hook): the
    status reports the timeout, that call's predictions are NaN rather than
    sums of whatever the shared array held, and the next call is correct."""
    import torch
    fn = _entry(aidw.load())
    w = inputs.uniform_kilo(n=20000, m=3000, seed=25)
    p = aidw.Params(k=10)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 10)
    out = torch.empty(w.m, dtype=torch.float32, device="cuda")
    assert _call(fn, g, qx, qy, p, out) == 0          # fills the array with sums
    aidw.aidw_test_expire_next_wait(50)
    out.fill_(0.0)
    assert _call(fn, g, qx, qy, p, out) == 0
    assert aidw.aidw_grid_status(g) == AIDW_ERR_TIMEOUT
    assert np.isnan(host(out)).all()
    assert _call(fn, g, qx, qy, p, out) == 0
    assert aidw.aidw_grid_status(g) == 0
    err = oracle.normalized_error(host(out), ref["z"], ref["scale"])
    assert err.max() <= TOL_FP32
    g.destroy()


def test_noalloc_rejects_oversized_calls(aidw):
    import torch
    fn = _entry(aidw.load())
    w = inputs.uniform_kilo(n=2000, m=MAX_QUERIES + 1, seed=22)
    p = aidw.Params(k=10)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    out_z = torch.empty(w.m, dtype=torch.float32, device="cuda")
    assert _call(fn, g, dev(w.qx), dev(w.qy), p, out_z) == AIDW_ERR_INVALID_ARG
    g.destroy()
