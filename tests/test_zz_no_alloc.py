"""aidw_interpolate_noalloc: interpolation for callers that cannot let the
library allocate device memory (an application that hands out all GPU memory
from its own pool, or a loop that cannot afford cudaMalloc's synchronisation
or a failed allocation halfway through).  It must give the results of
aidw_interpolate, call after call, from its fixed scratch array.

This file is collected last on purpose: it runs after every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_QUERIES = 65536


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
def test_noalloc_matches_interpolate_on_consecutive_calls(aidw, fp64):
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
    scale = np.abs(w.z).max()
    tol = (TOL_FP64 if fp64 else TOL_FP32) * scale
    # two calls in a row on the full size, then a smaller one that reuses the
    # same scratch after it held the larger call's contents
    for m in (MAX_QUERIES, MAX_QUERIES, 1000):
        out_z = torch.full((m,), float("nan"), dtype=dt, device="cuda")
        out_a = torch.full((m,), float("nan"), dtype=dt, device="cuda")
        assert _call(fn, g, qx[:m], qy[:m], p, out_z, out_a) == 0
        torch.cuda.synchronize()
        z = host(out_z).astype(np.float64)
        assert np.isfinite(z).all()
        np.testing.assert_allclose(z, ref_z[:m], rtol=0, atol=tol)
        np.testing.assert_array_equal(host(out_a), ref_a[:m])
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


def test_noalloc_rejects_oversized_calls(aidw):
    import torch
    fn = _entry(aidw.load())
    w = inputs.uniform_kilo(n=2000, m=MAX_QUERIES + 1, seed=22)
    p = aidw.Params(k=10)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    out_z = torch.empty(w.m, dtype=torch.float32, device="cuda")
    assert _call(fn, g, dev(w.qx), dev(w.qy), p, out_z) == 1   # AIDW_ERR_INVALID_ARG
    g.destroy()
