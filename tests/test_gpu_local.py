"""Local AIDW (Eq. 1 over the k nearest points) on the GPU against the oracle's
local mode."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _local(aidw, x, y, z, qx, qy, k, fp64=False, **kw):
    p = aidw.Params(k=k, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP, **kw)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(z), p)
    zq, al = aidw.aidw_interpolate_local(g, dev(qx), dev(qy), p, want_alpha=True)
    out = host(zq).astype(np.float64), host(al).astype(np.float64)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    return out


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("k", [1, 8, 10, 17, 32])
def test_local_matches_oracle(aidw, oracle, fp64, k):
    w = inputs.clustered_kilo(n=20000, m=3000, seed=31)
    zq, al = _local(aidw, w.x, w.y, w.z, w.qx, w.qy, k, fp64)
    ref = oracle.aidw_local(w.x, w.y, w.z, w.qx, w.qy, k)
    err = oracle.normalized_error(zq, ref["z"], ref["scale"])
    assert err.max() <= (TOL_FP64 if fp64 else TOL_FP32), err.max()
    np.testing.assert_allclose(al, ref["alpha"], atol=1e-9 if fp64 else 1e-5)


def test_local_hits_duplicates_and_k_equals_n(aidw, oracle):
    rng = np.random.default_rng(32)
    x = rng.integers(0, 20, 600).astype(np.float32)
    y = rng.integers(0, 20, 600).astype(np.float32)
    z = inputs.field_kilo(rng, x, y)
    qx = np.concatenate([x[:100], rng.uniform(-5, 25, 300)]).astype(np.float32)
    qy = np.concatenate([y[:100], rng.uniform(-5, 25, 300)]).astype(np.float32)
    for k in (4, 16, 32):
        zq, _ = _local(aidw, x, y, z, qx, qy, k)
        ref = oracle.aidw_local(x, y, z, qx, qy, k)
        assert oracle.normalized_error(zq, ref["z"], ref["scale"]).max() <= TOL_FP32
    xs, ys, zs = x[:32], y[:32] + np.float32(0.25) * np.arange(32, dtype=np.float32), z[:32]
    zq, _ = _local(aidw, xs, ys, zs, qx, qy, 32, fp64=True)
    ref = oracle.aidw(xs, ys, zs, qx, qy, 32)      # k = n: the all-points form
    assert oracle.normalized_error(zq, ref["z"], ref["scale"]).max() <= TOL_FP64


@pytest.mark.slow
def test_local_full_size_sampled(aidw, oracle):
    w = inputs.uniform_kilo(seed=1)
    zq, al = _local(aidw, w.x, w.y, w.z, w.qx, w.qy, 10)
    s = inputs.query_subsample(w.m, 256)
    ref = oracle.aidw_local(w.x, w.y, w.z, w.qx[s], w.qy[s], 10)
    assert oracle.normalized_error(zq[s], ref["z"], ref["scale"]).max() <= TOL_FP32
