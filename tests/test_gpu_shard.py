"""aidw_interpolate_shard: one slice of a query set per call, as each GPU of
a query-sharded run computes it.  The slices of all shards fill the output
exactly once and agree with the one-call result and with the oracle."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run_shards(aidw, g, qx, qy, p, n_shards, dt):
    import torch
    m = qx.numel()
    out = torch.full((m,), float("nan"), dtype=dt, device="cuda")
    alpha = torch.full((m,), float("nan"), dtype=dt, device="cuda")
    for s in range(n_shards):
        b, e = aidw.aidw_shard_range(m, s, n_shards)
        before = host(out).copy()
        aidw.aidw_interpolate_shard(g, qx, qy, s, n_shards, p, out_z=out, out_alpha=alpha)
        after = host(out)
        # only this shard's slice was written
        outside = np.ones(m, bool)
        outside[b:e] = False
        np.testing.assert_array_equal(after[outside], before[outside])
        assert np.isfinite(after[b:e]).all()
    return host(out), host(alpha)


@pytest.mark.parametrize("fp64", [False, True])
def test_one_shard_is_interpolate(aidw, fp64):
    import torch
    w = inputs.uniform_kilo(n=30000, m=5000, seed=41)
    p = aidw.Params(k=10, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
    dt = torch.float64 if fp64 else torch.float32
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    ref, ref_a = aidw.aidw_interpolate(g, qx, qy, p, want_alpha=True)
    z, a = _run_shards(aidw, g, qx, qy, p, 1, dt)
    np.testing.assert_array_equal(z, host(ref))
    np.testing.assert_array_equal(a, host(ref_a))
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


@pytest.mark.parametrize("n_shards,m", [(3, 10007), (4, 3), (8, 70000)])
@pytest.mark.parametrize("fp64", [False, True])
def test_shards_fill_the_output_and_match_the_oracle(aidw, oracle, n_shards, m, fp64):
    import torch
    w = inputs.clustered_kilo(n=20000, m=m, k=12, seed=43)
    p = aidw.Params(k=12, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
    dt = torch.float64 if fp64 else torch.float32
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    full, full_a = aidw.aidw_interpolate(g, qx, qy, p, want_alpha=True)
    z, a = _run_shards(aidw, g, qx, qy, p, n_shards, dt)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    # alpha comes from the kNN stage, which is per query: identical
    np.testing.assert_array_equal(a, host(full_a))
    s = inputs.query_subsample(m, 300, seed=44)
    ref = oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k)
    tol = TOL_FP64 if fp64 else TOL_FP32
    for zz in (z, host(full)):
        err = oracle.normalized_error(zz[s], ref["z"], ref["scale"])
        assert err.max() <= tol, err.max()


def test_sharded_helper_without_distributed_is_the_whole_set(aidw):
    """interpolate_sharded with no process group: one rank, the whole set."""
    from paper_1601_05904_gb300 import shard
    w = inputs.uniform_kilo(n=8000, m=2000, seed=45)
    p = aidw.Params(k=10)
    t = {k: dev(getattr(w, k)) for k in ("x", "y", "z", "qx", "qy")}
    z = shard.interpolate_sharded(t["x"], t["y"], t["z"], t["qx"], t["qy"], p)
    g = aidw.aidw_grid_build(t["x"], t["y"], t["z"], p)
    ref, _ = aidw.aidw_interpolate(g, t["qx"], t["qy"], p)
    g.destroy()
    np.testing.assert_array_equal(host(z), host(ref))


def test_bad_shard_is_rejected_without_work(aidw):
    w = inputs.uniform_kilo(n=3000, m=100, seed=46)
    p = aidw.Params(k=10)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    with pytest.raises(aidw.AidwError):
        aidw.aidw_interpolate_shard(g, dev(w.qx), dev(w.qy), 2, 2, p)
    g.destroy()
