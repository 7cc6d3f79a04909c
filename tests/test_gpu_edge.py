"""Edge cases of the GPU path against the oracle: queries far outside the
data, large or negative coordinates, a zero-area (collinear) data set,
extreme alpha levels, single queries and points, non-default streams and
several live grids."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, check_knn, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(aidw, x, y, z, qx, qy, k, fp64=False, stream=None, **kw):
    p = aidw.Params(k=k, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP, **kw)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(z), p, stream=stream)
    zq, al = aidw.aidw_interpolate(g, dev(qx), dev(qy), p, want_alpha=True, stream=stream)
    if stream is not None:
        stream.synchronize()
    out = host(zq).astype(np.float64), host(al).astype(np.float64)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    return out


def _check(oracle, x, y, z, qx, qy, k, zq, al, fp64=False, **kw):
    ref = oracle.aidw(x, y, z, qx, qy, k, **kw)
    err = oracle.normalized_error(zq, ref["z"], ref["scale"])
    assert err.max() <= (TOL_FP64 if fp64 else TOL_FP32), err.max()
    np.testing.assert_allclose(al, ref["alpha"], atol=1e-9 if fp64 else 1e-5)


@pytest.mark.parametrize("fp64", [False, True])
def test_queries_far_outside_the_data(aidw, oracle, fp64):
    w = inputs.clustered_kilo(n=5000, m=10, seed=51)
    rng = np.random.default_rng(51)
    ang = rng.uniform(0, 2 * np.pi, 300)
    r = rng.uniform(1500, 20000, 300)
    qx = (500 + r * np.cos(ang)).astype(np.float32)
    qy = (500 + r * np.sin(ang)).astype(np.float32)
    zq, al = _run(aidw, w.x, w.y, w.z, qx, qy, 10, fp64)
    _check(oracle, w.x, w.y, w.z, qx, qy, 10, zq, al, fp64)


@pytest.mark.parametrize("offset", [-3.0e5, 1.0e6])
def test_large_and_negative_coordinates(aidw, oracle, offset):
    rng = np.random.default_rng(52)
    x, y = inputs.uniform_points(rng, 8000, offset, offset + 1000.0)
    z = inputs.field_kilo(rng, x, y)
    qx, qy = inputs.uniform_points(rng, 1500, offset, offset + 1000.0)
    for fp64 in (False, True):
        zq, al = _run(aidw, x, y, z, qx, qy, 10, fp64)
        _check(oracle, x, y, z, qx, qy, 10, zq, al, fp64)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(z), aidw.Params())
    idx, dist, robs = aidw.aidw_knn(g, dev(qx), dev(qy), 12)
    g.destroy()
    check_knn(oracle, x, y, qx, qy, 12, host(idx), host(dist), host(robs))


@pytest.mark.parametrize("cell_scale", [0.5, 1.0, 2.0])
def test_stop_rule_at_coarse_float32_spacing(aidw, oracle, cell_scale):
    # around 1e7 float32 coordinates are spaced 1.0 apart, a tenth of a cell
    # here: the stop test's float32 edge bounds must stay lower bounds (an
    # early stop would lose a neighbour the oracle's brute force finds)
    rng = np.random.default_rng(54)
    x, y = inputs.uniform_points(rng, 8000, 1.0e7, 1.0e7 + 1000.0)
    qx, qy = inputs.uniform_points(rng, 2000, 1.0e7 - 50.0, 1.0e7 + 1050.0)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(np.zeros_like(x)),
                             aidw.Params(cell_scale=cell_scale))
    for k in (1, 12, 32):
        idx, dist, robs = aidw.aidw_knn(g, dev(qx), dev(qy), k)
        check_knn(oracle, x, y, qx, qy, k, host(idx), host(dist), host(robs))
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


def test_collinear_data_zero_area(aidw, oracle):
    rng = np.random.default_rng(53)
    y = rng.uniform(0, 100, 3000).astype(np.float32)
    x = np.full_like(y, 7.0)
    z = inputs.field_kilo(rng, x, y)
    qx = rng.uniform(-10, 20, 500).astype(np.float32)
    qy = rng.uniform(-10, 110, 500).astype(np.float32)
    for fp64 in (False, True):
        zq, al = _run(aidw, x, y, z, qx, qy, 8, fp64)
        _check(oracle, x, y, z, qx, qy, 8, zq, al, fp64)
        # r_exp = 0 (zero area): R = inf, mu = 1, alpha = alpha_5
        np.testing.assert_array_equal(al, 5.0)


@pytest.mark.parametrize("levels", [(0.1, 0.2, 0.3, 0.4, 0.5), (6, 7, 8, 9, 10)])
def test_extreme_alpha_levels(aidw, oracle, levels):
    w = inputs.uniform_kilo(n=6000, m=1500, seed=54)
    for fp64 in (False, True):
        zq, al = _run(aidw, w.x, w.y, w.z, w.qx, w.qy, 10, fp64, alpha=levels)
        _check(oracle, w.x, w.y, w.z, w.qx, w.qy, 10, zq, al, fp64, levels=levels)


def test_single_query_single_point_and_k1(aidw, oracle):
    w = inputs.unit_square(3000, m=1, seed=55)
    for k in (1, 32):
        zq, al = _run(aidw, w.x, w.y, w.z, w.qx, w.qy, k)
        _check(oracle, w.x, w.y, w.z, w.qx, w.qy, k, zq, al)
    zq, _ = _run(aidw, w.x[:1], w.y[:1], w.z[:1], w.qx, w.qy, 1)
    assert zq[0] == pytest.approx(float(w.z[0]), rel=1e-7)


def test_non_default_stream_and_two_live_grids(aidw, oracle):
    import torch
    s = torch.cuda.Stream()
    a = inputs.uniform_kilo(n=7000, m=2000, seed=56)
    b = inputs.clustered_kilo(n=9000, m=2000, seed=57)
    pa, pb = aidw.Params(k=10), aidw.Params(k=16)
    with torch.cuda.stream(s):
        ga = aidw.aidw_grid_build(dev(a.x), dev(a.y), dev(a.z), pa, stream=s)
        gb = aidw.aidw_grid_build(dev(b.x), dev(b.y), dev(b.z), pb, stream=s)
        za, _ = aidw.aidw_interpolate(ga, dev(a.qx), dev(a.qy), pa, stream=s)
        zb, _ = aidw.aidw_interpolate(gb, dev(b.qx), dev(b.qy), pb, stream=s)
        za2, _ = aidw.aidw_interpolate(ga, dev(a.qx), dev(a.qy), pa, stream=s)
    s.synchronize()
    ra = oracle.aidw(a.x, a.y, a.z, a.qx, a.qy, 10)
    rb = oracle.aidw(b.x, b.y, b.z, b.qx, b.qy, 16)
    assert oracle.normalized_error(host(za), ra["z"], ra["scale"]).max() <= TOL_FP32
    assert oracle.normalized_error(host(zb), rb["z"], rb["scale"]).max() <= TOL_FP32
    np.testing.assert_array_equal(host(za2), host(za))    # deterministic
    ga.destroy()
    gb.destroy()


def test_repeated_calls_are_bitwise_deterministic(aidw):
    w = inputs.clustered_kilo(n=20000, m=5000, seed=58)
    outs = [_run(aidw, w.x, w.y, w.z, w.qx, w.qy, 10)[0] for _ in range(3)]
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_memory_cap_reports_oom_and_recovers(aidw):
    """The OOM path, forced through the library's pool cap (no real
    exhaustion of the GPU)."""
    w = inputs.uniform_kilo(n=200000, m=5000, seed=59)
    p = aidw.Params()
    assert aidw.aidw_set_memory_limit(1 << 20) >= 0
    try:
        with pytest.raises(aidw.AidwError) as e:
            aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
        assert e.value.status == 4
    finally:
        aidw.aidw_set_memory_limit(0)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    # a cap between the grid and the call's scratch fails the call, not the grid
    held = aidw.aidw_set_memory_limit(0)
    aidw.aidw_set_memory_limit(held + 1024)
    try:
        with pytest.raises(aidw.AidwError) as e:
            aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p)
        assert e.value.status == 4
    finally:
        aidw.aidw_set_memory_limit(0)
    z, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p)
    assert np.isfinite(host(z)).all()
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


def test_data_order_permutation(aidw, oracle):
    """Permuting the data points changes nothing but the indices (ties are
    broken by index, so compare distances and mapped index sets)."""
    w = inputs.clustered_kilo(n=20000, m=3000, seed=60)
    perm = np.random.default_rng(60).permutation(w.n)
    p = aidw.Params(k=12)
    g1 = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    g2 = aidw.aidw_grid_build(dev(w.x[perm]), dev(w.y[perm]), dev(w.z[perm]), p)
    i1, d1, r1 = (host(t) for t in aidw.aidw_knn(g1, dev(w.qx), dev(w.qy), 12))
    i2, d2, r2 = (host(t) for t in aidw.aidw_knn(g2, dev(w.qx), dev(w.qy), 12))
    np.testing.assert_array_equal(d2, d1)
    np.testing.assert_array_equal(r2, r1)
    same = np.array([set(a) == set(b) for a, b in zip(i1.tolist(), perm[i2].tolist())])
    assert same.mean() > 0.999
    z1, a1 = aidw.aidw_interpolate(g1, dev(w.qx), dev(w.qy), p, want_alpha=True)
    z2, a2 = aidw.aidw_interpolate(g2, dev(w.qx), dev(w.qy), p, want_alpha=True)
    np.testing.assert_array_equal(host(a2), host(a1))
    # the data order changes only the rounding order of the sums: both are
    # within the float32 tolerance of the oracle
    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 12)
    for z in (z1, z2):
        assert oracle.normalized_error(host(z), ref["z"], ref["scale"]).max() <= TOL_FP32
    g1.destroy()
    g2.destroy()


def test_interpolate_replays_in_a_cuda_graph(aidw, oracle):
    """aidw_interpolate enqueues only stream-ordered allocations, memsets and
    kernels, so it can be captured once and replayed on new query values."""
    import torch
    w = inputs.clustered_kilo(n=30000, m=6000, seed=62)
    p = aidw.Params(k=10)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    qx, qy = dev(w.qx), dev(w.qy)
    out = torch.empty(w.m, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        aidw.aidw_interpolate(g, qx, qy, p, out_z=out, stream=s)   # first call outside
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        aidw.aidw_interpolate(g, qx, qy, p, out_z=out, stream=s)
    rng = np.random.default_rng(63)
    for _ in range(2):
        nqx, nqy = inputs.uniform_points(rng, w.m, 0.0, 1000.0)
        qx.copy_(dev(nqx))
        qy.copy_(dev(nqy))
        out.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        ref = oracle.aidw(w.x, w.y, w.z, nqx, nqy, 10)
        err = oracle.normalized_error(host(out), ref["z"], ref["scale"])
        assert err.max() <= TOL_FP32
    del graph
    g.destroy()


def test_expired_wait_reports_timeout_and_gpu_stays_usable(aidw, oracle):
    """The weighting kernel's bounded data-tile wait: a copy that is never
    issued makes the wait expire (50 tries); the kernel latches the timeout,
    sets the launch's failure flag, drains its own copies and returns; that
    call's predictions are all NaN (no partial sum cut short reaches the
    output); the next call is correct."""
    w = inputs.uniform_kilo(n=20000, m=3000, seed=64)
    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 10)
    for fp64 in (False, True):
        pp = aidw.Params(k=10, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
        tol = TOL_FP64 if fp64 else TOL_FP32
        g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), pp)
        aidw.aidw_test_expire_next_wait(50)
        z0, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), pp)
        assert aidw.aidw_grid_status(g) == 6          # AIDW_ERR_TIMEOUT
        assert aidw.aidw_grid_status(g) == 0          # cleared
        assert np.isnan(host(z0)).all()
        z, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), pp)
        assert aidw.aidw_grid_status(g) == 0
        assert oracle.normalized_error(host(z), ref["z"], ref["scale"]).max() <= tol
        g.destroy()
