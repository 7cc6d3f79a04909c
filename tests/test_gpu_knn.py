"""Grid kNN (Sec. 3.2.4 / 4.1.4) against the oracle's brute force (Sec. 2.3):
the same k nearest neighbours, in increasing (distance, index) order."""
import numpy as np
import pytest

from gpu_helpers import check_knn, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _knn(aidw, x, y, qx, qy, k, cell_scale=1.0):
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(np.zeros_like(x)),
                             aidw.Params(cell_scale=cell_scale))
    idx, dist, robs = aidw.aidw_knn(g, dev(qx), dev(qy), k)
    out = host(idx), host(dist), host(robs)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    return out


@pytest.mark.parametrize("k", [1, 2, 8, 10, 16, 17, 24, 32])
def test_knn_unit_square(aidw, oracle, k):
    w = inputs.unit_square(4096, seed=0)
    idx, dist, robs = _knn(aidw, w.x, w.y, w.qx, w.qy, k)
    assert check_knn(oracle, w.x, w.y, w.qx, w.qy, k, idx, dist, robs) > 0.999


@pytest.mark.parametrize("cell_scale", [0.5, 1.0, 2.0, 4.0, 8.0])
def test_knn_does_not_depend_on_cell_width(aidw, oracle, cell_scale):
    w = inputs.uniform_kilo(n=20000, m=3000, seed=5)
    base = _knn(aidw, w.x, w.y, w.qx, w.qy, 10, 1.0)
    got = _knn(aidw, w.x, w.y, w.qx, w.qy, 10, cell_scale)
    np.testing.assert_array_equal(got[0], base[0])
    np.testing.assert_array_equal(got[1], base[1])
    if cell_scale == 8.0:
        check_knn(oracle, w.x, w.y, w.qx, w.qy, 10, got[0], got[1], got[2])


@pytest.mark.parametrize("n,m", [(1, 5), (10, 1), (33, 1025), (1000, 7), (5000, 3001)])
def test_knn_ragged(aidw, oracle, n, m):
    rng = np.random.default_rng(n * 7 + m)
    x, y = inputs.uniform_points(rng, n, 0.0, 1000.0)
    qx, qy = inputs.uniform_points(rng, m, 0.0, 1000.0)
    k = min(10, n)
    idx, dist, robs = _knn(aidw, x, y, qx, qy, k)
    check_knn(oracle, x, y, qx, qy, k, idx, dist, robs)


def test_knn_k_equals_n(aidw, oracle):
    rng = np.random.default_rng(2)
    x, y = inputs.uniform_points(rng, 32, 0.0, 1.0)
    qx, qy = inputs.uniform_points(rng, 100, -0.5, 1.5)
    idx, dist, robs = _knn(aidw, x, y, qx, qy, 32)
    check_knn(oracle, x, y, qx, qy, 32, idx, dist, robs)
    assert all(sorted(r) == list(range(32)) for r in idx.tolist())


def test_knn_clustered(aidw, oracle):
    w = inputs.clustered_kilo(n=100000, m=2000, seed=2)
    for k in (10, 20):
        idx, dist, robs = _knn(aidw, w.x, w.y, w.qx, w.qy, k)
        check_knn(oracle, w.x, w.y, w.qx, w.qy, k, idx, dist, robs)


def test_knn_duplicates_ties_and_outside_queries(aidw, oracle):
    rng = np.random.default_rng(6)
    x = rng.integers(0, 30, 3000).astype(np.float32)
    y = rng.integers(0, 30, 3000).astype(np.float32)
    qx = np.concatenate([x[:200], rng.uniform(-40, 70, 800)]).astype(np.float32)
    qy = np.concatenate([y[:200], rng.uniform(-40, 70, 800)]).astype(np.float32)
    for k in (5, 12, 32):
        idx, dist, robs = _knn(aidw, x, y, qx, qy, k)
        ridx, rd = oracle.knn(x, y, qx, qy, k)
        # queries on the integer lattice: squared distances are small
        # integers, exact in float32, so the (distance, index) order is fully
        # determined, ties included, and must match
        np.testing.assert_array_equal(idx[:200], ridx[:200])
        np.testing.assert_allclose(dist[:200], rd[:200], rtol=1e-7)
        check_knn(oracle, x, y, qx[200:], qy[200:], k, idx[200:], dist[200:], robs[200:])


def test_knn_nonfinite_query_is_flagged(aidw):
    w = inputs.unit_square(1000, m=10, seed=1)
    qx = w.qx.copy()
    qx[3] = np.inf
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params())
    idx, dist, robs = aidw.aidw_knn(g, dev(qx), dev(w.qy), 4)
    idx = host(idx)
    assert (idx[3] == -1).all() and np.isnan(host(robs)[3])
    assert (idx[[0, 1, 2, 4]] >= 0).all()
    assert aidw.aidw_grid_status(g) == 3
    assert aidw.aidw_grid_status(g) == 0   # cleared after reading
    g.destroy()


def test_knn_argument_errors(aidw):
    w = inputs.unit_square(100, m=10, seed=1)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params())
    for k in (0, 33, 101):
        with pytest.raises(aidw.AidwError) as e:
            aidw.aidw_knn(g, dev(w.qx), dev(w.qy), k)
        assert e.value.status == 2
    g.destroy()


@pytest.mark.slow
@pytest.mark.parametrize("kind,k", [("uniform", 10), ("clustered", 32), ("clustered", 8)])
def test_knn_full_size_sampled(aidw, oracle, kind, k):
    """1,048,576 points and queries at the automatic cell width for k (the
    grid is built with the same k); the oracle checks a sample."""
    w = inputs.uniform_kilo(seed=1) if kind == "uniform" else inputs.clustered_kilo(seed=2)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params(k=k))
    idx, dist, robs = (host(t) for t in aidw.aidw_knn(g, dev(w.qx), dev(w.qy), k))
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    s = inputs.query_subsample(w.m, 256)
    check_knn(oracle, w.x, w.y, w.qx[s], w.qy[s], k, idx[s], dist[s], robs[s])


@pytest.mark.parametrize("k", [1, 10, 16, 32])
def test_bruteforce_knn_equals_grid_knn(aidw, oracle, k):
    """The paper's original all-points kNN and the grid kNN use the same
    float32 distance and (d^2, index) order: identical results."""
    w = inputs.clustered_kilo(n=30000, m=3000, seed=41)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params(cell_scale=1.0))
    a = [host(t) for t in aidw.aidw_knn(g, dev(w.qx), dev(w.qy), k)]
    b = [host(t) for t in aidw.aidw_knn_bruteforce(g, dev(w.qx), dev(w.qy), k)]
    g.destroy()
    np.testing.assert_array_equal(b[0], a[0])
    np.testing.assert_array_equal(b[1], a[1])
    np.testing.assert_array_equal(b[2], a[2])
    s = np.arange(0, w.m, 7)
    check_knn(oracle, w.x, w.y, w.qx[s], w.qy[s], k, b[0][s], b[1][s], b[2][s])


def test_query_cell_order_changes_nothing(aidw):
    """From 4096 queries the kNN visits queries in grid-cell order; the same
    queries below that size run in input order.  Results are identical."""
    w = inputs.clustered_kilo(n=50000, m=6000, seed=43)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params(cell_scale=1.0))
    big = [host(t) for t in aidw.aidw_knn(g, dev(w.qx), dev(w.qy), 20)]
    small = [host(t) for t in aidw.aidw_knn(g, dev(w.qx[:3000]), dev(w.qy[:3000]), 20)]
    for a, b in zip(big, small):
        np.testing.assert_array_equal(a[:3000], b)
    p = aidw.Params(k=20)
    zb, ab = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p, want_alpha=True)
    zs, as_ = aidw.aidw_interpolate(g, dev(w.qx[:3000]), dev(w.qy[:3000]), p, want_alpha=True)
    np.testing.assert_array_equal(host(ab)[:3000], host(as_))
    g.destroy()
