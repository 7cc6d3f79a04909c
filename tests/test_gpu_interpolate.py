"""AIDW predictions (Sec. 2.2, Eq. 1-6) on the GPU against the FP64 oracle:
float32-compensated path within 1e-5 and float64 path within 1e-9 of the
scale S_q = sum w|z| / sum w, alpha to rounding."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _interp(aidw, x, y, z, qx, qy, k, fp64=False, levels=(1, 2, 3, 4, 5), r_min=0.0,
            r_max=2.0, area=0.0, cell_scale=0.0):
    p = aidw.Params(k=k, alpha=tuple(float(a) for a in levels), r_min=r_min, r_max=r_max,
                    area=area, cell_scale=cell_scale,
                    precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(z), p)
    zq, al = aidw.aidw_interpolate(g, dev(qx), dev(qy), p, want_alpha=True)
    out = host(zq), host(al)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    return out


def _check(oracle, w_x, w_y, w_z, qx, qy, k, zq, al, tol, atol_alpha, **kw):
    ref = oracle.aidw(w_x, w_y, w_z, qx, qy, k, **kw)
    err = oracle.normalized_error(zq, ref["z"], ref["scale"])
    assert err.max() <= tol, f"max normalised error {err.max():.3e} (tol {tol:g})"
    np.testing.assert_allclose(al.astype(np.float64), ref["alpha"], rtol=0, atol=atol_alpha)
    return err.max()


@pytest.mark.parametrize("fp64", [False, True])
def test_unit_square_all_queries(aidw, oracle, fp64):
    w = inputs.unit_square(4096, seed=0)
    zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, w.k, fp64)
    _check(oracle, w.x, w.y, w.z, w.qx, w.qy, w.k, zq, al,
           TOL_FP64 if fp64 else TOL_FP32, 1e-9 if fp64 else 1e-5)


@pytest.mark.parametrize("levels", [(0.5, 1, 2, 3, 4), (2, 2, 2, 2, 2), (5, 4, 3, 2, 1)])
@pytest.mark.parametrize("fp64", [False, True])
def test_other_alpha_levels(aidw, oracle, levels, fp64):
    w = inputs.uniform_kilo(n=6000, m=2500, seed=4)
    zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10, fp64, levels=levels)
    _check(oracle, w.x, w.y, w.z, w.qx, w.qy, 10, zq, al,
           TOL_FP64 if fp64 else TOL_FP32, 1e-9 if fp64 else 1e-5, levels=levels)


@pytest.mark.parametrize("n,m,k", [(1, 3, 1), (10, 1, 10), (33, 1025, 8), (1000, 7, 16),
                                   (4097, 3001, 32), (2500, 1024, 24)])
@pytest.mark.parametrize("fp64", [False, True])
def test_ragged_sizes(aidw, oracle, n, m, k, fp64):
    rng = np.random.default_rng(n + 13 * m)
    x, y = inputs.uniform_points(rng, n, 0.0, 1000.0)
    z = inputs.field_kilo(rng, x, y)
    qx, qy = inputs.uniform_points(rng, m, 0.0, 1000.0)
    zq, al = _interp(aidw, x, y, z, qx, qy, k, fp64)
    _check(oracle, x, y, z, qx, qy, k, zq, al, TOL_FP64 if fp64 else TOL_FP32,
           1e-9 if fp64 else 1e-5)


def test_clustered(aidw, oracle):
    w = inputs.clustered_kilo(n=30000, m=3000, seed=2)
    for k in (10, 20):
        for fp64 in (False, True):
            zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, k, fp64)
            _check(oracle, w.x, w.y, w.z, w.qx, w.qy, k, zq, al,
                   TOL_FP64 if fp64 else TOL_FP32, 1e-9 if fp64 else 1e-5)


def test_hits_duplicates_and_hand_cases(aidw, oracle):
    # queries on data points return their values; coincident duplicates
    # return the mean of their values
    w = inputs.unit_square(2000, m=10, seed=9)
    x = np.concatenate([w.x, w.x[:50]])
    y = np.concatenate([w.y, w.y[:50]])
    z = np.concatenate([w.z, w.z[:50] + np.float32(1.0)])
    qx = np.concatenate([x[::13], w.qx]).astype(np.float32)
    qy = np.concatenate([y[::13], w.qy]).astype(np.float32)
    for fp64 in (False, True):
        zq, al = _interp(aidw, x, y, z, qx, qy, 10, fp64)
        _check(oracle, x, y, z, qx, qy, 10, zq, al, TOL_FP64 if fp64 else TOL_FP32,
               1e-9 if fp64 else 1e-5)


@pytest.mark.parametrize("k", [10, 32])
def test_more_coincident_points_than_k(aidw, oracle, k):
    """A query on a location held by more data points than k returns the mean
    z of all of them (reading Z12, the limit of Eq. 1), not of the k it keeps
    as neighbours; alpha still comes from the k nearest (all at distance 0
    there: R = 0, alpha = alpha_1)."""
    w = inputs.uniform_kilo(n=3000, m=20, seed=11)
    rng = np.random.default_rng(11)
    spots = [(123.25, 456.5, 40), (700.0, 10.75, 50), (999.5, 999.5, 33)]
    xs, ys, zs = [w.x], [w.y], [w.z]
    for sx, sy, c in spots:
        xs.append(np.full(c, sx, np.float32))
        ys.append(np.full(c, sy, np.float32))
        zs.append(rng.normal(0.0, 10.0, c).astype(np.float32))
    x, y, z = (np.concatenate(a) for a in (xs, ys, zs))
    qx = np.concatenate([np.float32([sx for sx, _, _ in spots]), w.qx]).astype(np.float32)
    qy = np.concatenate([np.float32([sy for _, sy, _ in spots]), w.qy]).astype(np.float32)
    for fp64 in (False, True):
        zq, al = _interp(aidw, x, y, z, qx, qy, k, fp64)
        _check(oracle, x, y, z, qx, qy, k, zq, al, TOL_FP64 if fp64 else TOL_FP32,
               1e-9 if fp64 else 1e-5)
        for i in range(len(spots)):
            mean = zs[1 + i].astype(np.float64).mean()
            assert abs(float(zq[i]) - mean) <= 1e-6 * max(1.0, abs(mean))
            assert float(al[i]) == 1.0


def test_constant_field_and_affine_map(aidw):
    w = inputs.uniform_kilo(n=20000, m=5000, seed=3)
    zq, _ = _interp(aidw, w.x, w.y, np.full(w.n, 7.5, np.float32), w.qx, w.qy, 10)
    np.testing.assert_allclose(zq, 7.5, rtol=1e-6)
    z1, _ = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10)
    z2, _ = _interp(aidw, w.x, w.y, (2.0 * w.z - 3.0).astype(np.float32), w.qx, w.qy, 10)
    np.testing.assert_allclose(z2, 2.0 * z1.astype(np.float64) - 3.0, rtol=0,
                               atol=2e-5 * np.abs(w.z).max())


def test_scale_and_translation_invariance(aidw):
    w = inputs.unit_square(5000, m=2000, seed=11)
    z1, a1 = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10)
    s = np.float32(16.0)     # exact power-of-two scaling
    z2, a2 = _interp(aidw, w.x * s, w.y * s, w.z, w.qx * s, w.qy * s, 10)
    np.testing.assert_allclose(a2, a1, atol=1e-6)
    np.testing.assert_allclose(z2, z1, rtol=0, atol=1e-5 * np.abs(w.z).max())
    t = np.float32(3.0)
    z3, _ = _interp(aidw, w.x + t, w.y + t, w.z, w.qx + t, w.qy + t, 10)
    np.testing.assert_allclose(z3, z1, rtol=0, atol=2e-3 * np.abs(w.z).max())


def test_result_does_not_depend_on_cell_width(aidw, oracle):
    """alpha comes from the kNN, which is exact whatever the cell width, so it
    is bit-identical; the width reorders the points, which changes only the
    rounding order of the compensated sums: every width is within the
    float32 tolerance of the oracle."""
    w = inputs.uniform_kilo(n=30000, m=4000, seed=12)
    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 10)
    base, a0 = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10, cell_scale=1.0)
    for c in (0.5, 1.0, 2.0, 4.0):
        got, a1 = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10, cell_scale=c)
        np.testing.assert_array_equal(a1, a0)
        assert oracle.normalized_error(got, ref["z"], ref["scale"]).max() <= TOL_FP32


def test_explicit_area_and_membership_bounds(aidw, oracle):
    w = inputs.uniform_kilo(n=8000, m=2000, seed=14)
    for area, r_min, r_max in ((2.0e6, 0.0, 2.0), (0.0, 0.5, 1.5), (5.0e5, 0.2, 3.0)):
        for fp64 in (False, True):
            zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10, fp64, area=area,
                             r_min=r_min, r_max=r_max)
            _check(oracle, w.x, w.y, w.z, w.qx, w.qy, 10, zq, al,
                   TOL_FP64 if fp64 else TOL_FP32, 1e-9 if fp64 else 1e-5,
                   area=area, r_min=r_min, r_max=r_max)


def test_empty_query_set(aidw):
    import torch
    w = inputs.unit_square(100, m=1, seed=1)
    p = aidw.Params()
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    zq, _ = aidw.aidw_interpolate(g, e, e, p)
    assert zq.numel() == 0
    g.destroy()


def test_nonfinite_query(aidw):
    w = inputs.unit_square(500, m=20, seed=1)
    qy = w.qy.copy()
    qy[5] = np.nan
    p = aidw.Params()
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    zq, _ = aidw.aidw_interpolate(g, dev(w.qx), dev(qy), p)
    zq = host(zq)
    assert np.isnan(zq[5]) and np.isfinite(np.delete(zq, 5)).all()
    assert aidw.aidw_grid_status(g) == 3
    g.destroy()


@pytest.mark.slow
@pytest.mark.parametrize("kind,k", [("uniform", 10), ("clustered", 10), ("clustered", 20)])
def test_full_size_sampled(aidw, oracle, kind, k):
    """n = m = 1,048,576 in [0,1000]^2 with every query on the GPU; the oracle
    checks a sample of 512 (float32 path) and the float64 path runs on a
    sample of 4096 queries."""
    w = inputs.uniform_kilo(seed=1) if kind == "uniform" else inputs.clustered_kilo(seed=2)
    zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, k)
    s = inputs.query_subsample(w.m, 512)
    _check(oracle, w.x, w.y, w.z, w.qx[s], w.qy[s], k, zq[s], al[s], TOL_FP32, 1e-5)
    s64 = inputs.query_subsample(w.m, 4096, seed=77)
    z64, a64 = _interp(aidw, w.x, w.y, w.z, w.qx[s64], w.qy[s64], k, fp64=True)
    s2 = np.arange(0, 4096, 32)
    _check(oracle, w.x, w.y, w.z, w.qx[s64][s2], w.qy[s64][s2], k, z64[s2], a64[s2],
           TOL_FP64, 1e-9)


def test_pipe_rate_probe(aidw):
    """The roofline denominator: SFU lg2/ex2 and packed-FMA lane rates."""
    r = aidw.aidw_probe_pipe_rates()
    assert r["lg2"] > 1 and r["ex2"] > 1 and r["ffma2_lanes"] > 1
    assert r["ex2"] >= 0.9 * r["lg2"]


def test_weight_loop_probe(aidw):
    """The weighting loop run alone: a positive rate no faster than its SFU
    ceiling allows (one lg2 and at least 3/4 of an ex2 per pair on the SFU),
    and argument checks."""
    r = aidw.aidw_probe_pipe_rates()
    ceiling = 1.0 / (1.0 / r["lg2"] + 0.75 / r["ex2"])
    for c in (2, 3):
        v = aidw.aidw_probe_weight_loop(c)
        assert 0.3 * ceiling < v <= 1.02 * ceiling, (c, v, ceiling)
    with pytest.raises(aidw.AidwError):
        aidw.aidw_probe_weight_loop(4)


@pytest.mark.slow
def test_precision_form_4M_sampled(aidw, oracle):
    """n = m = 4,194,304 uniform in [0,1000]^2: float32-compensated path on
    every query, float64 GPU path on the first 16,384 queries (compared with
    the float32 path on all of them), oracle on samples of both."""
    w = inputs.uniform_kilo(n=1 << 22, seed=3)
    zq, al = _interp(aidw, w.x, w.y, w.z, w.qx, w.qy, 10)
    s = inputs.query_subsample(w.m, 128)
    _check(oracle, w.x, w.y, w.z, w.qx[s], w.qy[s], 10, zq[s], al[s], TOL_FP32, 1e-5)
    q = 16384
    z64, a64 = _interp(aidw, w.x, w.y, w.z, w.qx[:q], w.qy[:q], 10, fp64=True)
    # float64 GPU path against the oracle
    s2 = np.arange(0, q, 256)
    ref = _check(oracle, w.x, w.y, w.z, w.qx[s2], w.qy[s2], 10, z64[s2], a64[s2], TOL_FP64, 1e-9)
    assert ref <= TOL_FP64
    # float32 path against the float64 GPU path on all q queries, scaled by
    # S_q = sum w|z| / sum w, which is Eq. 1 applied to |z| (same weights;
    # the float32 path gives it to about 1e-6 relative)
    s_abs, _ = _interp(aidw, w.x, w.y, np.abs(w.z), w.qx[:q], w.qy[:q], 10)
    err = np.abs(zq[:q].astype(np.float64) - z64) / s_abs.astype(np.float64)
    assert err.max() <= TOL_FP32, err.max()


@pytest.mark.parametrize("fp64", [False, True])
def test_interpolate_from_host_arrays(aidw, oracle, fp64):
    """aidw_interpolate_host (copies in, grid build, interpolation, copies
    out, all inside the library) gives exactly the device-array path's
    predictions and alphas, from pageable numpy arrays and pinned tensors."""
    import torch
    w = inputs.clustered_kilo(n=15000, m=3000, k=12, seed=71)
    p = aidw.Params(k=12, precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    ref_z, ref_a = aidw.aidw_interpolate(g, dev(w.qx), dev(w.qy), p, want_alpha=True)
    g.destroy()
    z, a = aidw.interpolate_host(w.x, w.y, w.z, w.qx, w.qy, p, want_alpha=True)
    np.testing.assert_array_equal(z.numpy(), host(ref_z))
    np.testing.assert_array_equal(a.numpy(), host(ref_a))
    pinned = [torch.from_numpy(getattr(w, k)).pin_memory() for k in ("x", "y", "z", "qx", "qy")]
    z2 = aidw.interpolate_host(*pinned, p)
    np.testing.assert_array_equal(z2.numpy(), host(ref_z))
    ref = oracle.aidw(w.x, w.y, w.z, w.qx[:300], w.qy[:300], 12)
    err = oracle.normalized_error(z.numpy()[:300], ref["z"], ref["scale"])
    assert err.max() <= (TOL_FP64 if fp64 else TOL_FP32)
    assert aidw.interpolate_host(w.x, w.y, w.z, w.qx[:0], w.qy[:0], p).numel() == 0
