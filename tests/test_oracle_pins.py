"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a hand-derived
closed form (tests/golden), a library routine that computes the same
special case (scipy's k-d tree for kNN, numpy's piecewise-linear interp for
Eq. 6), an invariant of Eq. 1, or a statistical law (Clark-Evans for Eq. 2).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1601_05904_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "aidw_hand_cases.json")


def _eval_closed_form(s: str) -> float:
    if "sqrt" in s:
        return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt}))
    return float(Fraction(s))


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_derived_cases(oracle, case):
    out = oracle.aidw(case["x"], case["y"], case["z"], case["qx"], case["qy"], case["k"],
                      levels=case["levels"], r_min=case["r_min"], r_max=case["r_max"])
    want = [_eval_closed_form(s) for s in case["expected_z"]]
    np.testing.assert_allclose(out["z"], want, rtol=1e-13, atol=1e-13)
    if case["expected_alpha"] is not None:
        want_a = [_eval_closed_form(s) for s in case["expected_alpha"]]
        np.testing.assert_allclose(out["alpha"], want_a, rtol=1e-12, atol=1e-12)


# ---- Eq. 2 ---------------------------------------------------------------

@pytest.mark.parametrize("n,area,want", [(100, 100.0, 0.5), (4, 1.0, 0.25), (1, 4.0, 1.0),
                                         (10 ** 6, 10 ** 6, 0.5), (16, 0.0, 0.0)])
def test_r_exp_closed_form(oracle, n, area, want):
    assert oracle.r_exp(n, area) == pytest.approx(want, rel=1e-15, abs=0)


def test_r_exp_matches_clark_evans_for_uniform_points(oracle):
    """For uniform points the mean distance from a random location to its
    nearest data point is 1/(2 sqrt(density)) up to edge effects (Eq. 2)."""
    rng = np.random.default_rng(7)
    x, y = inputs.uniform_points(rng, 20000, 0.0, 1.0)
    qx, qy = inputs.uniform_points(rng, 1000, 0.05, 0.95)  # away from the edges
    _, d = oracle.knn(x, y, qx, qy, 1)
    assert d[:, 0].mean() == pytest.approx(oracle.r_exp(20000, 1.0), rel=0.05)


# ---- Eq. 3 / 4 -------------------------------------------------------------

def test_r_obs_is_the_mean(oracle):
    assert oracle.r_obs([1.0, 2.0, 6.0]) == 3.0
    assert oracle.r_obs([0.25]) == 0.25


def test_R_cases(oracle):
    assert oracle.R(1.0, 0.5) == 2.0
    assert oracle.R(0.0, 0.5) == 0.0
    assert oracle.R(0.0, 0.0) == 0.0
    assert math.isinf(oracle.R(1.0, 0.0))


# ---- Eq. 5 -----------------------------------------------------------------

def test_mu_closed_forms(oracle):
    assert oracle.mu(1.0, 0.0, 2.0) == pytest.approx(0.5, abs=1e-15)
    assert oracle.mu(2.0 / 3.0, 0.0, 2.0) == pytest.approx(0.25, abs=1e-15)   # cos(pi/3)
    assert oracle.mu(4.0 / 3.0, 0.0, 2.0) == pytest.approx(0.75, abs=1e-15)   # cos(2pi/3)
    assert oracle.mu(0.0, 0.0, 2.0) == 0.0
    assert oracle.mu(-1.0, 0.0, 2.0) == 0.0
    assert oracle.mu(2.0, 0.0, 2.0) == 1.0
    assert oracle.mu(7.0, 0.0, 2.0) == 1.0
    # R_min shifts the argument; the printed pi/R_max factor stays
    assert oracle.mu(1.5, 0.5, 2.0) == pytest.approx(0.5, abs=1e-15)


def test_mu_is_monotone_and_bounded(oracle):
    Rs = np.linspace(-0.5, 2.5, 301)
    m = np.array([oracle.mu(r) for r in Rs])
    assert (np.diff(m) >= 0).all()
    assert m.min() == 0.0 and m.max() == 1.0


# ---- Eq. 6 -----------------------------------------------------------------

@pytest.mark.parametrize("levels", [(1, 2, 3, 4, 5), (0.5, 1, 2, 3, 4), (5, 1, 4, 2, 3)])
def test_alpha_is_piecewise_linear_through_the_knots(oracle, levels):
    """Eq. 6 is the linear interpolation through (0.1, a1) ... (0.9, a5),
    flat outside: exactly what numpy.interp computes."""
    knots = np.array([0.1, 0.3, 0.5, 0.7, 0.9])
    for m in np.linspace(0.0, 1.0, 1001):
        want = float(np.interp(m, knots, np.asarray(levels, dtype=np.float64)))
        assert oracle.alpha(m, levels) == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_alpha_at_knots_and_midpoints(oracle):
    lv = (1.0, 2.0, 3.0, 4.0, 5.0)
    for j, m in enumerate((0.1, 0.3, 0.5, 0.7, 0.9)):
        assert oracle.alpha(m, lv) == pytest.approx(lv[j], abs=1e-14)
    assert oracle.alpha(0.2, lv) == pytest.approx(1.5, abs=1e-14)
    assert oracle.alpha(0.8, lv) == pytest.approx(4.5, abs=1e-14)


def test_knot_mu_maps_back_through_eq5(oracle):
    """R = (R_max/pi) acos(1 - 2 mu) inverts Eq. 5; at the knots alpha is a level."""
    lv = (1.0, 2.0, 3.0, 4.0, 5.0)
    for j, m in enumerate((0.1, 0.3, 0.5, 0.7, 0.9)):
        R = (2.0 / math.pi) * math.acos(1.0 - 2.0 * m)
        assert oracle.alpha(oracle.mu(R), lv) == pytest.approx(lv[j], abs=1e-12)


# ---- Sec. 2.3 brute-force kNN -----------------------------------------------

@pytest.mark.parametrize("k", [1, 5, 10, 32])
def test_knn_matches_scipy_kdtree(oracle, k):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(11)
    x, y = inputs.uniform_points(rng, 3000, 0.0, 1000.0)
    qx, qy = inputs.uniform_points(rng, 400, -50.0, 1050.0)
    idx, dist = oracle.knn(x, y, qx, qy, k)
    tree = spatial.cKDTree(np.stack([x, y], 1).astype(np.float64))
    d_ref, i_ref = tree.query(np.stack([qx, qy], 1).astype(np.float64), k=k)
    d_ref = np.asarray(d_ref).reshape(len(qx), k)
    i_ref = np.asarray(i_ref).reshape(len(qx), k)
    np.testing.assert_allclose(dist, d_ref, rtol=1e-12)
    # random float data: no exact distance ties, so the index lists agree
    np.testing.assert_array_equal(idx, i_ref)


def test_knn_ties_break_by_index(oracle):
    x = [1, -1, 0, 0, 3]
    y = [0, 0, 1, -1, 0]
    idx, dist = oracle.knn(x, y, [0.0], [0.0], 4)
    assert idx.tolist() == [[0, 1, 2, 3]]
    assert dist.tolist() == [[1.0, 1.0, 1.0, 1.0]]


def test_knn_k_equals_n_sorts_everything(oracle):
    rng = np.random.default_rng(3)
    x, y = inputs.uniform_points(rng, 50, 0.0, 1.0)
    idx, dist = oracle.knn(x, y, [0.5], [0.5], 50)
    assert sorted(idx[0].tolist()) == list(range(50))
    assert (np.diff(dist[0]) >= 0).all()


# ---- Eq. 1 invariants ---------------------------------------------------------

def _small(seed=5, n=700, m=300):
    w = inputs.unit_square(n=n, m=m, k=10, seed=seed)
    return w


def test_constant_field_is_reproduced(oracle):
    w = _small()
    out = oracle.aidw(w.x, w.y, np.full(w.n, 3.25, np.float32), w.qx, w.qy, w.k)
    np.testing.assert_allclose(out["z"], 3.25, rtol=1e-14)


def test_affine_map_commutes(oracle):
    w = _small()
    a, b = -2.5, 7.0
    z1 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)["z"]
    z2 = oracle.aidw(w.x, w.y, (a * w.z.astype(np.float64) + b).astype(np.float32),
                     w.qx, w.qy, w.k)["z"]
    # the affine map itself is rounded to float32 on the inputs
    np.testing.assert_allclose(z2, a * z1 + b, rtol=0, atol=1e-5)


def test_predictions_stay_within_data_range(oracle):
    w = _small()
    out = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)
    assert out["z"].min() >= w.z.min() - 1e-12
    assert out["z"].max() <= w.z.max() + 1e-12


def test_alpha_within_levels(oracle):
    w = _small()
    for lv in [(1, 2, 3, 4, 5), (0.5, 1, 2, 3, 4), (4, 3, 2, 1, 0.5)]:
        a = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k, levels=lv)["alpha"]
        assert a.min() >= min(lv) - 1e-12 and a.max() <= max(lv) + 1e-12


def test_query_on_data_point_returns_its_value(oracle):
    w = _small()
    sel = np.arange(0, w.n, 37)
    out = oracle.aidw(w.x, w.y, w.z, w.x[sel], w.y[sel], w.k)
    np.testing.assert_array_equal(out["z"], w.z[sel].astype(np.float64))


def test_single_data_point(oracle):
    out = oracle.aidw([0.3], [0.7], [4.5], [0.0, 1.0, 0.3], [0.0, 5.0, 0.7], 1)
    np.testing.assert_array_equal(out["z"], [4.5, 4.5, 4.5])


def test_symmetric_pair_gives_the_average(oracle):
    out = oracle.aidw([0.0, 2.0], [0.0, 0.0], [1.0, 4.0], [1.0, 1.0], [0.0, 3.0], 1)
    np.testing.assert_allclose(out["z"], [2.5, 2.5], rtol=1e-15)


def test_eq1_sums_over_all_points_not_only_knn(oracle):
    """With k = 1 the prediction still feels every point (Eq. 1 runs over
    all n data points): two far points change it."""
    base = oracle.aidw([0.0, 10.0], [0.0, 0.0], [0.0, 1.0], [1.0], [0.0], 1,
                       levels=(2, 2, 2, 2, 2))["z"][0]
    # by hand: w = 1, 1/81 -> z = (1/81)/(82/81) = 1/82
    assert base == pytest.approx(1.0 / 82.0, rel=1e-14)


def test_power_of_two_scaling_invariance(oracle):
    """Scaling all coordinates by s scales r_obs and r_exp alike, so R, alpha
    and the normalised weights do not change (s = 8 is exact in float32)."""
    w = _small()
    s = np.float32(8.0)
    o1 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)
    o2 = oracle.aidw(w.x * s, w.y * s, w.z, w.qx * s, w.qy * s, w.k)
    np.testing.assert_allclose(o2["alpha"], o1["alpha"], rtol=1e-12)
    np.testing.assert_allclose(o2["z"], o1["z"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(o2["r_obs"], 8.0 * o1["r_obs"], rtol=1e-14)


def test_translation_invariance(oracle):
    w = _small()
    t = np.float32(16.0)
    o1 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)
    o2 = oracle.aidw(w.x + t, w.y + t, w.z, w.qx + t, w.qy + t, w.k)
    # the shifted coordinates are rounded to float32, so distances move by
    # about one float32 ulp of 17 relative to spacings of ~0.02
    np.testing.assert_allclose(o2["z"], o1["z"], rtol=0, atol=5e-4 * np.abs(w.z).max())


def test_area_override_changes_only_alpha(oracle):
    w = _small()
    o1 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k, area=1.0)
    o2 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k, area=4.0)
    # quadrupling A doubles r_exp and halves R: alpha moves down
    assert (o2["alpha"] <= o1["alpha"] + 1e-12).all()
    assert (o2["alpha"] < o1["alpha"]).any()


# ---- even grid (Sec. 3.2.1-3.2.3) -----------------------------------------------

@pytest.mark.parametrize("cell_scale", [0.5, 1.0, 2.0, 4.0])
def test_grid_invariants(oracle, cell_scale):
    w = inputs.clustered_kilo(n=5000, m=10, seed=9)
    g = oracle.grid(w.x, w.y, cell_scale=cell_scale)
    n = w.n
    ncells = g["ncol"] * g["nrow"]
    st = g["cell_start"]
    assert st[0] == 0 and st[-1] == n and (np.diff(st) >= 0).all()
    perm = g["perm"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    key = g["key"]
    # counts are the histogram of keys (segmented reduce in Fig. 3a)
    np.testing.assert_array_equal(np.diff(st), np.bincount(key, minlength=ncells))
    # cell order, stable within a cell
    kp = key[perm]
    assert (np.diff(kp) >= 0).all()
    same = np.diff(kp) == 0
    assert (np.diff(perm)[same] > 0).all()
    # every point lies inside its cell (closed at the clamped far edges)
    col, row = key % g["ncol"], key // g["ncol"]
    x0 = g["min_x"] + col * g["cw"]
    y0 = g["min_y"] + row * g["cw"]
    xd, yd = w.x.astype(np.float64), w.y.astype(np.float64)
    assert (xd >= x0 - 1e-9).all() and (yd >= y0 - 1e-9).all()
    assert ((xd <= x0 + g["cw"] + 1e-9) | (col == g["ncol"] - 1)).all()
    assert ((yd <= y0 + g["cw"] + 1e-9) | (row == g["nrow"] - 1)).all()


def test_grid_dims_follow_eq2(oracle):
    rng = np.random.default_rng(1)
    x, y = inputs.uniform_points(rng, 10000, 0.0, 1000.0)
    g = oracle.grid(x, y, cell_scale=1.0)
    W = float(x.max()) - float(x.min())
    H = float(y.max()) - float(y.min())
    assert g["area"] == W * H
    assert g["r_exp"] == pytest.approx(1.0 / (2.0 * math.sqrt(10000 / (W * H))), rel=1e-15)
    assert g["cw"] == g["r_exp"]
    # the paper's nCol = (maxX - minX + cw) / cw
    assert g["ncol"] == int((W + g["cw"]) / g["cw"])
    assert g["nrow"] == int((H + g["cw"]) / g["cw"])


def test_grid_degenerate_boxes(oracle):
    # collinear points: zero area, 1-D fallback spacing, one row
    g = oracle.grid(np.linspace(0, 10, 101), np.zeros(101), cell_scale=1.0)
    assert g["nrow"] == 1 and g["r_exp"] == 0.0 and g["cw"] > 0
    assert g["cell_start"][-1] == 101
    # all points identical: a single cell
    g = oracle.grid(np.full(7, 3.0), np.full(7, -2.0))
    assert g["ncol"] == 1 and g["nrow"] == 1
    assert g["perm"].tolist() == list(range(7))


# ---- local AIDW (Eq. 1 over the k nearest points) --------------------------------

def _local_cases():
    with open(GOLDEN) as f:
        return json.load(f)["local_cases"]


@pytest.mark.parametrize("case", _local_cases(), ids=lambda c: c["name"])
def test_local_hand_derived_cases(oracle, case):
    out = oracle.aidw_local(case["x"], case["y"], case["z"], case["qx"], case["qy"], case["k"],
                            levels=case["levels"], r_min=case["r_min"], r_max=case["r_max"])
    want = [_eval_closed_form(s) for s in case["expected_z"]]
    np.testing.assert_allclose(out["z"], want, rtol=1e-13)


def test_local_with_k_equal_n_is_the_all_points_form(oracle):
    w = inputs.unit_square(32, m=200, seed=3)
    a = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 32)
    b = oracle.aidw_local(w.x, w.y, w.z, w.qx, w.qy, 32)
    np.testing.assert_allclose(b["z"], a["z"], rtol=1e-12)
    np.testing.assert_array_equal(b["alpha"], a["alpha"])


def test_local_alpha_matches_all_points_alpha(oracle):
    w = _small()
    a = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 10)
    b = oracle.aidw_local(w.x, w.y, w.z, w.qx, w.qy, 10)
    np.testing.assert_array_equal(b["alpha"], a["alpha"])
    # a local average stays within the range of the k neighbours' values
    idx, _ = oracle.knn(w.x, w.y, w.qx, w.qy, 10)
    zn = w.z[idx].astype(np.float64)
    assert (b["z"] >= zn.min(1) - 1e-12).all() and (b["z"] <= zn.max(1) + 1e-12).all()


def test_local_constant_field_and_hits(oracle):
    w = _small()
    out = oracle.aidw_local(w.x, w.y, np.full(w.n, -1.5, np.float32), w.qx, w.qy, 8)
    np.testing.assert_allclose(out["z"], -1.5, rtol=1e-14)
    sel = np.arange(0, w.n, 41)
    out = oracle.aidw_local(w.x, w.y, w.z, w.x[sel], w.y[sel], 8)
    np.testing.assert_array_equal(out["z"], w.z[sel].astype(np.float64))


# ---- grid kNN with the paper's level rule (Sec. 3.2.4) -------------------------
PAPER_RULE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "knn_paper_rule_cases.json")


def _paper_rule_cases():
    with open(PAPER_RULE_GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _paper_rule_cases(), ids=lambda c: c["name"])
def test_paper_rule_hand_derived_cases(oracle, case):
    g = oracle.grid(case["x"], case["y"], cell_scale=case["cell_scale"])
    assert (g["cw"], g["ncol"], g["nrow"]) == (1.0, 11, 11)
    idx, _ = oracle.knn_paper_rule(case["x"], case["y"], case["qx"], case["qy"], case["k"],
                                   cell_scale=case["cell_scale"])
    np.testing.assert_array_equal(idx, case["expected_paper_rule_idx"])
    idx, _ = oracle.knn(case["x"], case["y"], case["qx"], case["qy"], case["k"])
    np.testing.assert_array_equal(idx, case["expected_exact_idx"])


@pytest.mark.parametrize("seed,cell_scale,k", [(0, 1.0, 10), (1, 0.5, 5), (2, 2.0, 20)])
def test_paper_rule_never_beats_the_exact_knn(oracle, seed, cell_scale, k):
    """The rule picks the k best of a subset of the points, so its j-th
    distance is never below the exact j-th distance; where the two index
    lists agree, the distances agree exactly."""
    w = inputs.clustered_kilo(n=3000, m=800, k=k, seed=seed)
    pi, pd = oracle.knn_paper_rule(w.x, w.y, w.qx, w.qy, k, cell_scale=cell_scale)
    ei, ed = oracle.knn(w.x, w.y, w.qx, w.qy, k)
    assert (pd >= ed).all()
    same = (pi == ei).all(1)
    np.testing.assert_array_equal(pd[same], ed[same])
    assert same.mean() > 0.5


def test_paper_rule_is_exact_when_the_block_covers_the_grid(oracle):
    """With a few large cells the widened block is the whole grid, and the
    rule reduces to the brute-force kNN."""
    w = inputs.unit_square(200, m=300, seed=4)
    g = oracle.grid(w.x, w.y, cell_scale=20.0)
    assert g["ncol"] <= 2 and g["nrow"] <= 2     # level 1 spans the grid from any cell
    pi, pd = oracle.knn_paper_rule(w.x, w.y, w.qx, w.qy, 7, cell_scale=20.0)
    ei, ed = oracle.knn(w.x, w.y, w.qx, w.qy, 7)
    np.testing.assert_array_equal(pi, ei)
    np.testing.assert_array_equal(pd, ed)
