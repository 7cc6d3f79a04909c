"""The grid kNN with the paper's own level rule (Sec. 3.2.4, Step 2 and the
remark on Fig. 4) against the oracle's statement of the same rule, and its
relation to the exact kNN: the hand-derived cases of the golden file, a
random parity check on the same grids, and the subset property (the rule
chooses among fewer points, so none of its distances beats the exact one)."""
import json
import os

import numpy as np
import pytest

from gpu_helpers import check_knn, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "knn_paper_rule_cases.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _f32(a):
    return np.asarray(a, dtype=np.float32)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_derived_cases(aidw, case):
    x, y = _f32(case["x"]), _f32(case["y"])
    qx, qy = _f32(case["qx"]), _f32(case["qy"])
    p = aidw.Params(k=case["k"], cell_scale=case["cell_scale"])
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(np.zeros_like(x)), p)
    info = aidw.aidw_grid_get_info(g)
    assert (info["cell_width"], info["n_col"], info["n_row"]) == (1.0, 11, 11)
    ip, _, _ = aidw.aidw_knn_paper_rule(g, dev(qx), dev(qy), case["k"])
    ie, _, _ = aidw.aidw_knn(g, dev(qx), dev(qy), case["k"])
    np.testing.assert_array_equal(host(ip), case["expected_paper_rule_idx"])
    np.testing.assert_array_equal(host(ie), case["expected_exact_idx"])
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()


@pytest.mark.parametrize("gen,k,cell_scale", [
    ("uniform", 10, 1.0), ("uniform", 10, 2.0), ("clustered", 10, 1.0),
    ("clustered", 20, 3.0), ("clustered", 32, 0.5), ("uniform", 1, 1.0)])
def test_matches_the_oracle_rule(aidw, oracle, gen, k, cell_scale):
    mk = inputs.uniform_kilo if gen == "uniform" else inputs.clustered_kilo
    w = mk(n=20000, m=4000, k=k, seed=81)
    p = aidw.Params(k=k, cell_scale=cell_scale)
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), p)
    ip, dp, rp = aidw.aidw_knn_paper_rule(g, dev(w.qx), dev(w.qy), k)
    ie, de, _ = aidw.aidw_knn(g, dev(w.qx), dev(w.qy), k)
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    ref = oracle.knn_paper_rule(w.x, w.y, w.qx, w.qy, k, cell_scale=cell_scale, n_out=k + 1)
    check_knn(oracle, w.x, w.y, w.qx, w.qy, k, host(ip), host(dp), host(rp), ref=ref)
    # both searches use the same float32 distances and order: the rule's
    # j-th distance is never below the exact one, and equal lists mean the
    # rule found every neighbour
    dp, de = host(dp), host(de)
    assert (dp >= de).all()
    same = (host(ip) == host(ie)).all(1)
    np.testing.assert_array_equal(dp[same], de[same])


def test_nonfinite_query_is_reported(aidw):
    w = inputs.uniform_kilo(n=5000, m=100, seed=82)
    qx = w.qx.copy()
    qx[7] = np.nan
    g = aidw.aidw_grid_build(dev(w.x), dev(w.y), dev(w.z), aidw.Params(k=5))
    ip, dp, rp = aidw.aidw_knn_paper_rule(g, dev(qx), dev(w.qy), 5)
    assert aidw.aidw_grid_status(g) == 3
    ip = host(ip)
    assert (ip[7] == -1).all() and np.isnan(host(dp)[7]).all() and np.isnan(host(rp)[7])
    assert (ip[np.arange(100) != 7] >= 0).all()
    g.destroy()
