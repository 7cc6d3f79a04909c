"""Seeded random configurations of the whole method (Sec. 2.2, Eq. 1-6, the
grid kNN of Sec. 3.2) against the oracle: data size and layout, query count,
k, the five alpha levels (any positive values, in any order), R_min/R_max,
an explicit area, the cell width, both precision forms.  Each case checks the
predictions (normalised error) and alpha.

Where R_min > 0, Eq. 5 as printed jumps at R = R_max (reading Z4), and the
float32 path takes the R >= R_max test in float32: queries whose R lies
within 1e-5 of R_max are left out of that case's alpha and z comparison."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 20000))
    m = int(rng.integers(1, 3000))
    k = int(rng.integers(1, min(32, n) + 1))
    lo, hi = (0.0, 1000.0) if rng.random() < 0.5 else (-50.0, 50.0)
    frac = float(rng.uniform(0.0, 0.9)) if rng.random() < 0.5 else 0.0
    if frac > 0:
        x, y = inputs.mixed_points(rng, n, frac, int(rng.integers(1, 9)))
        x = (lo + (x / 1000.0) * (hi - lo)).astype(np.float32)
        y = (lo + (y / 1000.0) * (hi - lo)).astype(np.float32)
    else:
        x, y = inputs.uniform_points(rng, n, lo, hi)
    z = inputs.field_kilo(rng, x, y)
    qx, qy = inputs.uniform_points(rng, m, lo, hi)
    levels = tuple(float(v) for v in rng.uniform(0.2, 6.0, 5))
    r_min = float(rng.uniform(0.0, 1.0)) if rng.random() < 0.5 else 0.0
    r_max = float(rng.uniform(r_min + 0.2, 4.0))
    area = float(rng.uniform(0.5, 2.0) * (hi - lo) ** 2) if rng.random() < 0.3 else 0.0
    cell_scale = float(rng.uniform(0.3, 6.0)) if rng.random() < 0.5 else 0.0
    return dict(x=x, y=y, z=z, qx=qx, qy=qy, k=k, levels=levels, r_min=r_min, r_max=r_max,
                area=area, cell_scale=cell_scale)


@pytest.mark.parametrize("seed", range(24))
def test_random_configuration(aidw, oracle, seed):
    c = _case(7000 + seed)
    ref = oracle.aidw(c["x"], c["y"], c["z"], c["qx"], c["qy"], c["k"], levels=c["levels"],
                      r_min=c["r_min"], r_max=c["r_max"], area=c["area"])
    keep = np.ones(len(c["qx"]), bool)
    if c["r_min"] > 0.0:
        area = c["area"] if c["area"] > 0 else \
            (float(c["x"].max()) - float(c["x"].min())) * (float(c["y"].max()) - float(c["y"].min()))
        r_exp = oracle.r_exp(len(c["x"]), area)
        if r_exp > 0:
            keep = np.abs(ref["r_obs"] / r_exp - c["r_max"]) > 1e-5 * c["r_max"]
    for fp64 in (False, True):
        p = aidw.Params(k=c["k"], alpha=c["levels"], r_min=c["r_min"], r_max=c["r_max"],
                        area=c["area"], cell_scale=c["cell_scale"],
                        precision=aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP)
        g = aidw.aidw_grid_build(dev(c["x"]), dev(c["y"]), dev(c["z"]), p)
        zq, al = aidw.aidw_interpolate(g, dev(c["qx"]), dev(c["qy"]), p, want_alpha=True)
        assert aidw.aidw_grid_status(g) == 0
        g.destroy()
        err = oracle.normalized_error(host(zq), ref["z"], ref["scale"])[keep]
        assert err.max(initial=0.0) <= (TOL_FP64 if fp64 else TOL_FP32), err.max()
        np.testing.assert_allclose(host(al).astype(np.float64)[keep], ref["alpha"][keep],
                                   rtol=0, atol=1e-9 if fp64 else 1e-5)
