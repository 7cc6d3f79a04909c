"""Even-grid build (Sec. 3.2.1-3.2.3): the GPU grid equals the oracle's CPU
grid exactly - dimensions, cell heads and the stable cell-ordered permutation."""
import numpy as np
import pytest

from gpu_helpers import dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _compare(aidw, oracle, x, y, cell_scale, area=0.0):
    p = aidw.Params(cell_scale=cell_scale, area=area)
    g = aidw.aidw_grid_build(dev(x), dev(y), dev(np.zeros_like(x)), p)
    info = aidw.aidw_grid_get_info(g)
    cs, perm = aidw.aidw_grid_export(g)
    ref = oracle.grid(x, y, cell_scale=cell_scale, area=area)
    for a, b in (("min_x", "min_x"), ("min_y", "min_y"), ("max_x", "max_x"),
                 ("max_y", "max_y"), ("area", "area"), ("r_exp", "r_exp"),
                 ("cell_width", "cw")):
        assert info[a] == ref[b], (a, info[a], ref[b])
    assert info["n_col"] == ref["ncol"] and info["n_row"] == ref["nrow"]
    np.testing.assert_array_equal(host(cs), ref["cell_start"])
    np.testing.assert_array_equal(host(perm).astype(np.int64), ref["perm"])
    assert aidw.aidw_grid_status(g) == 0
    g.destroy()
    return info


@pytest.mark.parametrize("cell_scale", [0.5, 1.0, 2.0, 4.0])
def test_grid_uniform_unit(aidw, oracle, cell_scale):
    w = inputs.unit_square(4096, seed=0)
    _compare(aidw, oracle, w.x, w.y, cell_scale)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1000, 4097, 65537])
def test_grid_ragged_sizes(aidw, oracle, n):
    rng = np.random.default_rng(n)
    x, y = inputs.uniform_points(rng, n, 0.0, 1000.0)
    _compare(aidw, oracle, x, y, 1.0)


def test_grid_clustered(aidw, oracle):
    w = inputs.clustered_kilo(n=200000, m=1, seed=2)
    _compare(aidw, oracle, w.x, w.y, 1.0)
    _compare(aidw, oracle, w.x, w.y, 2.0)


def test_grid_beyond_l2_size(aidw, oracle):
    """Point sets whose sort arrays (16-byte records, cell heads, keys) are
    larger than the 129 MB L2, where the scatter and the fix-up work out of
    DRAM: 8M uniform points (about one per cell) and 4M clustered points
    (long cell segments for the stable fix-up)."""
    rng = np.random.default_rng(8)
    x, y = inputs.uniform_points(rng, 1 << 23, 0.0, 1000.0)
    _compare(aidw, oracle, x, y, 2.0)
    w = inputs.clustered_kilo(n=1 << 22, m=1, seed=9)
    _compare(aidw, oracle, w.x, w.y, 1.0)


def test_grid_duplicates_and_cell_boundaries(aidw, oracle):
    # integer lattice with repeats: many points exactly on cell edges
    rng = np.random.default_rng(4)
    x = rng.integers(0, 50, 5000).astype(np.float32)
    y = rng.integers(0, 50, 5000).astype(np.float32)
    for c in (0.5, 1.0, 3.0):
        _compare(aidw, oracle, x, y, c)


@pytest.mark.parametrize("cell_scale", [100 / 49, 50 / 49, 200 / 49, 1.0, 0.5])
def test_grid_lattice_on_cell_edges(aidw, oracle, cell_scale):
    # a 50 x 50 integer lattice has r_exp = 49 / 100, so these scales give
    # cell widths at or within rounding of 1, 1/2, 2: most coordinates fall
    # on a cell edge or within a float64 rounding of one, where the cell
    # index must still equal the floor of the correctly rounded quotient
    g = np.arange(50, dtype=np.float32)
    x, y = np.meshgrid(g, g)
    x, y = x.ravel(), y.ravel()
    rng = np.random.default_rng(9)
    extra = rng.integers(0, 2500, 700)
    x, y = np.concatenate([x, x[extra]]), np.concatenate([y, y[extra]])
    _compare(aidw, oracle, x, y, cell_scale)


def test_grid_degenerate_boxes(aidw, oracle):
    x = np.linspace(0, 10, 1001, dtype=np.float32)
    _compare(aidw, oracle, x, np.zeros_like(x), 1.0)           # collinear
    _compare(aidw, oracle, np.full(50, 3.0, np.float32), np.full(50, -2.0, np.float32), 1.0)
    # elongated box: the cell cap doubles the width
    rng = np.random.default_rng(8)
    xs, ys = inputs.uniform_points(rng, 20000, 0.0, 1.0)
    info = _compare(aidw, oracle, xs * np.float32(4096.0), ys * np.float32(0.001), 1.0)
    assert info["n_cells"] <= 4 * 20000 + 16 * 20000 ** 0.5 + 16


def test_grid_explicit_area(aidw, oracle):
    w = inputs.unit_square(3000, seed=3)
    _compare(aidw, oracle, w.x, w.y, 1.0, area=2.0)


def test_grid_rejects_nonfinite(aidw):
    x = np.linspace(0, 1, 100, dtype=np.float32)
    y = x.copy()
    y[17] = np.nan
    with pytest.raises(aidw.AidwError) as e:
        aidw.aidw_grid_build(dev(x), dev(y), dev(x), aidw.Params())
    assert e.value.status == 3
