"""The cell index floor((x - minX) / cw) of the even grid (Sec. 3.2.2) is
taken on the GPU as floor(a * fl(1/cw)) unless that product lies within
2^-49 |q| of an integer, where the float64 division is used instead.  This
checks, in float64 numpy arithmetic (IEEE, no fused operations), that the
rule gives exactly floor of the correctly rounded quotient on random,
lattice and near-edge inputs."""
import numpy as np


def _fast_floor(a, cw):
    inv = 1.0 / cw
    q = a * inv
    f = np.floor(q)
    tol = np.abs(q) * 2.0 ** -49
    near = ~((q - f > tol) & ((f + 1.0) - q > tol))
    return np.where(near, np.floor(a / cw), f), near


def _check(a, cw):
    got, near = _fast_floor(a, cw)
    np.testing.assert_array_equal(got, np.floor(a / cw))
    return near.mean()


def test_random_widths_and_offsets():
    rng = np.random.default_rng(0)
    for _ in range(200):
        cw = float(rng.uniform(1e-3, 10.0)) * 10.0 ** float(rng.integers(-3, 4))
        a = rng.uniform(0.0, 5000.0 * cw, 20000).astype(np.float32).astype(np.float64)
        assert _check(a, cw) < 1e-3


def test_points_on_and_next_to_cell_edges():
    rng = np.random.default_rng(1)
    for cw in (1.0, 0.5, 0.49, 0.1, 1.0 / 3.0, 0.49 * (100 / 49), 1000.0 / 1024.0):
        k = np.arange(0, 4096, dtype=np.float64)
        edge = k * cw
        a = np.concatenate([edge, np.nextafter(edge, -np.inf), np.nextafter(edge, np.inf),
                            edge.astype(np.float32).astype(np.float64)])
        a = a[a >= 0.0]
        _check(a, cw)
        jitter = edge * (1.0 + rng.uniform(-4e-16, 4e-16, edge.size))
        _check(jitter[jitter >= 0.0], cw)


def test_integer_lattice_with_unit_width_uses_the_division():
    a = np.arange(0, 1000, dtype=np.float64)
    got, near = _fast_floor(a, 1.0)
    np.testing.assert_array_equal(got, a)
    assert near[1:].all()          # exact integers always take the division
