"""The cell index floor((x - minX) / cw) of the even grid (Sec. 3.2.2) is
defined on float64 (the difference of the float32 inputs, correctly rounded
quotient).  The GPU takes it in float32 - q = fl32(fl32(x - minX) *
fl32(1/cw)) - unless q lies within 2^-21 |q| of an integer, where it falls
back to the float64 division.  This checks, in IEEE float32 / float64 numpy
arithmetic (no fused operations), that the rule gives exactly the defined
floor on random, lattice and near-edge inputs, and that the fallback stays
rare on ordinary data."""
import numpy as np


def _rule(x32, min32, cw):
    inv = np.float32(1.0 / cw)
    q = (x32 - min32) * inv                       # float32 sub, then float32 mul
    f = np.floor(q)
    tol = np.abs(q) * np.float32(2.0 ** -21)
    near = ~(((q - f) > tol) & (((f + np.float32(1.0)) - q) > tol))
    exact = np.floor((x32.astype(np.float64) - np.float64(min32)) / cw)
    return np.where(near, exact, f.astype(np.float64)), exact, near


def _check(x32, min32, cw):
    got, exact, near = _rule(np.asarray(x32, np.float32), np.float32(min32), float(cw))
    np.testing.assert_array_equal(got, exact)
    return near.mean()


def test_random_widths_and_offsets():
    rng = np.random.default_rng(0)
    for _ in range(200):
        cw = float(rng.uniform(1e-3, 10.0)) * 10.0 ** float(rng.integers(-3, 4))
        lo = np.float32(rng.uniform(-1000.0, 1000.0) * cw)
        x = (lo + rng.uniform(0.0, 2000.0 * cw, 20000)).astype(np.float32)
        x = np.maximum(x, lo)
        assert _check(x, lo, cw) < 0.01


def test_points_on_and_next_to_cell_edges():
    for cw in (1.0, 0.5, 0.49, 0.1, 1.0 / 3.0, 0.49 * (100 / 49), 1000.0 / 1024.0):
        edge = (np.arange(0, 4096, dtype=np.float64) * cw).astype(np.float32)
        x = np.concatenate([edge, np.nextafter(edge, np.float32(-np.inf)),
                            np.nextafter(edge, np.float32(np.inf))])
        _check(x[x >= 0.0], np.float32(0.0), cw)


def test_integer_lattice_with_unit_width_uses_the_division():
    x = np.arange(0, 1000, dtype=np.float32)
    got, exact, near = _rule(x, np.float32(0.0), 1.0)
    np.testing.assert_array_equal(got, exact)
    np.testing.assert_array_equal(got, np.arange(1000))
    assert near.all()              # exact integers always take the division


def test_uniform_data_rarely_falls_back():
    rng = np.random.default_rng(2)
    x = rng.uniform(0.0, 1000.0, 1 << 20).astype(np.float32)
    lo = x.min()
    cw = 2.0 * 1000.0 / (2.0 * np.sqrt(1 << 20))   # a typical cell width, 2 r_exp
    assert _check(x, lo, cw) < 2e-3



def test_fma_pipe_polynomials_are_the_generators_fits():
    """The exp2 / log2 polynomial coefficients in the kernel source are the
    float32-rounded minimax fits that fit_poly.py computes, and meet their
    stated error bounds (the generator, not the kernel, is under test: its
    output is what the kernel must carry)."""
    import os
    import re

    from paper_1601_05904_gb300 import fit_poly
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_1601_05904_gb300", "csrc", "aidw_device.cuh")).read()

    def consts(fn):
        body = src[src.index(f"__device__ __forceinline__ F2 {fn}("):]
        body = body[: body.index("\n}\n")]
        # coefficients are the scientific-notation literals packed into both lanes
        return [float(np.float32(v)) for v in re.findall(r"f2_pack\(([-+0-9.]+e[-+0-9]+)f, \1f\)", body)]
    e = consts("f2_exp2_poly")
    lg = consts("f2_log2_poly")
    assert len(e) == 6 and len(lg) == 8
    assert e == [float(v) for v in fit_poly.exp2_coefficients().astype(np.float32)]
    assert lg == [float(v) for v in fit_poly.log2_coefficients().astype(np.float32)]
    assert fit_poly.exp2_error(np.array(e)) < 2e-7
    assert fit_poly.log2_error(np.array(lg)) < 6e-8
