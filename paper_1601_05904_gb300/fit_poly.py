"""Generator of the coefficients of the FMA-pipe exp2 and log2 polynomials
used by the float32 weighting kernel (``f2_exp2_poly`` and ``f2_log2_poly``
in ``csrc/aidw_device.cuh``).

Both are best approximations in the maximum norm, found with Lawson's
algorithm: iteratively reweighted least squares on a dense grid, where each
iteration multiplies every point's weight by its current error, which
converges to the minimax (equioscillating) solution.

  exp2:  2^f ~ P5(f) on [-1/2, 1/2], minimising the relative error
  log2:  log2(1 + s) ~ s * P7(s) on [sqrt(1/2) - 1, sqrt(2) - 1],
         minimising the absolute error

The coefficients are rounded to float32, the precision the kernel
evaluates them in.  ``python -m paper_1601_05904_gb300.fit_poly`` prints
them (highest degree first) with their errors in float64 and after the
rounding.
"""
from __future__ import annotations

import numpy as np

GRID = 40001
ITERS = 200


def lawson(x, target, basis, scale, iters: int = ITERS):
    """Coefficients c minimising max |basis @ c - target| * scale."""
    a = basis * scale[:, None]
    b = target * scale
    w = np.full(x.size, 1.0 / x.size)
    c = None
    for _ in range(iters):
        r = np.sqrt(w)
        c, *_ = np.linalg.lstsq(a * r[:, None], b * r, rcond=None)
        e = np.abs(a @ c - b)
        w = w * e
        w /= w.sum()
    return c


def exp2_coefficients():
    f = np.linspace(-0.5, 0.5, GRID)
    y = np.exp2(f)
    return lawson(f, y, np.vander(f, 6), 1.0 / y)


def log2_coefficients():
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    s = np.linspace(lo, hi, GRID)
    return lawson(s, np.log2(1.0 + s), np.vander(s, 8) * s[:, None], np.ones_like(s))


def exp2_error(c) -> float:
    f = np.linspace(-0.5, 0.5, GRID)
    return float(np.abs(np.polyval(c, f) / np.exp2(f) - 1.0).max())


def log2_error(c) -> float:
    s = np.linspace(np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0, GRID)
    return float(np.abs(s * np.polyval(c, s) - np.log2(1.0 + s)).max())


def main():
    for name, fit, err in (("exp2", exp2_coefficients, exp2_error),
                           ("log2", log2_coefficients, log2_error)):
        c = fit()
        c32 = c.astype(np.float32)
        print(f"{name}: max error {err(c):.3e} (float64), {err(c32.astype(np.float64)):.3e} "
              "(coefficients rounded to float32)")
        for v in c32:
            print(f"    {float(v):.16e}f")


if __name__ == "__main__":
    main()
