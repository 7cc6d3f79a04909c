"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the CUDA path's callers (tests,
bench) and by the oracle's callers: it only draws random numbers and holds
none of the interpolation method's arithmetic.

The paper's test data are random points in a square with as many data
points as interpolated points (Sec. 5.1); its files are not available, so
these generators stand in for them.  Every array is drawn in float64 with
``numpy.random.default_rng(seed)`` and cast to float32.

Workloads (sizes n = data points, m = query points):
  unit      n = m = 4096 in [0,1]^2, z = sin(6x)cos(6y) + N(0, 0.01^2)
  uniform   n = m (default 1,048,576) in [0,1000]^2,
            z = 100 sin(x/50) cos(y/70) + N(0, 1)
  clustered data: 90 % from 32 isotropic Gaussians (sigma in U[5, 40],
            centres in U[0,1000]^2, samples outside the square redrawn) and
            10 % uniform; queries uniform; same z field as ``uniform``
  batch     512 jobs, n_j log-uniform in [1e3, 2e5], m_j = n_j,
            k_j in {8, 10, 16, 24, 32}, per-job mix of uniform and
            clustered points with a random clustered fraction and count
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SIDE_KILO = 1000.0
BATCH_K_CHOICES = (8, 10, 16, 24, 32)


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    qx: np.ndarray
    qy: np.ndarray
    k: int
    seed: int
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.size)

    @property
    def m(self) -> int:
        return int(self.qx.size)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def uniform_points(rng: np.random.Generator, n: int, lo: float, hi: float):
    x = rng.uniform(lo, hi, n)
    y = rng.uniform(lo, hi, n)
    return _f32(x), _f32(y)


def gaussian_mixture_points(rng: np.random.Generator, n: int, n_clusters: int,
                            lo: float = 0.0, hi: float = SIDE_KILO,
                            sigma_lo: float = 5.0, sigma_hi: float = 40.0):
    """n points from n_clusters equally weighted isotropic Gaussians with
    centres uniform in the square; points falling outside are redrawn."""
    cx = rng.uniform(lo, hi, n_clusters)
    cy = rng.uniform(lo, hi, n_clusters)
    sig = rng.uniform(sigma_lo, sigma_hi, n_clusters)
    lab = rng.integers(0, n_clusters, n)
    x = cx[lab] + sig[lab] * rng.standard_normal(n)
    y = cy[lab] + sig[lab] * rng.standard_normal(n)
    bad = (x < lo) | (x > hi) | (y < lo) | (y > hi)
    while bad.any():
        nb = int(bad.sum())
        lb = lab[bad]
        x[bad] = cx[lb] + sig[lb] * rng.standard_normal(nb)
        y[bad] = cy[lb] + sig[lb] * rng.standard_normal(nb)
        bad = (x < lo) | (x > hi) | (y < lo) | (y > hi)
    return _f32(x), _f32(y)


def mixed_points(rng: np.random.Generator, n: int, clustered_fraction: float,
                 n_clusters: int, lo: float = 0.0, hi: float = SIDE_KILO):
    """A clustered part from a Gaussian mixture plus a uniform background,
    shuffled together."""
    nc = int(round(clustered_fraction * n))
    xc, yc = gaussian_mixture_points(rng, nc, n_clusters, lo, hi) if nc else (
        np.empty(0, np.float32), np.empty(0, np.float32))
    xu, yu = uniform_points(rng, n - nc, lo, hi)
    x = np.concatenate([xc, xu])
    y = np.concatenate([yc, yu])
    order = rng.permutation(n)
    return _f32(x[order]), _f32(y[order])


def field_unit(rng: np.random.Generator, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    return _f32(np.sin(6.0 * xd) * np.cos(6.0 * yd) + 0.01 * rng.standard_normal(x.size))


def field_kilo(rng: np.random.Generator, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    return _f32(100.0 * np.sin(xd / 50.0) * np.cos(yd / 70.0) + rng.standard_normal(x.size))


def unit_square(n: int = 4096, m: int | None = None, k: int = 10, seed: int = 0) -> Workload:
    """Small unit-square workload the oracle finishes in seconds."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    x, y = uniform_points(rng, n, 0.0, 1.0)
    z = field_unit(rng, x, y)
    qx, qy = uniform_points(rng, m, 0.0, 1.0)
    return Workload(f"unit n={n} m={m} in [0,1]^2", x, y, z, qx, qy, k, seed)


def uniform_kilo(n: int = 1 << 20, m: int | None = None, k: int = 10, seed: int = 1) -> Workload:
    """n data and m query points uniform in [0,1000]^2."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    x, y = uniform_points(rng, n, 0.0, SIDE_KILO)
    z = field_kilo(rng, x, y)
    qx, qy = uniform_points(rng, m, 0.0, SIDE_KILO)
    return Workload(f"uniform n={n} m={m} in [0,1000]^2", x, y, z, qx, qy, k, seed)


def clustered_kilo(n: int = 1 << 20, m: int | None = None, k: int = 10, seed: int = 2,
                   n_clusters: int = 32, clustered_fraction: float = 0.9) -> Workload:
    """Data from a Gaussian mixture plus uniform background; queries uniform."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    x, y = mixed_points(rng, n, clustered_fraction, n_clusters)
    z = field_kilo(rng, x, y)
    qx, qy = uniform_points(rng, m, 0.0, SIDE_KILO)
    return Workload(f"clustered n={n} m={m} ({n_clusters} gaussians, "
                    f"{clustered_fraction:.0%} clustered)", x, y, z, qx, qy, k, seed)


def batch_jobs(n_jobs: int = 512, seed_base: int = 1000, n_lo: float = 1e3, n_hi: float = 2e5,
               k_choices=BATCH_K_CHOICES) -> list[Workload]:
    """Independent jobs of uneven size: n_j log-uniform in [n_lo, n_hi],
    m_j = n_j, k_j uniform over k_choices, each its own random mix of
    uniform and clustered points in [0,1000]^2 (seed seed_base + j)."""
    jobs = []
    for j in range(n_jobs):
        rng = np.random.default_rng(seed_base + j)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = int(k_choices[int(rng.integers(0, len(k_choices)))])
        frac = float(rng.uniform(0.0, 0.9))
        g = int(rng.integers(1, 33))
        x, y = mixed_points(rng, n, frac, g)
        z = field_kilo(rng, x, y)
        qx, qy = uniform_points(rng, n, 0.0, SIDE_KILO)
        jobs.append(Workload(f"job {j}", x, y, z, qx, qy, k, seed_base + j,
                             {"clustered_fraction": frac, "n_clusters": g}))
    return jobs


def query_subsample(m: int, count: int, seed: int = 12345) -> np.ndarray:
    """Sorted, distinct query indices for sampled checks at full size."""
    rng = np.random.default_rng(seed)
    count = min(count, m)
    return np.sort(rng.choice(m, size=count, replace=False)).astype(np.int64)
