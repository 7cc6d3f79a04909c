"""Plain FP64 CPU oracle for AIDW interpolation with kNN (arXiv 1601.05904).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import this
package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``aidw_oracle.c`` (plain C, double precision, one
query at a time).  This module compiles it with gcc into ``oracle/_build``
and wraps its functions with numpy marshalling only:

  r_exp / r_obs / R / mu / alpha   Eq. 2, 3, 4, 5, 6
  knn                              Sec. 2.3 brute force (full sort, first k)
  aidw                             Sec. 2.2 steps 1-3 and Eq. 1 (all points)
  aidw_local                       the same with Eq. 1 over the k nearest points
  grid                             Sec. 3.2.1-3.2.3 even grid, cell order
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aidw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None
_openmp = False

DEFAULT_ALPHA = (1.0, 2.0, 3.0, 4.0, 5.0)
DEFAULT_R_MIN = 0.0
DEFAULT_R_MAX = 2.0


def _src_tag() -> str:
    with open(_SRC, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def build(verbose: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path.

    Tries OpenMP first (the loop over queries is the only parallel part and
    does not change any result) and falls back to a serial build.
    """
    global _openmp
    os.makedirs(_BUILD, exist_ok=True)
    tag = _src_tag()
    for omp in (True, False):
        out = os.path.join(_BUILD, f"liboracle_{tag}{'_omp' if omp else ''}.so")
        if os.path.exists(out):
            _openmp = omp
            return out
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", out + ".tmp", "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose and r.returncode != 0:
            print(r.stderr)
        if r.returncode == 0:
            os.replace(out + ".tmp", out)
            _openmp = omp
            return out
    raise RuntimeError("could not compile the oracle with gcc")


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_f = ctypes.POINTER(ctypes.c_float)
        c_d = ctypes.POINTER(ctypes.c_double)
        c_i32 = ctypes.POINTER(ctypes.c_int32)
        c_i64 = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        lib.oracle_r_exp.restype = ctypes.c_double
        lib.oracle_r_exp.argtypes = [i64, ctypes.c_double]
        lib.oracle_r_obs.restype = ctypes.c_double
        lib.oracle_r_obs.argtypes = [c_d, ctypes.c_int]
        lib.oracle_R.restype = ctypes.c_double
        lib.oracle_R.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.oracle_mu.restype = ctypes.c_double
        lib.oracle_mu.argtypes = [ctypes.c_double] * 3
        lib.oracle_alpha.restype = ctypes.c_double
        lib.oracle_alpha.argtypes = [ctypes.c_double, c_d]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_has_openmp.restype = ctypes.c_int
        lib.oracle_has_openmp.argtypes = []
        lib.oracle_knn.restype = None
        lib.oracle_knn.argtypes = [c_f, c_f, i64, c_f, c_f, i64, ctypes.c_int,
                                   c_i32, c_d, ctypes.c_int]
        lib.oracle_knn_paper_rule.restype = None
        lib.oracle_knn_paper_rule.argtypes = [c_f, c_f, i64, c_d, c_i64, c_i64, c_f, c_f, i64,
                                              ctypes.c_int, ctypes.c_int, c_i32, c_d,
                                              ctypes.c_int]
        lib.oracle_aidw.restype = None
        lib.oracle_aidw.argtypes = [c_f, c_f, c_f, i64, c_f, c_f, i64, ctypes.c_int,
                                    c_d, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, c_d, c_d, c_d, c_d, ctypes.c_int]
        lib.oracle_aidw_local.restype = None
        lib.oracle_aidw_local.argtypes = [c_f, c_f, c_f, i64, c_f, c_f, i64, ctypes.c_int,
                                          c_d, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, c_d, c_d, c_d, ctypes.c_int]
        lib.oracle_grid_dims.restype = None
        lib.oracle_grid_dims.argtypes = [c_f, c_f, i64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, c_d]
        lib.oracle_grid_fill.restype = None
        lib.oracle_grid_fill.argtypes = [c_f, c_f, i64, c_d, c_i64, c_i64, c_i64]
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    """Threads the oracle's query loop uses by default (1 without OpenMP)."""
    return int(_load().oracle_num_threads())


def has_openmp() -> bool:
    """Whether the query loops can run on several threads (``nthreads``)."""
    return bool(_load().oracle_has_openmp())


def r_exp(n: int, area: float) -> float:
    """Eq. 2."""
    return float(_load().oracle_r_exp(int(n), float(area)))


def r_obs(d) -> float:
    """Eq. 3 over the given k distances."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    return float(_load().oracle_r_obs(_ptr(d, ctypes.c_double), int(d.size)))


def R(r_obs_: float, r_exp_: float) -> float:
    """Eq. 4."""
    return float(_load().oracle_R(float(r_obs_), float(r_exp_)))


def mu(R_: float, r_min: float = DEFAULT_R_MIN, r_max: float = DEFAULT_R_MAX) -> float:
    """Eq. 5."""
    return float(_load().oracle_mu(float(R_), float(r_min), float(r_max)))


def alpha(mu_: float, levels=DEFAULT_ALPHA) -> float:
    """Eq. 6."""
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    assert lv.size == 5
    return float(_load().oracle_alpha(float(mu_), _ptr(lv, ctypes.c_double)))


def knn(x, y, qx, qy, k: int, nthreads: int = 0):
    """Brute-force kNN (Sec. 2.3).  Returns (idx int32 [m,k], dist f64 [m,k])
    in increasing (distance, index) order."""
    x, y, qx, qy = _f32(x), _f32(y), _f32(qx), _f32(qy)
    n, m = x.size, qx.size
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= n")
    idx = np.empty((m, k), dtype=np.int32)
    dist = np.empty((m, k), dtype=np.float64)
    if m:
        _load().oracle_knn(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                           _ptr(qx, ctypes.c_float), _ptr(qy, ctypes.c_float), m, int(k),
                           _ptr(idx, ctypes.c_int32), _ptr(dist, ctypes.c_double),
                           int(nthreads))
    return idx, dist


def knn_paper_rule(x, y, qx, qy, k: int, cell_scale: float = 1.0, area: float = 0.0,
                   cw_override: float = 0.0, n_out: int | None = None, nthreads: int = 0):
    """Grid kNN with the paper's level rule (Sec. 3.2.4: the first level of
    cell expanding whose block holds k points, plus one level), on the grid
    of ``grid`` with the same arguments.  Returns (idx int32 [m,n_out], dist
    f64 [m,n_out]), the block's points in increasing (distance, index)
    order; k fixes the level, n_out >= k (default k) columns are returned
    (-1 / inf past the block's count).  Not always the exact kNN."""
    x, y, qx, qy = _f32(x), _f32(y), _f32(qx), _f32(qy)
    n, m = x.size, qx.size
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= n")
    lib = _load()
    info = np.zeros(9, dtype=np.float64)
    lib.oracle_grid_dims(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                         float(cell_scale), float(area), float(cw_override),
                         _ptr(info, ctypes.c_double))
    ncol, nrow = int(info[7]), int(info[8])
    key = np.empty(n, dtype=np.int64)
    start = np.empty(ncol * nrow + 1, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    lib.oracle_grid_fill(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                         _ptr(info, ctypes.c_double), _ptr(key, ctypes.c_int64),
                         _ptr(start, ctypes.c_int64), _ptr(perm, ctypes.c_int64))
    n_out = k if n_out is None else int(n_out)
    if n_out < k:
        raise ValueError("need n_out >= k")
    idx = np.empty((m, n_out), dtype=np.int32)
    dist = np.empty((m, n_out), dtype=np.float64)
    if m:
        lib.oracle_knn_paper_rule(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                                  _ptr(info, ctypes.c_double), _ptr(start, ctypes.c_int64),
                                  _ptr(perm, ctypes.c_int64), _ptr(qx, ctypes.c_float),
                                  _ptr(qy, ctypes.c_float), m, int(k), n_out,
                                  _ptr(idx, ctypes.c_int32), _ptr(dist, ctypes.c_double),
                                  int(nthreads))
    return idx, dist


def aidw(x, y, z, qx, qy, k: int, levels=DEFAULT_ALPHA, r_min: float = DEFAULT_R_MIN,
         r_max: float = DEFAULT_R_MAX, area: float = 0.0, nthreads: int = 0):
    """AIDW prediction (Sec. 2.2 and Eq. 1 over all data points).

    Returns a dict of float64 arrays [m]: ``z`` prediction, ``alpha`` (Eq. 6),
    ``r_obs`` (Eq. 3) and ``scale`` = sum w|z| / sum w, the magnitude against
    which an error in ``z`` is measured."""
    x, y, z, qx, qy = _f32(x), _f32(y), _f32(z), _f32(qx), _f32(qy)
    n, m = x.size, qx.size
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= n")
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    out = {key: np.empty(m, dtype=np.float64) for key in ("z", "alpha", "r_obs", "scale")}
    if m:
        _load().oracle_aidw(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float),
                            _ptr(z, ctypes.c_float), n,
                            _ptr(qx, ctypes.c_float), _ptr(qy, ctypes.c_float), m, int(k),
                            _ptr(lv, ctypes.c_double), float(r_min), float(r_max),
                            float(area), _ptr(out["z"], ctypes.c_double),
                            _ptr(out["alpha"], ctypes.c_double),
                            _ptr(out["r_obs"], ctypes.c_double),
                            _ptr(out["scale"], ctypes.c_double), int(nthreads))
    return out


def aidw_local(x, y, z, qx, qy, k: int, levels=DEFAULT_ALPHA, r_min: float = DEFAULT_R_MIN,
               r_max: float = DEFAULT_R_MAX, area: float = 0.0, nthreads: int = 0):
    """Local AIDW: alpha as in ``aidw``, Eq. 1 over the k nearest points.
    Returns a dict of float64 arrays [m]: ``z``, ``alpha``, ``scale``."""
    x, y, z, qx, qy = _f32(x), _f32(y), _f32(z), _f32(qx), _f32(qy)
    n, m = x.size, qx.size
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= n")
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    out = {key: np.empty(m, dtype=np.float64) for key in ("z", "alpha", "scale")}
    if m:
        _load().oracle_aidw_local(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float),
                                  _ptr(z, ctypes.c_float), n,
                                  _ptr(qx, ctypes.c_float), _ptr(qy, ctypes.c_float), m, int(k),
                                  _ptr(lv, ctypes.c_double), float(r_min), float(r_max),
                                  float(area), _ptr(out["z"], ctypes.c_double),
                                  _ptr(out["alpha"], ctypes.c_double),
                                  _ptr(out["scale"], ctypes.c_double), int(nthreads))
    return out


def grid(x, y, cell_scale: float = 1.0, area: float = 0.0, cw_override: float = 0.0):
    """Even grid of the data points (Sec. 3.2.1-3.2.3).

    Returns a dict: bbox/area/r_exp/cw/ncol/nrow scalars, ``key`` [n] int64,
    ``cell_start`` [ncol*nrow+1] int64 and ``perm`` [n] int64 (original
    indices in cell order, stable)."""
    x, y = _f32(x), _f32(y)
    n = x.size
    if n < 1:
        raise ValueError("need n >= 1")
    lib = _load()
    info = np.zeros(9, dtype=np.float64)
    lib.oracle_grid_dims(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                         float(cell_scale), float(area), float(cw_override),
                         _ptr(info, ctypes.c_double))
    ncol, nrow = int(info[7]), int(info[8])
    key = np.empty(n, dtype=np.int64)
    start = np.empty(ncol * nrow + 1, dtype=np.int64)
    perm = np.empty(n, dtype=np.int64)
    lib.oracle_grid_fill(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), n,
                         _ptr(info, ctypes.c_double), _ptr(key, ctypes.c_int64),
                         _ptr(start, ctypes.c_int64), _ptr(perm, ctypes.c_int64))
    return {"min_x": info[0], "min_y": info[1], "max_x": info[2], "max_y": info[3],
            "area": info[4], "r_exp": info[5], "cw": info[6], "ncol": ncol, "nrow": nrow,
            "key": key, "cell_start": start, "perm": perm}


def normalized_error(z_test, z_ref, scale):
    """err_q = |z_test - z_ref| / S_q (the error measure for Eq. 1, whose
    numerator cancels when z changes sign)."""
    z_test = np.asarray(z_test, dtype=np.float64)
    z_ref = np.asarray(z_ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    return np.abs(z_test - z_ref) / np.maximum(scale, np.finfo(np.float64).tiny)
