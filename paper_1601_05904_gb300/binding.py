"""Python binding of the C ABI in ``include/aidw.h`` (ctypes, marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but check tensor arguments, pass device pointers and the current
CUDA stream, and turn status codes into exceptions.  All computation runs in
``libaidw.so``; if the library is missing this module raises instead of
falling back to anything else.

Tensors are torch CUDA tensors (torch is used for device memory and streams
only): float32, contiguous, on the current device.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libaidw.so")
# the bounds-checked build of the same sources (build(checked=True))
LIB_CHECKED_PATH = os.path.join(PKG, "libaidw_checked.so")

AIDW_OK = 0
AIDW_FP32_COMP = 0
AIDW_FP64_PLAIN = 1
AIDW_MAX_K = 32
STAGES = ("grid_build", "knn", "weight", "finalize", "batch")

_STATUS_NAMES = {0: "AIDW_OK", 1: "AIDW_ERR_INVALID_ARG", 2: "AIDW_ERR_K_RANGE",
                 3: "AIDW_ERR_NONFINITE", 4: "AIDW_ERR_OOM", 5: "AIDW_ERR_CUDA",
                 6: "AIDW_ERR_TIMEOUT"}


class AidwError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)} "
                         f"({aidw_status_string(status)})")


class CParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("alpha", ctypes.c_double * 5),
                ("r_min", ctypes.c_double), ("r_max", ctypes.c_double),
                ("area", ctypes.c_double), ("cell_scale", ctypes.c_double),
                ("precision", ctypes.c_int)]


class CGridInfo(ctypes.Structure):
    _fields_ = [("n_data", ctypes.c_int64), ("n_col", ctypes.c_int64),
                ("n_row", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("min_x", ctypes.c_double), ("min_y", ctypes.c_double),
                ("max_x", ctypes.c_double), ("max_y", ctypes.c_double),
                ("area", ctypes.c_double), ("r_exp", ctypes.c_double),
                ("cell_width", ctypes.c_double), ("cell_scale", ctypes.c_double)]


@dataclass
class Params:
    """Mirror of aidw_params (defaults as aidw_params_default)."""
    k: int = 10
    alpha: tuple = (1.0, 2.0, 3.0, 4.0, 5.0)
    r_min: float = 0.0
    r_max: float = 2.0
    area: float = 0.0
    cell_scale: float = 0.0
    precision: int = AIDW_FP32_COMP

    def to_c(self) -> CParams:
        c = CParams()
        c.k = int(self.k)
        for i, a in enumerate(self.alpha):
            c.alpha[i] = float(a)
        c.r_min = float(self.r_min)
        c.r_max = float(self.r_max)
        c.area = float(self.area)
        c.cell_scale = float(self.cell_scale)
        c.precision = int(self.precision)
        return c


class CJob(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("n_data", ctypes.c_int64), ("qx", ctypes.c_void_p), ("qy", ctypes.c_void_p),
                ("n_query", ctypes.c_int64), ("k", ctypes.c_int), ("out_z", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libaidw.so (built in-tree by ``paper_1601_05904_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        P = ctypes.POINTER
        lib.aidw_params_default.restype = None
        lib.aidw_params_default.argtypes = [P(CParams)]
        lib.aidw_status_string.restype = ctypes.c_char_p
        lib.aidw_status_string.argtypes = [c_int]
        lib.aidw_grid_build.restype = c_int
        lib.aidw_grid_build.argtypes = [vp, vp, vp, i64, P(CParams), vp, P(vp)]
        lib.aidw_grid_destroy.restype = c_int
        lib.aidw_grid_destroy.argtypes = [vp]
        lib.aidw_grid_get_info.restype = c_int
        lib.aidw_grid_get_info.argtypes = [vp, P(CGridInfo)]
        lib.aidw_grid_export.restype = c_int
        lib.aidw_grid_export.argtypes = [vp, vp, vp, vp]
        lib.aidw_grid_status.restype = c_int
        lib.aidw_grid_status.argtypes = [vp]
        lib.aidw_knn.restype = c_int
        lib.aidw_knn.argtypes = [vp, vp, vp, i64, c_int, vp, vp, vp, vp]
        lib.aidw_interpolate.restype = c_int
        lib.aidw_interpolate.argtypes = [vp, vp, vp, i64, P(CParams), vp, vp, vp]
        lib.aidw_knn_bruteforce.restype = c_int
        lib.aidw_knn_bruteforce.argtypes = [vp, vp, vp, i64, c_int, vp, vp, vp, vp]
        lib.aidw_knn_paper_rule.restype = c_int
        lib.aidw_knn_paper_rule.argtypes = [vp, vp, vp, i64, c_int, vp, vp, vp, vp]
        lib.aidw_interpolate_local.restype = c_int
        lib.aidw_interpolate_local.argtypes = [vp, vp, vp, i64, P(CParams), vp, vp, vp]
        lib.aidw_test_expire_next_wait.restype = c_int
        lib.aidw_test_expire_next_wait.argtypes = [c_int]
        lib.aidw_set_memory_limit.restype = c_int
        lib.aidw_set_memory_limit.argtypes = [i64, P(i64)]
        lib.aidw_profile_enable.restype = c_int
        lib.aidw_profile_enable.argtypes = [c_int]
        lib.aidw_profile_read.restype = c_int
        lib.aidw_profile_read.argtypes = [P(ctypes.c_double), P(ctypes.c_int64)]
        lib.aidw_probe_pipe_rates.restype = c_int
        lib.aidw_probe_pipe_rates.argtypes = [P(ctypes.c_double)] * 3
        lib.aidw_probe_weight_loop.restype = c_int
        lib.aidw_probe_weight_loop.argtypes = [c_int, P(ctypes.c_double)]
        lib.aidw_interpolate_host.restype = c_int
        lib.aidw_interpolate_host.argtypes = [vp, vp, vp, i64, vp, vp, i64, P(CParams), vp, vp, vp]
        lib.aidw_shard_range.restype = c_int
        lib.aidw_shard_range.argtypes = [i64, c_int, c_int, P(i64), P(i64)]
        lib.aidw_interpolate_shard.restype = c_int
        lib.aidw_interpolate_shard.argtypes = [vp, vp, vp, i64, c_int, c_int, P(CParams), vp,
                                               vp, vp]
        lib.aidw_bounds_report.restype = c_int
        lib.aidw_bounds_report.argtypes = [P(c_int), P(ctypes.c_uint64), P(ctypes.c_uint64)]
        lib.aidw_test_bounds_check.restype = c_int
        lib.aidw_test_bounds_check.argtypes = [i64, i64, P(c_int)]
        lib.aidw_weight_mix.restype = c_int
        lib.aidw_weight_mix.argtypes = [P(c_int), P(c_int), P(c_int), P(ctypes.c_double),
                                        P(ctypes.c_double)]
        lib.aidw_batch_plan_create.restype = c_int
        lib.aidw_batch_plan_create.argtypes = [P(CJob), c_int, P(CParams), P(vp)]
        lib.aidw_batch_run.restype = c_int
        lib.aidw_batch_run.argtypes = [vp, P(CJob), vp]
        lib.aidw_batch_plan_tune.restype = c_int
        lib.aidw_batch_plan_tune.argtypes = [vp, P(CJob), vp, P(ctypes.c_double)]
        lib.aidw_batch_plan_get.restype = c_int
        lib.aidw_batch_plan_get.argtypes = [vp, P(ctypes.c_double), P(c_int), P(i64), P(i64)]
        lib.aidw_batch_plan_get_classes.restype = c_int
        lib.aidw_batch_plan_get_classes.argtypes = [vp, P(c_int), P(ctypes.c_double), P(c_int),
                                                    P(i64), P(c_int)]
        lib.aidw_batch_plan_status.restype = c_int
        lib.aidw_batch_plan_status.argtypes = [vp]
        lib.aidw_batch_plan_destroy.restype = c_int
        lib.aidw_batch_plan_destroy.argtypes = [vp]
        lib.aidw_batch.restype = c_int
        lib.aidw_batch.argtypes = [P(CJob), c_int, P(CParams), vp]
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != AIDW_OK:
        raise AidwError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32_dev(t, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 1:
        raise TypeError(f"{name} must be a contiguous 1-D float32 tensor")
    return t


def aidw_status_string(status: int) -> str:
    if _lib is None:
        return _STATUS_NAMES.get(status, str(status))
    return _lib.aidw_status_string(int(status)).decode()


def aidw_params_default() -> Params:
    c = CParams()
    load().aidw_params_default(ctypes.byref(c))
    return Params(k=c.k, alpha=tuple(c.alpha), r_min=c.r_min, r_max=c.r_max, area=c.area,
                  cell_scale=c.cell_scale, precision=c.precision)


@dataclass
class Grid:
    """Owner of an aidw_grid handle; destroy() (or garbage collection) frees it."""
    handle: ctypes.c_void_p
    n_data: int
    _alive: bool = field(default=True, repr=False)

    def destroy(self) -> None:
        if self._alive:
            self._alive = False
            _check(load().aidw_grid_destroy(self.handle), "aidw_grid_destroy")

    def __del__(self):
        if getattr(self, "_alive", False):
            try:
                self._alive = False
                load().aidw_grid_destroy(self.handle)
            except Exception:
                pass


def aidw_grid_build(x, y, z, params: Params | None = None, stream=None) -> Grid:
    x, y, z = _f32_dev(x, "x"), _f32_dev(y, "y"), _f32_dev(z, "z")
    if not (x.numel() == y.numel() == z.numel()):
        raise ValueError("x, y, z must have the same length")
    p = (params or Params()).to_c()
    h = ctypes.c_void_p()
    _check(load().aidw_grid_build(_ptr(x), _ptr(y), _ptr(z), x.numel(), ctypes.byref(p),
                                  _stream(stream), ctypes.byref(h)), "aidw_grid_build")
    return Grid(h, x.numel())


def aidw_grid_destroy(grid: Grid) -> None:
    grid.destroy()


def aidw_grid_get_info(grid: Grid) -> dict:
    info = CGridInfo()
    _check(load().aidw_grid_get_info(grid.handle, ctypes.byref(info)), "aidw_grid_get_info")
    return {name: getattr(info, name) for name, _ in CGridInfo._fields_}


def aidw_grid_export(grid: Grid, stream=None):
    """Returns (cell_start int64 [n_cells+1], perm int32 [n_data]) device tensors."""
    import torch
    info = aidw_grid_get_info(grid)
    cs = torch.empty(info["n_cells"] + 1, dtype=torch.int64, device="cuda")
    perm = torch.empty(grid.n_data, dtype=torch.int32, device="cuda")
    _check(load().aidw_grid_export(grid.handle, _ptr(cs), _ptr(perm), _stream(stream)),
           "aidw_grid_export")
    return cs, perm


def aidw_grid_status(grid: Grid) -> int:
    """Synchronises and returns the latched device status code (0 = ok)."""
    return int(load().aidw_grid_status(grid.handle))


def _knn_call(name: str, grid: Grid, qx, qy, k: int, out_idx, out_dist, out_robs, want, stream):
    import torch
    qx, qy = _f32_dev(qx, "qx"), _f32_dev(qy, "qy")
    m = qx.numel()
    if qy.numel() != m:
        raise ValueError("qx and qy must have the same length")
    if out_idx is None and "idx" in want:
        out_idx = torch.empty((m, k), dtype=torch.int32, device=qx.device)
    if out_dist is None and "dist" in want:
        out_dist = torch.empty((m, k), dtype=torch.float32, device=qx.device)
    if out_robs is None and "robs" in want:
        out_robs = torch.empty(m, dtype=torch.float32, device=qx.device)
    _check(getattr(load(), name)(grid.handle, _ptr(qx), _ptr(qy), m, int(k), _ptr(out_idx),
                                 _ptr(out_dist), _ptr(out_robs), _stream(stream)), name)
    return out_idx, out_dist, out_robs


def aidw_knn(grid: Grid, qx, qy, k: int, out_idx=None, out_dist=None, out_robs=None,
             want=("idx", "dist", "robs"), stream=None):
    """Grid kNN.  Allocates the outputs named in ``want`` that are not given.
    Returns (idx int32 [m,k] | None, dist float32 [m,k] | None, robs float32 [m] | None)."""
    return _knn_call("aidw_knn", grid, qx, qy, k, out_idx, out_dist, out_robs, want, stream)


def aidw_knn_bruteforce(grid: Grid, qx, qy, k: int, out_idx=None, out_dist=None, out_robs=None,
                        want=("idx", "dist", "robs"), stream=None):
    """All-points per-thread kNN (the paper's original algorithm); same
    outputs as aidw_knn."""
    return _knn_call("aidw_knn_bruteforce", grid, qx, qy, k, out_idx, out_dist, out_robs, want,
                     stream)


def aidw_knn_paper_rule(grid: Grid, qx, qy, k: int, out_idx=None, out_dist=None, out_robs=None,
                        want=("idx", "dist", "robs"), stream=None):
    """Grid kNN with the paper's level rule (not always exact); same outputs
    as aidw_knn."""
    return _knn_call("aidw_knn_paper_rule", grid, qx, qy, k, out_idx, out_dist, out_robs, want,
                     stream)


def aidw_interpolate(grid: Grid, qx, qy, params: Params | None = None, out_z=None,
                     out_alpha=None, want_alpha: bool = False, stream=None):
    """AIDW predictions.  Output dtype is float32 (FP32_COMP) or float64
    (FP64_PLAIN).  Returns (z, alpha | None)."""
    import torch
    p = params or Params()
    qx, qy = _f32_dev(qx, "qx"), _f32_dev(qy, "qy")
    m = qx.numel()
    if qy.numel() != m:
        raise ValueError("qx and qy must have the same length")
    dt = torch.float64 if p.precision == AIDW_FP64_PLAIN else torch.float32
    if out_z is None:
        out_z = torch.empty(m, dtype=dt, device=qx.device)
    if out_alpha is None and want_alpha:
        out_alpha = torch.empty(m, dtype=dt, device=qx.device)
    for t, name in ((out_z, "out_z"), (out_alpha, "out_alpha")):
        if t is not None and (t.dtype != dt or t.numel() != m or not t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous {dt} tensor of length {m}")
    pc = p.to_c()
    _check(load().aidw_interpolate(grid.handle, _ptr(qx), _ptr(qy), m, ctypes.byref(pc),
                                   _ptr(out_z), _ptr(out_alpha), _stream(stream)),
           "aidw_interpolate")
    return out_z, out_alpha


def aidw_interpolate_local(grid: Grid, qx, qy, params: Params | None = None, out_z=None,
                           out_alpha=None, want_alpha: bool = False, stream=None):
    """Local AIDW (Eq. 1 over the k nearest points).  Returns (z, alpha | None)."""
    import torch
    p = params or Params()
    qx, qy = _f32_dev(qx, "qx"), _f32_dev(qy, "qy")
    m = qx.numel()
    dt = torch.float64 if p.precision == AIDW_FP64_PLAIN else torch.float32
    if out_z is None:
        out_z = torch.empty(m, dtype=dt, device=qx.device)
    if out_alpha is None and want_alpha:
        out_alpha = torch.empty(m, dtype=dt, device=qx.device)
    pc = p.to_c()
    _check(load().aidw_interpolate_local(grid.handle, _ptr(qx), _ptr(qy), m, ctypes.byref(pc),
                                         _ptr(out_z), _ptr(out_alpha), _stream(stream)),
           "aidw_interpolate_local")
    return out_z, out_alpha


def aidw_shard_range(n_query: int, shard: int, n_shards: int) -> tuple[int, int]:
    """Query slice [begin, end) of shard ``shard`` of ``n_shards`` (host only)."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    _check(load().aidw_shard_range(int(n_query), int(shard), int(n_shards), ctypes.byref(b),
                                   ctypes.byref(e)), "aidw_shard_range")
    return b.value, e.value


def aidw_interpolate_shard(grid: Grid, qx, qy, shard: int, n_shards: int,
                           params: Params | None = None, out_z=None, out_alpha=None,
                           want_alpha: bool = False, stream=None):
    """Interpolates this shard's slice of the full query set (qx, qy) into
    full-length outputs; elements outside the slice are left as they were.
    Returns (z, alpha | None) full-length."""
    import torch
    p = params or Params()
    qx, qy = _f32_dev(qx, "qx"), _f32_dev(qy, "qy")
    m = qx.numel()
    if qy.numel() != m:
        raise ValueError("qx and qy must have the same length")
    dt = torch.float64 if p.precision == AIDW_FP64_PLAIN else torch.float32
    if out_z is None:
        out_z = torch.full((m,), float("nan"), dtype=dt, device=qx.device)
    if out_alpha is None and want_alpha:
        out_alpha = torch.full((m,), float("nan"), dtype=dt, device=qx.device)
    for t, name in ((out_z, "out_z"), (out_alpha, "out_alpha")):
        if t is not None and (t.dtype != dt or t.numel() != m or not t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous {dt} tensor of length {m}")
    pc = p.to_c()
    _check(load().aidw_interpolate_shard(grid.handle, _ptr(qx), _ptr(qy), m, int(shard),
                                         int(n_shards), ctypes.byref(pc), _ptr(out_z),
                                         _ptr(out_alpha), _stream(stream)),
           "aidw_interpolate_shard")
    return out_z, out_alpha


def aidw_test_expire_next_wait(tries: int = 50) -> None:
    """Test hook: the next weighting launch's bounded wait expires after tries."""
    _check(load().aidw_test_expire_next_wait(int(tries)), "aidw_test_expire_next_wait")


def aidw_set_memory_limit(nbytes: int) -> int:
    """Caps the library's pool memory (0: no cap); returns the bytes held now."""
    held = ctypes.c_int64()
    _check(load().aidw_set_memory_limit(int(nbytes), ctypes.byref(held)),
           "aidw_set_memory_limit")
    return held.value


def aidw_profile_enable(on: bool = True) -> None:
    _check(load().aidw_profile_enable(1 if on else 0), "aidw_profile_enable")


def aidw_profile_read() -> dict:
    """Per stage: (total ms, kernel launches) since the last read."""
    ms = (ctypes.c_double * len(STAGES))()
    ln = (ctypes.c_int64 * len(STAGES))()
    _check(load().aidw_profile_read(ms, ln), "aidw_profile_read")
    return {s: (ms[i], int(ln[i])) for i, s in enumerate(STAGES)}


def aidw_probe_pipe_rates() -> dict:
    """Per-SM per-clock rates of SFU lg2, SFU ex2 and packed FMA lanes."""
    r = [ctypes.c_double() for _ in range(3)]
    _check(load().aidw_probe_pipe_rates(*(ctypes.byref(v) for v in r)), "aidw_probe_pipe_rates")
    return {"lg2": r[0].value, "ex2": r[1].value, "ffma2_lanes": r[2].value}


def aidw_probe_weight_loop(ctas_per_sm: int = 2) -> float:
    """Pairs per SM per clock of the float32 weighting loop run alone (no
    copies, waits or barriers) at 2 or 3 CTAs per SM."""
    r = ctypes.c_double()
    _check(load().aidw_probe_weight_loop(int(ctas_per_sm), ctypes.byref(r)),
           "aidw_probe_weight_loop")
    return r.value


def aidw_bounds_report() -> dict:
    """Index-check record of the loaded library: whether it is the checked
    build, how many checks failed since it was loaded, and the site and
    index of the first failure (None if none)."""
    c, v, f = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().aidw_bounds_report(ctypes.byref(c), ctypes.byref(v), ctypes.byref(f)),
           "aidw_bounds_report")
    first = None if f.value == (1 << 64) - 1 else (f.value >> 48, f.value & ((1 << 48) - 1))
    return {"checked_build": bool(c.value), "violations": v.value, "first": first}


def aidw_test_bounds_check(index: int, n: int) -> bool:
    """Evaluates one index check on the GPU (no memory behind it); in the
    checked build an index outside [0, n) is recorded as a failure."""
    r = ctypes.c_int()
    _check(load().aidw_test_bounds_check(int(index), int(n), ctypes.byref(r)),
           "aidw_test_bounds_check")
    return bool(r.value)


def aidw_weight_mix() -> dict:
    """Instruction mix of the float32 weighting loop: products per inner
    step, how many take exp2 / log2 from FMA-pipe polynomials, and the
    FMA-pipe lane operations and other instructions per pair of the base
    loop and of each polynomial (host only, no GPU needed)."""
    prod, pe, pl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lanes = (ctypes.c_double * 3)()
    instr = (ctypes.c_double * 3)()
    _check(load().aidw_weight_mix(ctypes.byref(prod), ctypes.byref(pe), ctypes.byref(pl), lanes,
                                  instr), "aidw_weight_mix")
    return {"products": prod.value, "poly_exp2": pe.value, "poly_lg2": pl.value,
            "fma_lanes": {"base": lanes[0], "exp2_poly": lanes[1], "lg2_poly": lanes[2]},
            "instr": {"base": instr[0], "exp2_poly": instr[1], "lg2_poly": instr[2]}}


@dataclass
class BatchJob:
    """One job of a batch: device tensors (float32) and k (<= 0: params.k).
    out_z is allocated by ``batch_jobs_alloc`` when left None."""
    x: object
    y: object
    z: object
    qx: object
    qy: object
    k: int = 0
    out_z: object = None


def _c_jobs(jobs, params: Params):
    import torch
    arr = (CJob * len(jobs))()
    dt = torch.float64 if params.precision == AIDW_FP64_PLAIN else torch.float32
    for i, j in enumerate(jobs):
        for name in ("x", "y", "z", "qx", "qy"):
            _f32_dev(getattr(j, name), name)
        if j.out_z is None:
            j.out_z = torch.empty(j.qx.numel(), dtype=dt, device=j.qx.device)
        if j.out_z.dtype != dt or j.out_z.numel() != j.qx.numel():
            raise TypeError(f"job {i}: out_z must be {dt} of length {j.qx.numel()}")
        arr[i].x, arr[i].y, arr[i].z = j.x.data_ptr(), j.y.data_ptr(), j.z.data_ptr()
        arr[i].n_data = j.x.numel()
        arr[i].qx, arr[i].qy = j.qx.data_ptr(), j.qy.data_ptr()
        arr[i].n_query = j.qx.numel()
        arr[i].k = int(j.k)
        arr[i].out_z = j.out_z.data_ptr()
    return arr


@dataclass
class BatchPlan:
    """Owner of an aidw_batch_plan handle."""
    handle: ctypes.c_void_p
    params: Params
    n_jobs: int
    _alive: bool = field(default=True, repr=False)

    def destroy(self) -> None:
        if self._alive:
            self._alive = False
            _check(load().aidw_batch_plan_destroy(self.handle), "aidw_batch_plan_destroy")

    def __del__(self):
        if getattr(self, "_alive", False):
            try:
                self._alive = False
                load().aidw_batch_plan_destroy(self.handle)
            except Exception:
                pass


def aidw_batch_plan_create(jobs, params: Params | None = None) -> BatchPlan:
    p = params or Params()
    arr = _c_jobs(jobs, p)
    pc = p.to_c()
    h = ctypes.c_void_p()
    _check(load().aidw_batch_plan_create(arr, len(jobs), ctypes.byref(pc), ctypes.byref(h)),
           "aidw_batch_plan_create")
    return BatchPlan(h, p, len(jobs))


def aidw_batch_run(plan: BatchPlan, jobs, stream=None):
    arr = _c_jobs(jobs, plan.params)
    _check(load().aidw_batch_run(plan.handle, arr, _stream(stream)), "aidw_batch_run")
    return [j.out_z for j in jobs]


def aidw_batch_plan_tune(plan: BatchPlan, jobs, stream=None) -> float:
    arr = _c_jobs(jobs, plan.params)
    best = ctypes.c_double()
    _check(load().aidw_batch_plan_tune(plan.handle, arr, _stream(stream), ctypes.byref(best)),
           "aidw_batch_plan_tune")
    return best.value


def aidw_batch_plan_get(plan: BatchPlan) -> dict:
    cs, th = ctypes.c_double(), ctypes.c_int()
    pairs, pool = ctypes.c_int64(), ctypes.c_int64()
    _check(load().aidw_batch_plan_get(plan.handle, ctypes.byref(cs), ctypes.byref(th),
                                      ctypes.byref(pairs), ctypes.byref(pool)),
           "aidw_batch_plan_get")
    return {"cell_scale": cs.value, "knn_threads": th.value, "total_pairs": pairs.value,
            "pool_bytes": pool.value}


BATCH_CLASSES = 4


def aidw_batch_plan_get_classes(plan: BatchPlan) -> dict:
    """Per top-k class: slots, cell scale, kNN block size (0: warp per
    query), queries; and where the choices came from (defaults / tuner /
    cache)."""
    n = BATCH_CLASSES
    kmax, th = (ctypes.c_int * n)(), (ctypes.c_int * n)()
    sc, q = (ctypes.c_double * n)(), (ctypes.c_int64 * n)()
    src = ctypes.c_int()
    _check(load().aidw_batch_plan_get_classes(plan.handle, kmax, sc, th, q, ctypes.byref(src)),
           "aidw_batch_plan_get_classes")
    return {"classes": [{"kmax": kmax[c], "cell_scale": sc[c], "knn_threads": th[c],
                         "queries": q[c]} for c in range(n)],
            "source": ("defaults", "tuner", "cache")[src.value]}


def aidw_batch_plan_status(plan: BatchPlan) -> int:
    return int(load().aidw_batch_plan_status(plan.handle))


def aidw_batch_plan_destroy(plan: BatchPlan) -> None:
    plan.destroy()


def aidw_batch(jobs, params: Params | None = None, stream=None):
    p = params or Params()
    arr = _c_jobs(jobs, p)
    pc = p.to_c()
    _check(load().aidw_batch(arr, len(jobs), ctypes.byref(pc), _stream(stream)), "aidw_batch")
    return [j.out_z for j in jobs]


def interpolate_host(x, y, z, qx, qy, params: Params | None = None, stream=None,
                     want_alpha: bool = False):
    """End-to-end call from host arrays (aidw_interpolate_host): the library
    copies the inputs to the current device, builds the grid, interpolates
    and copies the predictions back.

    Inputs are numpy arrays or CPU tensors of float32 (pinned tensors copy
    asynchronously).  Returns a CPU tensor of predictions (float32, or
    float64 for AIDW_FP64_PLAIN), pinned, or (z, alpha) with want_alpha."""
    import numpy as np
    import torch
    p = params or Params()

    def host(a, name):
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        if t.is_cuda or t.dtype != torch.float32 or t.dim() != 1 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous 1-D float32 host array")
        return t
    x, y, z, qx, qy = (host(a, n) for a, n in ((x, "x"), (y, "y"), (z, "z"), (qx, "qx"),
                                               (qy, "qy")))
    if not (x.numel() == y.numel() == z.numel()) or qx.numel() != qy.numel():
        raise ValueError("x, y, z (and qx, qy) must have the same length")
    dt = torch.float64 if p.precision == AIDW_FP64_PLAIN else torch.float32
    m = qx.numel()
    out = torch.empty(m, dtype=dt, pin_memory=True)
    alpha = torch.empty(m, dtype=dt, pin_memory=True) if want_alpha else None
    pc = p.to_c()
    _check(load().aidw_interpolate_host(_ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(qx),
                                        _ptr(qy), m, ctypes.byref(pc), _ptr(out), _ptr(alpha),
                                        _stream(stream)), "aidw_interpolate_host")
    return (out, alpha) if want_alpha else out
