"""The C ABI library loads and exports every entry point include/aidw.h
declares, and its host-side argument checks answer without a GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aidw.h")


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(aidw_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1601_05904_gb300 import binding, build
    build.build()
    return binding.load()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("aidw_grid_build", "aidw_grid_destroy", "aidw_knn", "aidw_interpolate",
              "aidw_status_string", "aidw_params_default"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    from paper_1601_05904_gb300 import binding
    for code in range(7):
        s = binding.aidw_status_string(code)
        assert isinstance(s, str) and s
    assert binding.aidw_status_string(0) == "ok"


def test_params_default(lib):
    from paper_1601_05904_gb300 import binding
    p = binding.aidw_params_default()
    assert p.k == 10 and tuple(p.alpha) == (1.0, 2.0, 3.0, 4.0, 5.0)
    assert p.r_min == 0.0 and p.r_max == 2.0 and p.precision == binding.AIDW_FP32_COMP


def _params(**kw):
    from paper_1601_05904_gb300 import binding
    p = binding.Params(**kw).to_c()
    return p


@pytest.mark.parametrize("bad", [dict(alpha=(1, 2, -3, 4, 5)), dict(alpha=(0, 1, 2, 3, 4)),
                                 dict(r_min=2.0, r_max=1.0), dict(r_max=0.0),
                                 dict(cell_scale=1000.0), dict(precision=7),
                                 dict(area=float("nan")), dict(alpha=(1, 2, float("inf"), 4, 5))])
def test_grid_build_rejects_bad_params_before_any_cuda_call(lib, bad):
    p = _params(**bad)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    st = lib.aidw_grid_build(fake, fake, fake, 10, ctypes.byref(p), None, ctypes.byref(h))
    assert st == 1 and not h.value


def test_null_and_size_checks(lib):
    p = _params()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    assert lib.aidw_grid_build(None, fake, fake, 10, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert lib.aidw_grid_build(fake, fake, fake, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert lib.aidw_grid_build(fake, fake, fake, -5, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert lib.aidw_grid_build(fake, fake, fake, 10, None, None, ctypes.byref(h)) == 1
    assert lib.aidw_grid_build(fake, fake, fake, 10, ctypes.byref(p), None, None) == 1
    assert lib.aidw_knn(None, fake, fake, 10, 5, None, None, None, None) == 1
    assert lib.aidw_interpolate(None, fake, fake, 10, ctypes.byref(p), fake, None, None) == 1
    assert lib.aidw_grid_destroy(None) == 1
    assert lib.aidw_grid_status(None) == 1
    assert lib.aidw_grid_get_info(None, None) == 1
    assert lib.aidw_grid_export(None, None, None, None) == 1


def test_profile_toggle_without_work(lib):
    from paper_1601_05904_gb300 import binding
    binding.aidw_profile_enable(True)
    binding.aidw_profile_enable(False)
    r = binding.aidw_profile_read()
    assert set(r) == set(binding.STAGES)
    assert all(v == (0.0, 0) for v in r.values())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1601_05904_gb300 import binding
    with pytest.raises(RuntimeError, match="missing"):
        # a fresh loader pointed at a path that does not exist
        saved = binding._lib
        binding._lib = None
        try:
            binding.load(str(tmp_path / "nope.so"))
        finally:
            binding._lib = saved


def test_weight_mix_is_host_only(lib):
    """The weighting loop's instruction mix (roofline accounting) answers
    without a GPU; the default split takes 4 of 16 exp2s (over two inner
    steps) from the FMA pipe."""
    from paper_1601_05904_gb300 import binding
    mix = binding.aidw_weight_mix()
    assert mix["products"] == 16
    assert (mix["poly_exp2"], mix["poly_lg2"]) == (4, 0)
    assert mix["fma_lanes"] == {"base": 7.0, "exp2_poly": 8.0, "lg2_poly": 10.0}
    assert mix["instr"]["base"] == 3.5


@pytest.mark.parametrize("n,world", [(0, 1), (0, 3), (1, 4), (10, 3), (1 << 20, 8), (1000003, 7)])
def test_shard_range_partitions_the_queries(lib, n, world):
    """Shards are contiguous, in shard order, cover [0, n) exactly once and
    differ in size by at most one (the rule of aidw_shard_range)."""
    from paper_1601_05904_gb300 import binding
    sl = [binding.aidw_shard_range(n, r, world) for r in range(world)]
    assert sl[0][0] == 0 and sl[-1][1] == n
    for (b0, e0), (b1, e1) in zip(sl, sl[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in sl]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)


def test_shard_range_rejects_bad_shards(lib):
    b, e = ctypes.c_int64(), ctypes.c_int64()
    for n, r, w in ((-1, 0, 1), (10, 1, 1), (10, -1, 2), (10, 0, 0)):
        assert lib.aidw_shard_range(n, r, w, ctypes.byref(b), ctypes.byref(e)) == 1
    assert lib.aidw_shard_range(10, 0, 1, None, ctypes.byref(e)) == 1


def test_host_entry_point_checks_arguments_without_a_gpu(lib):
    """aidw_interpolate_host rejects bad arguments before any CUDA call."""
    from paper_1601_05904_gb300 import binding
    pc = _params(k=2)
    a = (ctypes.c_float * 4)()
    out = (ctypes.c_float * 4)()
    f = lib.aidw_interpolate_host
    assert f(None, a, a, 4, a, a, 4, ctypes.byref(pc), out, None, None) == 1
    assert f(a, a, a, 0, a, a, 4, ctypes.byref(pc), out, None, None) == 1
    assert f(a, a, a, 4, None, a, 4, ctypes.byref(pc), out, None, None) == 1
    assert f(a, a, a, 4, a, a, 4, ctypes.byref(pc), None, None, None) == 1
    assert f(a, a, a, 4, a, a, -1, ctypes.byref(pc), out, None, None) == 1
    p5 = _params(k=5)
    assert f(a, a, a, 4, a, a, 4, ctypes.byref(p5), out, None, None) == 2   # k > n_data
    del binding


def _nvtx_recorder(tmp_path):
    """Builds the test NVTX tool (tests/c_abi/nvtx_recorder.c)."""
    cuda_inc = "/usr/local/cuda/include"
    nvcc = shutil.which("nvcc")
    if nvcc:
        cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    out = str(tmp_path / "nvtx_recorder.so")
    import subprocess
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-I", cuda_inc,
                        os.path.join(ROOT, "tests", "c_abi", "nvtx_recorder.c"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_entry_points_open_and_close_named_nvtx_ranges(lib, tmp_path):
    """Every C-ABI call opens an NVTX range named after it and closes it on
    every return path, the argument errors included (no GPU needed)."""
    import subprocess
    import sys
    rec = _nvtx_recorder(tmp_path)
    log = tmp_path / "nvtx.log"
    script = (
        "import ctypes\n"
        "from paper_1601_05904_gb300 import binding\n"
        "lib = binding.load()\n"
        "pc = binding.Params(k=2).to_c()\n"
        "a = (ctypes.c_float * 4)(); out = (ctypes.c_float * 4)()\n"
        "assert lib.aidw_interpolate_host(None, a, a, 4, a, a, 4, ctypes.byref(pc), out, None, None) == 1\n"
        "assert lib.aidw_interpolate_shard(None, None, None, 4, 0, 1, ctypes.byref(pc), None, None, None) == 1\n"
        "assert lib.aidw_batch_run(None, None, None) == 1\n")
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, AIDW_NVTX_LOG=str(log),
               PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert log.read_text().split("\n")[:-1] == [
        "push aidw_interpolate_host", "pop", "push aidw_interpolate_shard", "pop",
        "push aidw_batch_run", "pop"]


def test_weight_loop_probe_checks_arguments_without_a_gpu(lib):
    """aidw_probe_weight_loop takes 2 or 3 CTAs per SM and a non-NULL output,
    checked before any CUDA call."""
    d = ctypes.c_double(-1.0)
    assert lib.aidw_probe_weight_loop(4, ctypes.byref(d)) == 1
    assert lib.aidw_probe_weight_loop(1, ctypes.byref(d)) == 1
    assert lib.aidw_probe_weight_loop(2, None) == 1


def test_bounds_report_of_the_normal_build(lib):
    """The normal build carries no index checks: the report says so, with
    no failures, and needs no GPU."""
    c, v, f = ctypes.c_int(-1), ctypes.c_uint64(7), ctypes.c_uint64(0)
    assert lib.aidw_bounds_report(ctypes.byref(c), ctypes.byref(v), ctypes.byref(f)) == 0
    assert c.value == 0 and v.value == 0 and f.value == (1 << 64) - 1
    assert lib.aidw_bounds_report(None, None, None) == 0


def test_checked_build_exports_every_symbol():
    """The bounds-checked build of the same sources links and exports every
    entry point include/aidw.h declares."""
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1601_05904_gb300 import build
    checked = ctypes.CDLL(build.build(checked=True))
    missing = [n for n in declared_functions() if not hasattr(checked, n)]
    assert not missing, missing
