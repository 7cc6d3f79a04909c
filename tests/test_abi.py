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
