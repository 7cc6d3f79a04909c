"""The C ABI from C: a plain C program (tests/c_abi/abi_client.c) links
libaidw.so and the CUDA runtime and calls the library through
include/aidw.h alone; its outputs are checked against the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, check_knn
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


@pytest.fixture(scope="module")
def client(tmp_path_factory, aidw):
    from paper_1601_05904_gb300 import build
    lib = build.build()
    cuda = _cuda_home()
    out = str(tmp_path_factory.mktemp("c_abi") / "abi_client")
    cmd = ["gcc", "-O2", "-std=c11", os.path.join(HERE, "c_abi", "abi_client.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           "-o", out, "-L", os.path.dirname(lib), "-laidw", f"-Wl,-rpath,{os.path.dirname(lib)}",
           "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_c_client_matches_the_oracle(client, oracle, tmp_path):
    w = inputs.clustered_kilo(n=12000, m=2500, k=10, seed=61)
    for name in ("x", "y", "z", "qx", "qy"):
        getattr(w, name).astype(np.float32).tofile(tmp_path / f"{name}.bin")
    r = subprocess.run([client, str(tmp_path), str(w.n), str(w.m), str(w.k)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr + r.stdout
    assert r.stdout.startswith("ok")

    def load(name, dt, shape=None):
        a = np.fromfile(tmp_path / name, dtype=dt)
        return a.reshape(shape) if shape else a

    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k)
    for name, dt, tol in (("z32.bin", np.float32, TOL_FP32), ("z64.bin", np.float64, TOL_FP64),
                          ("zbatch0.bin", np.float32, TOL_FP32)):
        err = oracle.normalized_error(load(name, dt), ref["z"], ref["scale"])
        assert err.max() <= tol, (name, err.max())
    np.testing.assert_allclose(load("alpha32.bin", np.float32), ref["alpha"], atol=1e-5)
    # the end-to-end call from host arrays runs the same kernels
    np.testing.assert_array_equal(load("zhost.bin", np.float32), load("z32.bin", np.float32))
    np.testing.assert_array_equal(load("alphahost.bin", np.float32),
                                  load("alpha32.bin", np.float32))
    ref4 = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, 4)
    assert oracle.normalized_error(load("zbatch1.bin", np.float32), ref4["z"],
                                   ref4["scale"]).max() <= TOL_FP32
    loc = oracle.aidw_local(w.x, w.y, w.z, w.qx, w.qy, w.k)
    assert oracle.normalized_error(load("zlocal.bin", np.float32), loc["z"],
                                   loc["scale"]).max() <= TOL_FP32
    check_knn(oracle, w.x, w.y, w.qx, w.qy, w.k, load("idx.bin", np.int32, (w.m, w.k)),
              load("dist.bin", np.float32, (w.m, w.k)), load("robs.bin", np.float32))


def _nvtx_tree(lines):
    """Parses the recorder's "push name" / "pop" lines into (name, children)."""
    root = ("", [])
    stack = [root]
    for ln in lines:
        if ln.startswith("push "):
            node = (ln[5:], [])
            stack[-1][1].append(node)
            stack.append(node)
        else:
            assert ln == "pop" and len(stack) > 1, "pop without push"
            stack.pop()
    assert len(stack) == 1, "ranges left open"
    return root[1]


def test_nvtx_ranges_name_each_call_and_its_stages(aidw, tmp_path):
    """With an NVTX tool attached, the grid build, the interpolation and the
    batch each appear as a range named after the C-ABI call, with the stages
    they launch (grid build; kNN, weighting; graph capture) nested inside."""
    import sys
    from paper_1601_05904_gb300 import build
    build.build()
    rec = str(tmp_path / "nvtx_recorder.so")
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                        "-I", os.path.join(_cuda_home(), "include"),
                        os.path.join(HERE, "c_abi", "nvtx_recorder.c"), "-o", rec],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    log = tmp_path / "nvtx.log"
    script = (
        "import numpy as np, torch\n"
        "from paper_1601_05904_gb300 import binding as b, inputs\n"
        "w = inputs.uniform_kilo(n=5000, m=700, seed=62)\n"
        "d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()\n"
        "p = b.Params(k=10)\n"
        "g = b.aidw_grid_build(d(w.x), d(w.y), d(w.z), p)\n"
        "z, _ = b.aidw_interpolate(g, d(w.qx), d(w.qy), p)\n"
        "jobs = [b.BatchJob(d(w.x), d(w.y), d(w.z), d(w.qx), d(w.qy), k) for k in (6, 10)]\n"
        "b.aidw_batch(jobs, p)\n"
        "torch.cuda.synchronize()\n"
        "assert bool(torch.isfinite(z).all())\n")
    env = dict(os.environ, NVTX_INJECTION64_PATH=rec, AIDW_NVTX_LOG=str(log), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    tree = _nvtx_tree(log.read_text().split("\n")[:-1])
    top = [n for n, _ in tree]
    assert top == ["aidw_grid_build", "aidw_interpolate", "aidw_batch"], top
    kids = {n: [c for c, _ in ch] for n, ch in tree}
    assert kids["aidw_grid_build"] == ["grid build"]
    assert kids["aidw_interpolate"] == ["knn", "weighting"]
    assert kids["aidw_batch"] == ["aidw_batch_plan_create", "aidw_batch_run"]
    run = dict(tree)["aidw_batch"][1][1]
    assert [c for c, _ in run] == ["graph capture"]
