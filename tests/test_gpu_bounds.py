"""The bounds-checked build (libaidw_checked.so): with no GPU memory checker
available, the kernels of that build test every index they compute against
the array it indexes (cells, cell heads, scatter and fix-up destinations,
kNN ring segments, weighting tile copies and partial-sum slots) and count
the failures.  A child
process runs a spread of workloads through it - ragged and clustered grids
at several cell widths, a tiny grid, queries far outside the data, k from 1
to 32, both precisions, the local form, pieces of weighting tiles, a batch,
the no-allocation call and a query shard - and must report no failure and
the results of the normal build bit for bit (the checks change no
arithmetic).  A failure planted through a test hook (a check with no memory
access behind it) shows that the record keeps its site and index."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
def run(b, torch):
    import ctypes
    import numpy as np
    from paper_1601_05904_gb300 import inputs
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    h = lambda t: t.cpu().numpy()
    out = {}
    w = inputs.uniform_kilo(n=20011, m=3001, seed=91)
    for scale in (0.5, 2.0, 8.0):
        g = b.aidw_grid_build(d(w.x), d(w.y), d(w.z), b.Params(k=10, cell_scale=scale))
        cs, perm = b.aidw_grid_export(g)
        out[f"cs{scale}"], out[f"perm{scale}"] = h(cs), h(perm)
        for k in (1, 10, 32):
            idx, dist, robs = b.aidw_knn(g, d(w.qx), d(w.qy), k)
            out[f"idx{scale}_{k}"], out[f"dist{scale}_{k}"] = h(idx), h(dist)
        g.destroy()
    qx, qy = d(w.qx), d(w.qy)
    for prec in (b.AIDW_FP32_COMP, b.AIDW_FP64_PLAIN):
        p = b.Params(k=10, precision=prec)
        g = b.aidw_grid_build(d(w.x), d(w.y), d(w.z), p)
        z, a = b.aidw_interpolate(g, qx, qy, p, want_alpha=True)
        zl, _ = b.aidw_interpolate_local(g, qx, qy, p)
        out[f"z{prec}"], out[f"a{prec}"], out[f"zl{prec}"] = h(z), h(a), h(zl)
        g.destroy()
    # clustered data, 32 slots; queries far outside the data
    c = inputs.clustered_kilo(n=30000, m=4000, k=32, seed=92)
    g = b.aidw_grid_build(d(c.x), d(c.y), d(c.z), b.Params(k=32))
    fx = np.concatenate([c.qx, np.float32([-5000.0, 7000.0, 500.0])]).astype(np.float32)
    fy = np.concatenate([c.qy, np.float32([-5000.0, 300.0, 9000.0])]).astype(np.float32)
    z, _ = b.aidw_interpolate(g, d(fx), d(fy), b.Params(k=32))
    out["zc"] = h(z)
    # one query shard of two
    zs = torch.zeros(c.m, dtype=torch.float32, device="cuda")
    b.aidw_interpolate_shard(g, d(c.qx), d(c.qy), 1, 2, b.Params(k=32), out_z=zs)
    out["zshard"] = h(zs)
    # the no-allocation entry point
    lib = b.load()
    fn = lib.aidw_interpolate_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64] + [ctypes.c_void_p] * 4
    zn = torch.zeros(c.m, dtype=torch.float32, device="cuda")
    pc = b.Params(k=32).to_c()
    cqx, cqy = d(c.qx), d(c.qy)
    assert fn(g.handle, ctypes.c_void_p(cqx.data_ptr()), ctypes.c_void_p(cqy.data_ptr()), c.m,
              ctypes.byref(pc), ctypes.c_void_p(zn.data_ptr()), None,
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    out["znoalloc"] = h(zn)
    g.destroy()
    # a tiny grid (k = n) and a lattice with points on cell edges
    t = inputs.unit_square(n=5, m=50, k=5, seed=93)
    g = b.aidw_grid_build(d(t.x), d(t.y), d(t.z), b.Params(k=5))
    z, _ = b.aidw_interpolate(g, d(t.qx), d(t.qy), b.Params(k=5))
    out["ztiny"] = h(z)
    g.destroy()
    lx, ly = np.meshgrid(np.arange(64, dtype=np.float32), np.arange(64, dtype=np.float32))
    lx, ly = lx.ravel(), ly.ravel()
    lz = (lx * 0.5 - ly).astype(np.float32)
    g = b.aidw_grid_build(d(lx), d(ly), d(lz), b.Params(k=16, cell_scale=1.0))
    z, _ = b.aidw_interpolate(g, d(lx[::7] + 0.5), d(ly[::7]), b.Params(k=16))
    out["zlattice"] = h(z)
    g.destroy()
    # a batch of uneven jobs
    ws = inputs.batch_jobs(n_jobs=12, seed_base=94, n_lo=50, n_hi=20000)
    jobs = [b.BatchJob(d(j.x), d(j.y), d(j.z), d(j.qx), d(j.qy), j.k) for j in ws]
    outs = b.aidw_batch(jobs, b.Params(k=10))
    for i, o in enumerate(outs):
        out[f"batch{i}"] = h(o)
    torch.cuda.synchronize()
    return out
'''

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1601_05904_gb300 import binding as b
b.load(sys.argv[3])
ns = {}
exec(sys.argv[4], ns)
out = ns["run"](b, torch)
rep = b.aidw_bounds_report()
out["checked_build"] = np.int64(rep["checked_build"])
out["violations"] = np.int64(rep["violations"])
out["first"] = np.int64(-1 if rep["first"] is None else (rep["first"][0] << 48) | rep["first"][1])
# a failure planted through the test hook (a check with no access behind
# it) is recorded with its site and index
assert b.aidw_test_bounds_check(2, 3) is True
assert b.aidw_test_bounds_check(5, 3) is False
after = b.aidw_bounds_report()
out["planted"] = np.int64(after["violations"] - rep["violations"])
out["planted_first"] = np.int64(-1 if after["first"] is None else
                                (after["first"][0] << 48) | after["first"][1])
np.savez(sys.argv[2], **out)
'''


def test_checked_build_finds_no_out_of_range_index(aidw, tmp_path):
    import torch
    from paper_1601_05904_gb300 import build
    lib = build.build(checked=True)
    out = str(tmp_path / "checked.npz")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, out, lib, RUN],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = dict(np.load(out))
    assert got.pop("checked_build") == 1
    first = int(got.pop("first"))
    assert got.pop("violations") == 0, f"first failed check: site {first >> 48}, " \
                                        f"index {first & ((1 << 48) - 1)}"
    assert got.pop("planted") == 1
    assert int(got.pop("planted_first")) == (12 << 48) | 5
    ns = {}
    exec(RUN, ns)
    ref = ns["run"](aidw, torch)
    assert sorted(got) == sorted(ref)
    for key, v in ref.items():
        np.testing.assert_array_equal(got[key], v, err_msg=key)
    # the normal build: the check is the constant true, nothing is recorded
    assert aidw.aidw_test_bounds_check(5, 3) is True
    assert aidw.aidw_bounds_report() == {"checked_build": False, "violations": 0,
                                         "first": None}
