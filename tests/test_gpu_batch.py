"""Batched AIDW (many independent jobs in one pass): every job's predictions
equal the single-job path's and the oracle's, across job sizes, k, graph
replays with new buffers, the autotuner and error paths."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, dev, host
from paper_1601_05904_gb300 import inputs

pytestmark = pytest.mark.gpu


def _jobs(aidw, spec, seed=0):
    """spec: list of (n, m, k, clustered_fraction)."""
    jobs, raw = [], []
    for j, (n, m, k, frac) in enumerate(spec):
        rng = np.random.default_rng(seed * 1000 + j)
        x, y = inputs.mixed_points(rng, n, frac, 4)
        z = inputs.field_kilo(rng, x, y)
        qx, qy = inputs.uniform_points(rng, m, 0.0, 1000.0)
        raw.append((x, y, z, qx, qy, k))
        jobs.append(aidw.BatchJob(dev(x), dev(y), dev(z), dev(qx), dev(qy), k))
    return jobs, raw


SPEC = [(1, 5, 1, 0.0), (10, 0, 8, 0.0), (33, 100, 8, 0.5), (1000, 1500, 10, 0.3),
        (4097, 3001, 16, 0.9), (2500, 1024, 24, 0.0), (700, 2049, 32, 0.6),
        (12000, 5000, 10, 0.8), (64, 64, 17, 0.0), (3000, 1, 12, 0.2)]


@pytest.mark.parametrize("fp64", [False, True])
def test_batch_matches_single_job_and_oracle(aidw, oracle, fp64):
    prec = aidw.AIDW_FP64_PLAIN if fp64 else aidw.AIDW_FP32_COMP
    p = aidw.Params(k=10, precision=prec)
    jobs, raw = _jobs(aidw, SPEC, seed=1)
    plan = aidw.aidw_batch_plan_create(jobs, p)
    outs = aidw.aidw_batch_run(plan, jobs)
    assert aidw.aidw_batch_plan_status(plan) == 0
    tol = TOL_FP64 if fp64 else TOL_FP32
    for (x, y, z, qx, qy, k), o in zip(raw, outs):
        if qx.size == 0:
            assert o.numel() == 0
            continue
        got = host(o).astype(np.float64)
        ref = oracle.aidw(x, y, z, qx, qy, k)
        err = oracle.normalized_error(got, ref["z"], ref["scale"])
        assert err.max() <= tol, err.max()
        ps = aidw.Params(k=k, precision=prec)
        g = aidw.aidw_grid_build(dev(x), dev(y), dev(z), ps)
        single, _ = aidw.aidw_interpolate(g, dev(qx), dev(qy), ps)
        g.destroy()
        np.testing.assert_allclose(got, host(single).astype(np.float64), rtol=0,
                                   atol=(2 * tol) * np.abs(z).max())
    plan.destroy()


def test_graph_replay_with_new_buffers(aidw, oracle):
    p = aidw.Params(k=10)
    jobs_a, raw_a = _jobs(aidw, SPEC, seed=2)
    jobs_b, raw_b = _jobs(aidw, SPEC, seed=3)   # same shapes, other data
    plan = aidw.aidw_batch_plan_create(jobs_a, p)
    for jobs, raw in ((jobs_a, raw_a), (jobs_b, raw_b), (jobs_a, raw_a)):
        for j in jobs:
            j.out_z = None
        outs = aidw.aidw_batch_run(plan, jobs)
        assert aidw.aidw_batch_plan_status(plan) == 0
        for (x, y, z, qx, qy, k), o in zip(raw, outs):
            if qx.size:
                ref = oracle.aidw(x, y, z, qx, qy, k)
                assert oracle.normalized_error(host(o), ref["z"], ref["scale"]).max() <= TOL_FP32
    plan.destroy()


def test_autotuner_keeps_results(aidw, oracle):
    """Retuning changes the cell width and kNN shape, hence the rounding
    order of the sums only: before and after, every job is within the
    float32 tolerance of the oracle."""
    p = aidw.Params(k=10)
    jobs, raw = _jobs(aidw, [(20000, 4000, 10, 0.9), (5000, 3000, 24, 0.0)] * 3, seed=4)
    plan = aidw.aidw_batch_plan_create(jobs, p)
    before = [host(o).copy() for o in aidw.aidw_batch_run(plan, jobs)]
    best = aidw.aidw_batch_plan_tune(plan, jobs)
    info = aidw.aidw_batch_plan_get(plan)
    assert best > 0 and info["cell_scale"] in (1.0, 1.5, 2.0, 3.0, 4.0)
    assert info["knn_threads"] in (0, 64, 128, 256)   # 0: warp per query
    for j in jobs:
        j.out_z = None
    after = [host(o) for o in aidw.aidw_batch_run(plan, jobs)]
    assert aidw.aidw_batch_plan_status(plan) == 0
    for a, b, (x, y, z, qx, qy, k) in zip(before, after, raw):
        ref = oracle.aidw(x, y, z, qx, qy, k)
        for out in (a, b):
            assert oracle.normalized_error(out, ref["z"], ref["scale"]).max() <= TOL_FP32
    plan.destroy()


def test_one_shot_batch(aidw, oracle):
    jobs, raw = _jobs(aidw, SPEC[:5], seed=5)
    outs = aidw.aidw_batch(jobs, aidw.Params(k=10))
    for (x, y, z, qx, qy, k), o in zip(raw, outs):
        if qx.size:
            ref = oracle.aidw(x, y, z, qx, qy, k)
            assert oracle.normalized_error(host(o), ref["z"], ref["scale"]).max() <= TOL_FP32


def test_batch_workload_sampled(aidw, oracle):
    """A slice of the 512-job workload (n_j log-uniform in [1e3, 2e5],
    k_j in {8,10,16,24,32}, mixed clustering): the first 48 jobs, every job
    checked on a sample of its queries."""
    ws = inputs.batch_jobs(n_jobs=48)
    jobs = [aidw.BatchJob(dev(w.x), dev(w.y), dev(w.z), dev(w.qx), dev(w.qy), w.k) for w in ws]
    outs = aidw.aidw_batch(jobs, aidw.Params(k=10))
    for w, o in zip(ws, outs):
        s = inputs.query_subsample(w.m, 24, seed=w.seed)
        ref = oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k)
        err = oracle.normalized_error(host(o)[s], ref["z"], ref["scale"])
        assert err.max() <= TOL_FP32, (w.name, err.max())


def test_batch_errors(aidw):
    p = aidw.Params(k=10)
    jobs, raw = _jobs(aidw, [(100, 10, 10, 0.0), (50, 10, 8, 0.0)], seed=6)
    plan = aidw.aidw_batch_plan_create(jobs, p)
    other, _ = _jobs(aidw, [(100, 10, 10, 0.0), (51, 10, 8, 0.0)], seed=6)
    with pytest.raises(aidw.AidwError) as e:
        aidw.aidw_batch_run(plan, other)
    assert e.value.status == 1
    plan.destroy()
    bad, _ = _jobs(aidw, [(5, 10, 8, 0.0)], seed=7)
    with pytest.raises(aidw.AidwError) as e:
        aidw.aidw_batch_plan_create(bad, p)
    assert e.value.status == 2
    # a non-finite data value in one job is reported by the plan status
    jobs, raw = _jobs(aidw, [(100, 10, 10, 0.0), (200, 10, 10, 0.0)], seed=8)
    zz = raw[1][2].copy()
    zz[7] = np.nan
    jobs[1].z = dev(zz)
    plan = aidw.aidw_batch_plan_create(jobs, p)
    outs = aidw.aidw_batch_run(plan, jobs)
    assert aidw.aidw_batch_plan_status(plan) == 3
    # the failed job's predictions are NaN; the other job is unaffected
    assert np.isnan(host(outs[1])).all()
    x, y, z, qx, qy, k = raw[0]
    assert np.isfinite(host(outs[0])).all()
    plan.destroy()


SPEC_CLASSES = [(6000, 2000, 8, 0.5), (6000, 2000, 12, 0.0), (4000, 2500, 20, 0.7),
                (3000, 1000, 32, 0.2)] * 2


def test_tuning_per_top_k_class_and_cache(aidw, oracle):
    """Jobs fall into the top-k classes 8/16/24/32; the tuner chooses a cell
    scale and kNN block size per class; a new plan for jobs of the same
    shapes starts from the cached choice; results stay within tolerance."""
    p = aidw.Params(k=10)
    jobs, raw = _jobs(aidw, SPEC_CLASSES, seed=9)
    plan = aidw.aidw_batch_plan_create(jobs, p)
    info = aidw.aidw_batch_plan_get_classes(plan)
    assert info["source"] == "defaults"
    cls = info["classes"]
    assert [c["kmax"] for c in cls] == [8, 16, 24, 32]
    assert [c["queries"] for c in cls] == [4000, 4000, 5000, 2000]
    assert [c["cell_scale"] for c in cls] == [2.0, 2.0, 3.0, 3.0]
    aidw.aidw_batch_plan_tune(plan, jobs)
    tuned = aidw.aidw_batch_plan_get_classes(plan)
    assert tuned["source"] == "tuner"
    for c in tuned["classes"]:
        assert c["cell_scale"] in (1.0, 1.5, 2.0, 3.0, 4.0)
        assert c["knn_threads"] in (0, 64, 128, 256)
    outs = aidw.aidw_batch_run(plan, jobs)
    assert aidw.aidw_batch_plan_status(plan) == 0
    for (x, y, z, qx, qy, k), o in zip(raw, outs):
        ref = oracle.aidw(x, y, z, qx, qy, k)
        assert oracle.normalized_error(host(o), ref["z"], ref["scale"]).max() <= TOL_FP32
    plan.destroy()
    # same shapes, other data: the cached tuning applies at creation
    jobs2, raw2 = _jobs(aidw, SPEC_CLASSES, seed=10)
    plan2 = aidw.aidw_batch_plan_create(jobs2, p)
    cached = aidw.aidw_batch_plan_get_classes(plan2)
    assert cached["source"] == "cache"
    assert cached["classes"] == tuned["classes"]
    outs = aidw.aidw_batch_run(plan2, jobs2)
    assert aidw.aidw_batch_plan_status(plan2) == 0
    for (x, y, z, qx, qy, k), o in zip(raw2, outs):
        ref = oracle.aidw(x, y, z, qx, qy, k)
        assert oracle.normalized_error(host(o), ref["z"], ref["scale"]).max() <= TOL_FP32
    plan2.destroy()


_CACHE_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_1601_05904_gb300 as aidw
from test_gpu_batch import SPEC_CLASSES, _jobs
aidw.load()
jobs, _ = _jobs(aidw, SPEC_CLASSES, seed=11)
plan = aidw.aidw_batch_plan_create(jobs, aidw.Params(k=10))
if sys.argv[1] == "tune":
    aidw.aidw_batch_plan_tune(plan, jobs)
print(json.dumps(aidw.aidw_batch_plan_get_classes(plan)))
plan.destroy()
"""


def test_tuning_cache_file_reaches_a_new_process(tmp_path):
    """With AIDW_TUNE_CACHE=<file>, a tuning measured in one process is the
    starting choice of a plan for the same shapes in the next process."""
    import json
    import os
    import subprocess
    import sys
    tests = os.path.dirname(os.path.abspath(__file__))
    script = tmp_path / "cache_probe.py"
    script.write_text(_CACHE_SCRIPT.format(root=os.path.dirname(tests), tests=tests))
    env = dict(os.environ, AIDW_TUNE_CACHE=str(tmp_path / "tune.txt"))

    def run(mode):
        r = subprocess.run([sys.executable, str(script), mode], capture_output=True, text=True,
                           env=env, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])
    first = run("tune")
    assert first["source"] == "tuner"
    lines = (tmp_path / "tune.txt").read_text().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])        # one JSON object per line
    assert entry["cell_scale"] == [c["cell_scale"] for c in first["classes"]]
    assert entry["knn_threads"] == [c["knn_threads"] for c in first["classes"]]
    second = run("create")
    assert second["source"] == "cache"
    assert second["classes"] == first["classes"]
