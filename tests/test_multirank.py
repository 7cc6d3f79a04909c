"""Host-side logic of the multi-GPU paths, run as two gloo ranks on CPU:
the query-sharded benchmark (every rank gets the same data points and its
own queries, and the reported time is the slowest rank's), and the
sharding of one query set (each rank computes its slice, the all-gathered
slices equal the one-process result)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)

        class A:
            n, k, workload = 4096, 10, "uniform"
        w = bench.make_workload(A, rank)
        sums = torch.tensor([float(np.float64(w.x).sum()), float(np.float64(w.qx).sum())],
                            dtype=torch.float64)
        gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, sums)
        t = bench.max_over_ranks(1.0 + rank)
        out.put((rank, [g.tolist() for g in gathered], t,
                 bench.whole_job_value(world, w.m, 3, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_data_shard_queries_and_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, gathered, t, value in res:
        (x0, q0), (x1, q1) = gathered
        assert x0 == x1          # same data points on every rank
        assert q0 != q1          # each rank its own queries
        assert t == 2.0          # max over ranks
        assert value == pytest.approx(2 * 4096 * 3 / 2.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero(tmp_path):
    """`bench.py --impl reference` launched as two ranks: rank 0 alone times
    the oracle (on all of the host's cores, although the launcher sets
    OMP_NUM_THREADS=1 per rank) and prints the one JSON line; the other rank
    exits 0 without work."""
    import json
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    import oracle
    if oracle.has_openmp():
        assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))


def _shard_rank(rank, world, port, out):
    """One rank of a sharded interpolation with the oracle standing in for
    the GPU: the slice comes from the library's aidw_shard_range (host
    only), the gather is the package's gather_slices."""
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1601_05904_gb300 import binding, inputs, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        binding.load()
        w = inputs.unit_square(n=1500, m=301, k=7, seed=5)
        b, e = binding.aidw_shard_range(w.m, rank, world)
        local = torch.full((w.m,), float("nan"), dtype=torch.float64)
        if e > b:
            local[b:e] = torch.from_numpy(
                oracle.aidw(w.x, w.y, w.z, w.qx[b:e], w.qy[b:e], w.k, nthreads=1)["z"])
        full = shard.gather_slices(local, w.m)
        out.put((rank, (b, e), full.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_queries_gather_to_the_one_process_result(world):
    import multiprocessing as mp
    oracle = pytest.importorskip("oracle")
    from paper_1601_05904_gb300 import build, inputs
    build.build()
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = inputs.unit_square(n=1500, m=301, k=7, seed=5)
    ref = oracle.aidw(w.x, w.y, w.z, w.qx, w.qy, w.k, nthreads=1)["z"]
    # the slices tile the query set, and every rank holds the whole result
    assert [r[1] for r in res][0][0] == 0 and res[-1][1][1] == w.m
    for rank, _, full in res:
        np.testing.assert_array_equal(full, ref)
