"""The multi-rank host logic of the benchmark on CPU: two ranks over gloo.

The counting path shards by recording (every rank mines its own recording, no data
exchange), so the only cross-rank steps are the barrier around the timed region and
the reduction of (max time, summed work) that gives the whole-job throughput."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      FEM_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    r, w, loc = bench.dist_setup()
    try:
        bench.barrier(w)
        tmax, tsum = bench.reduce_max_sum(w, 1.5 + rank, 10.0 * (rank + 1))
        cfg = bench.workload(r)
        out_q.put((r, w, loc, tmax, tsum, int(cfg["stream"].n), float(cfg["stream"].t[-1])))
        bench.barrier(w)
    finally:
        import torch.distributed as dist
        dist.destroy_process_group()


def test_two_rank_barrier_and_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, loc, tmax, tsum, n, tlast in got:
        assert w == 2 and loc == r
        assert tmax == 2.5          # max over ranks of the step time
        assert tsum == 30.0         # sum over ranks of the work units
    # weak scaling: each rank mines a recording of its own (different seed)
    assert (got[0][5], got[0][6]) != (got[1][5], got[1][6])


def test_reference_arm_two_ranks_prints_one_line():
    """Under torchrun the reference arm runs on rank 0 only; rank 1 exits 0 without work."""
    port = free_port()
    env = dict(os.environ, FEM_BENCH_BACKEND="gloo", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle"
