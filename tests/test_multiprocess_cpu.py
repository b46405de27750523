"""The bench's N > 1 path on CPU with the gloo backend (world size 2): ranks are
independent replicas joined only by a barrier and the max of their timed
regions; the whole-job value counts every rank's output over the slowest
rank's time; under torchrun the reference arm prints one line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), NVISR_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank  # the replicas' own timed regions
    ms_max = bench.allmax(ms, w)
    out.put((rank, ms_max, bench.job_value(w, 3, 1000000, ms_max)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]  # every rank sees the slowest rank's time
    # 2 ranks x 3 steps x 1 Mpix over 15 ms
    assert res[0][2] == pytest.approx(2 * 3 * 1.0 / 15e-3)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    env = dict(os.environ, NVISR_BENCH_GLOO="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
