"""The N > 1 path of bench.py on the CPU: ranks are replicas (each searches its own batch, no
collective on the data path); the job's time is the slowest rank's and its throughput counts every
rank's queries. Two gloo ranks on 127.0.0.1."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r ran its 5 steps of 10,000 queries in (r + 1) * 100 ms
    total, qps = bench.job_totals(100.0 * (rank + 1), world, 10_000, 5, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(out, "w") as f:
        f.write(f"{total} {qps}")


def test_two_replicas_report_the_slowest_rank_and_all_queries(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    outs = [str(tmp_path / f"r{r}.txt") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for o in outs:
        total, qps = map(float, open(o).read().split())
        assert total == 200.0                         # the slowest rank's time
        assert qps == pytest.approx(2 * 10_000 * 5 / 0.2)


def test_single_process_totals_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    total, qps = bench.job_totals(50.0, 1, 1000, 10)
    assert total == 50.0 and qps == pytest.approx(1000 * 10 / 0.05)


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun only rank 0 times the oracle; the other ranks exit 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
