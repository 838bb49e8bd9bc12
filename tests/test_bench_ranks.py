"""The multi-rank bench path on CPU: N independent replicas (one per rank, no collective on the
data path) report the slowest rank's time and the cells all ranks updated; the reference arm runs
on rank 0 only. World size 2 over gloo, no GPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    ms, mlups = bench.job_throughput(local_ms, 1000, 5, dist, torch, device="cpu")
    dist.destroy_process_group()
    q.put((rank, ms, mlups))


def test_replicas_report_max_time_and_whole_job_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, mlups in out:
        assert ms == 20.0  # max over ranks
        assert mlups == pytest.approx(1000 * 5 * 2 / 20e-3 / 1e6)


def test_single_rank_is_plain_throughput():
    sys.path.insert(0, ROOT)
    import torch
    import bench
    ms, mlups = bench.job_throughput(4.0, 2000, 10, None, torch, device="cpu")
    assert ms == 4.0 and mlups == pytest.approx(2000 * 10 / 4e-3 / 1e6)


def test_reference_arm_other_ranks_exit_without_output():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_oracle_per_config_rows():
    """The per-workload oracle timing (bench.py --mode oracle): one positive MLUPS row for each
    of the four workloads, on a tiny budget."""
    sys.path.insert(0, ROOT)
    import bench
    rows = bench.oracle_per_config(budget_s=0.05)
    assert [r[0][0] for r in rows] == ["1", "2", "3", "4"]
    assert all(r[1] > 0 for r in rows)
