"""Host logic of the multi-GPU run (replicas only): every rank runs its own
replica and the job reports the maximum time over ranks and the units of all
ranks.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate_over_ranks(10.0 * (rank + 1), 1000.0, world)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_replicas_report_the_slowest_rank_and_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000.0 / 0.020)


def test_single_rank_is_unchanged():
    import bench
    ms, value = bench.aggregate_over_ranks(4.0, 500.0, 1)
    assert ms == 4.0 and value == pytest.approx(500.0 / 0.004)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host cores) runs
    and prints on rank 0 alone; every other rank exits 0 without work."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
