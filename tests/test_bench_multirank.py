"""The bench's multi-process path on the CPU (gloo, world size 2): the
whole-job figures take the slowest rank's time and all ranks' converged
solves, and the reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [100.0 + 50.0 * rank, 80.0 - 10.0 * rank, 60.0]
    conv = [10, 10 + rank, 9]
    t, c = bench.reduce_over_ranks(times, conv, dist, "cpu")
    q.put((rank, t, c, bench.solves_per_second(c[0], 3, t[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, c, v in out:
        assert t == [150.0, 80.0, 60.0]          # slowest rank per figure
        assert c == [20, 21, 18]                 # all ranks' converged solves
        assert v == pytest.approx(20 * 3 / 0.150)


def test_one_process_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    t, c = bench.reduce_over_ranks([1.0, 2.0], [3, 4], None, "cpu")
    assert t == [1.0, 2.0] and c == [3, 4]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
