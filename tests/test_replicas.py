"""The N>1 path of bench.py on the CPU: replicas with no data-path collective, whose timing is
the maximum over ranks (gloo, world size 2, 127.0.0.1) and whose value is all ranks' units over
that time; and the reference arm, which rank 0 alone runs under torchrun."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.distributed.barrier()
        t = bench.max_over_ranks(times[rank], "cpu")
        q.put((rank, t, bench.job_rate(100, world, t[0])))
    finally:
        torch.distributed.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    times = [[1.0, 5.0], [2.5, 3.0]]  # (device time, end-to-end time) per rank
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (t, v)) for r, t, v in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t, v = out[r]
        assert t == [2.5, 5.0]            # each entry: the slowest rank's
        assert v == pytest.approx(200 / 2.5)  # both ranks' units over the slowest time


def test_max_over_ranks_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.0], "cpu") == [1.5, 2.0]
    assert bench.job_rate(8, 1, 2.0) == 4.0


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
