"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU), as
bench.py runs one independent replica per GPU under torchrun (weak scaling,
no collective on the data path).  The job's time is the slowest rank's, the
job's rate counts every rank's projections, and the reference arm does its
work on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + 5 r ms for its K steps
        t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        rate = bench.job_rate(2 * 4, world, t / 1e3)
        dist.barrier()
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in got:
        assert t == 15.0                       # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 4 * 2 / 0.015)


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun the reference arm runs on rank 0 only; rank 1 leaves at
    # once with status 0 and prints nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
