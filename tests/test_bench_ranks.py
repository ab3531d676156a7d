"""The N > 1 bench path on CPU: independent replicas with the max-over-ranks clock
(gloo, world size 2), and the reference arm staying silent on ranks other than 0."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms, e2e_ms = bench.max_over_ranks([10.0 + rank, 30.0 - 5.0 * rank], dist)
        dist.barrier()
        out[rank] = (step_ms, e2e_ms, bench.job_rate(world, step_ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        step_ms, e2e_ms, rate = res[r]
        assert step_ms == 11.0 and e2e_ms == 30.0   # the slowest rank of each entry
        assert rate == pytest.approx(2 * 1e3 / 11.0)


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], None) == [3.0, 4.0]
    assert bench.job_rate(1, 50.0) == pytest.approx(20.0)


def test_reference_arm_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
