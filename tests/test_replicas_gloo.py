"""The multi-GPU mode of bench.py is replicas only: runs are independent, so
ranks shard them by seed and exchange only their timing and counts.  Checked
here with two gloo ranks on the CPU (no GPU): disjoint seeds, the slowest
rank's time and the summed evaluations."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 5)
        t, e = bench.combine_ranks(1.5 + rank, 100 * (rank + 1), dist, "cpu")
        q.put((rank, seeds, t, e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    s0, s1 = set(out[0][1]), set(out[1][1])
    assert len(s0) == 5 and len(s1) == 5 and not (s0 & s1)
    for rank, seeds, t, e in out:
        assert t == 2.5 and e == 300.0


def test_single_process_combine():
    import bench
    assert bench.combine_ranks(2.0, 7, None, "cpu") == (2.0, 7.0)
