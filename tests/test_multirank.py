"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1). Under
torchrun every rank runs its own replica ("replicas only"); the step time
reported is the slowest rank's, and the reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, l = bench.dist_env()
        slowest = bench.slowest_over_ranks(10.0 + 5.0 * rank, w)
        ref = bench.run_reference(None, r, w) if r != 0 else "rank 0"
        q.put((r, w, l, slowest, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    # the slowest replica's time, on every rank
    assert all(o[3] == 15.0 for o in out)
    # the reference arm: rank 1 does no work and returns nothing
    assert out[1][4] is None


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_over_ranks(12.5, 1) == 12.5
