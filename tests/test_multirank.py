"""The multi-rank host logic of bench.py on the CPU: two gloo ranks (one process each, rendezvous on
127.0.0.1) meet at the barrier, agree on the slowest rank's time (the timed region is the max over ranks),
and only rank 0 runs the reference arm.  The ranks are independent replicas: nothing on the data path is
exchanged, so these host reductions are the only collectives of a multi-GPU run."""
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


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_init()
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.5 * (r + 1), w)  # rank r "took" 1.5 (r + 1) seconds

    class Args:
        workload, steps, warmup = "kh1024", 3, 3

    ran_reference = True
    if r != 0:
        bench.run_reference(Args, w, r, r)  # returns at once on ranks other than 0
        ran_reference = False
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, slowest, ran_reference))


def test_two_gloo_ranks_share_the_slowest_time():
    pytest.importorskip("torch")
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
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 and o[2] == 3.0 for o in out)
    assert out[1][3] is False


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        w, r, _ = bench.dist_init()
        assert (w, r) == (1, 0)
        bench.barrier(w)
        assert bench.max_over_ranks(2.5, w) == 2.5
    finally:
        os.environ.update(env)
