"""Multi-rank replica logic on CPU: two gloo ranks (127.0.0.1) exchange only the timing
frame; instance sets are disjoint."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2402_05598_gb300 import replicas as R
    seeds = list(R.rank_seeds(rank, 4))
    dist.barrier()
    t, s = R.reduce_timing(100.0 + 50.0 * rank, 3 + rank)
    out.put((rank, seeds, t, s))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_timing_frame():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, n0), (r1, s1, t1, n1) = res
    assert set(s0).isdisjoint(s1) and len(s0) == len(s1) == 4
    assert t0 == t1 == 150.0          # slowest rank's time
    assert n0 == n1 == 7              # all ranks' solves


def test_single_process_is_identity():
    from paper_2402_05598_gb300 import replicas as R
    assert R.reduce_timing(12.5, 3) == (12.5, 3)
    assert list(R.rank_seeds(1, 3)) == [10003, 10004, 10005]
