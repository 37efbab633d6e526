"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2): ranks solve
disjoint instances, the timed region is the max over ranks, throughput sums the ranks' work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    d = bench.init_dist(ws)
    seeds = bench.rank_seeds(r, 5)
    t = bench.max_over_ranks(d, 10.0 + r)          # rank 1 is the slow one
    n = bench.sum_over_ranks(d, float(len(seeds)))
    bench.barrier(d)
    out[rank] = (seeds, t, n)
    d.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    s0, t0, n0 = res[0]
    s1, t1, n1 = res[1]
    assert not set(s0) & set(s1)
    assert t0 == t1 == 11.0
    assert n0 == n1 == 10.0
