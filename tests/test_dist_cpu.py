"""The bench's multi-rank bookkeeping, on CPU with two gloo ranks: every
rank sees the maximum of the ranks' step times and the sum of their
queries, and the ranks serve disjoint query batches (weak scaling). No GPU:
the ranks hide CUDA before touching it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    import bench

    r, w, local, pg = bench.dist_setup(world)
    t = bench.max_over_ranks(pg, 1.0 + rank)
    s = bench.sum_over_ranks(pg, 1000.0 * (rank + 1))
    bench.barrier(pg)
    out[rank] = (r, w, local, t, s, bench.rank_batches(10, r, w))
    pg.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_split_batches():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, local, t, s, order) in res.items():
        assert (r, w, local) == (rank, world, rank)
        assert t == 2.0            # max of 1.0 and 2.0 on every rank
        assert s == 3000.0         # 1000 + 2000
    first = [set(res[r][5][:5]) for r in range(world)]
    assert first[0].isdisjoint(first[1])
    assert first[0] | first[1] == set(range(10))
