"""List-sharded search on CPU ranks (gloo, two ranks): each rank scans only
the probed lists it owns with the oracle's estimator, keeps its own n_sel
smallest (estimate, id) keys, and the ranks' keys are gathered and merged.
The merged selection, re-ranked exactly, equals the single-rank search for
every query -- the exchange step of the sharded form (Section 3.4). No GPU:
the oracle stands in for each rank's scan."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _index_and_queries():
    import workloads as W
    from oracle import rabitq as R

    mix = W.mixture("skewed")
    x = mix.base(6000)
    q = mix.queries(12)
    return x, q, R.build_index(x, 40, seed=3, iters=4)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), CUDA_VISIBLE_DEVICES="")
    import torch.distributed as dist

    from oracle import rabitq as R
    from paper_2605_16007_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, q, ix = _index_and_queries()
    owner = shard.partition_lists(np.diff(ix["offsets"]), world)
    qrot = R.rotate(q, ix["P"])
    pid, _ = R.probe(qrot, ix["cR"], 10)
    n_sel = 60
    mine = []
    for i in range(q.shape[0]):
        lists = [c for c in pid[i] if owner[c] == rank]       # probe order kept
        d2, cid, _ = R.list_candidates(ix, qrot[i], np.asarray(lists, np.int64))
        mine.append(R.select_candidates(d2, cid, n_sel, prune=True) if d2.size
                    else np.zeros(0, np.uint64))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        res = []
        for i in range(q.shape[0]):
            sel = shard.merge_selected([g[i] for g in gathered], n_sel)
            res.append(R.rerank(ix["raw"], q[i], R.key_id(sel), 10))
        out["merged"] = res
        out["owner"] = owner
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_balanced_and_deterministic():
    from paper_2605_16007_gb300 import shard

    rng = np.random.default_rng(0)
    lens = rng.zipf(1.5, 500).clip(max=5000)
    for world in (1, 2, 3, 8):
        owner = shard.partition_lists(lens, world)
        assert np.array_equal(owner, shard.partition_lists(lens, world))
        loads = np.bincount(owner, weights=lens, minlength=world)
        assert loads.max() - loads.min() <= lens.max()
    assert shard.partition_lists([5, 5, 5, 5], 2).tolist() == [0, 1, 0, 1]
    keys = [np.array([5, 9, 2**64 - 1], np.uint64), np.array([1, 7], np.uint64)]
    assert shard.merge_selected(keys, 3).tolist() == [1, 5, 7]


def test_two_gloo_ranks_sharded_search_equals_single_rank():
    from oracle import rabitq as R

    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        merged = out["merged"]
        owner = out["owner"]
    assert set(owner.tolist()) == {0, 1}
    x, q, ix = _index_and_queries()
    ids, dist = R.search(ix, q, 10, 10, 60)
    for i in range(q.shape[0]):
        assert np.array_equal(merged[i][0], ids[i])
        assert np.array_equal(merged[i][1].view(np.uint32), dist[i].view(np.uint32))
