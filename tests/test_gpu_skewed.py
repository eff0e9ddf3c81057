"""The skewed workload at full size, in every scan mode, against the oracle.

10,000,000 x 96 unit vectors from a 1024-component mixture with Zipf (s = 1)
component weights, nlist 4096: list lengths vary by more than 100x and the
longest lists hold thousands of vectors, so the plain scan cuts them into
many 1024-vector chunks and the persistent scans walk many 256-vector items
per list. One mixed batch (per-query nprobe in 8..256, k in {10, 100},
n_rerank 200) runs in all three scan modes: every dumped intermediate and
the results must agree across the modes bit for bit, and sixteen sampled
queries (including the largest nprobe and both k) are replayed stage by
stage in the CPU oracle from the GPU's own inputs to each stage.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import host_index, lib, replay_and_compare, search_dump

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def skewed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rq = lib()
    wl = W.WORKLOADS["skewed"]
    x = torch.from_numpy(wl["mix"].base(wl["n"])).cuda()
    ix = rq.rq_build(x, wl["nlist"], seed=0, kmeans_iters=4, train_size=1_000_000)
    del x
    torch.cuda.synchronize()
    return rq, ix


def _sorted_rows(a):
    return np.sort(a, axis=1)


def test_skewed_full_size_modes_agree_and_replay(skewed):
    rq, ix = skewed
    wl = W.WORKLOADS["skewed"]
    st = ix.stats()
    assert st["max_list"] > 8192 and st["max_list"] > 100 * max(1, st["min_list"])
    nq = 512
    q = wl["mix"].queries(nq)
    npb, kk = W.per_query_params(nq, 7, (8, 256), (10, 100))
    nr = np.full(nq, 200, np.int32)
    dumps = {m: search_dump(ix, q, npb, kk, nr, mixed=True, scan_mode=m) for m in (1, 2, 3)}
    base = dumps[2]
    for m in (1, 3):
        d = dumps[m]
        for key in ("qrot", "probe_ids", "probe_dist", "qparams", "planes", "bound",
                    "n_candidates", "ids", "dist"):
            assert np.array_equal(d[key].view(np.uint8), base[key].view(np.uint8)), (m, key)
        assert np.array_equal(_sorted_rows(d["selected"]), _sorted_rows(base["selected"])), m
    assert ix.device_error() == 0
    # sixteen queries replayed in the oracle: the largest nprobe, both k, and
    # a seeded sample of the rest
    rng = np.random.default_rng(9)
    rows = {int(np.argmax(npb)), int(np.argmin(npb)), int(np.flatnonzero(kk == 100)[0]),
            int(np.flatnonzero(kk == 10)[0])}
    while len(rows) < 16:
        rows.add(int(rng.integers(0, nq)))
    rows = np.array(sorted(rows))
    sub = {key: (v[rows] if isinstance(v, np.ndarray) and v.shape[:1] == (nq,) else v)
           for key, v in base.items()}
    h = host_index(ix)
    stats = replay_and_compare(h, q[rows], sub)
    assert stats["pairs"] == int(npb[rows].sum())
    # the FastScan estimator on the same batch, sampled replay
    lut = search_dump(ix, q, npb, kk, nr, mixed=True, estimator=rq.RQ_EST_LUT)
    sub = {key: (v[rows] if isinstance(v, np.ndarray) and v.shape[:1] == (nq,) else v)
           for key, v in lut.items()}
    replay_and_compare(h, q[rows], sub, estimator="lut")
    # the plain scan's chunking is exercised: probed lists longer than a chunk
    lens = np.diff(h["offsets"])
    assert lens[base["probe_ids"][rows][base["probe_ids"][rows] >= 0]].max() > 4 * 1024


def test_skewed_large_batch_split_equals_small_batches(skewed):
    """A batch whose workspace would pass the 12 GiB budget (8192 queries at
    nprobe 512 on the skewed index in the tensor-core form: survivor masks,
    key buffers and the per-list and window buckets) runs as sub-batches of
    one workspace; its results equal those of the same queries searched in
    small batches, in the tensor-core and the streaming form."""
    rq, ix = skewed
    wl = W.WORKLOADS["skewed"]
    nq = 8192
    q = wl["mix"].queries(nq)
    qd = torch.from_numpy(q).cuda()
    ref_i = torch.empty((nq, 10), dtype=torch.int64, device="cuda")
    ref_d = torch.empty((nq, 10), dtype=torch.float32, device="cuda")
    for b0 in range(0, nq, 128):
        ix.search(qd[b0:b0 + 128], 512, 10, 200, out_ids=ref_i[b0:b0 + 128],
                  out_dist=ref_d[b0:b0 + 128], scan_mode=3)
    torch.cuda.synchronize()
    for mode in (3, 2):
        oi = torch.empty((nq, 10), dtype=torch.int64, device="cuda")
        od = torch.empty((nq, 10), dtype=torch.float32, device="cuda")
        bound = torch.empty((nq,), dtype=torch.int32, device="cuda")
        ix.search(qd, 512, 10, 200, out_ids=oi, out_dist=od, scan_mode=mode,
                  dump={"bound": bound})
        torch.cuda.synchronize()
        assert torch.equal(oi, ref_i) and torch.equal(od, ref_d), mode
    assert ix.device_error() == 0


def test_skewed_unpruned_overflow_takes_streaming_finalize(skewed):
    """Without pruning every scanned vector survives: hundreds of thousands
    per query at nprobe 512, more than a query's key buffer holds, so the
    streaming finalize takes these queries. The results equal the pruned
    search's (the first bound drops no vector that could be selected), and
    the candidate count is every scanned pair."""
    rq, ix = skewed
    wl = W.WORKLOADS["skewed"]
    q = wl["mix"].queries(16)
    pruned = search_dump(ix, q, 512, 10, 200, scan_mode=3)
    h = host_index(ix)
    lens = np.diff(h["offsets"])
    for mode in (3, 1):
        full = search_dump(ix, q, 512, 10, 200, scan_mode=mode, no_prune=True)
        assert np.array_equal(full["ids"], pruned["ids"]), mode
        assert np.array_equal(full["dist"].view(np.uint32), pruned["dist"].view(np.uint32)), mode
        assert np.array_equal(np.sort(full["selected"], axis=1),
                              np.sort(pruned["selected"], axis=1)), mode
        pairs = lens[full["probe_ids"]].sum(axis=1)
        assert np.array_equal(full["n_candidates"].astype(np.int64), pairs), mode
        assert pairs.min() > 65536
    assert ix.device_error() == 0
