"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (codes, probe ids, bit-planes, Sq, candidate keys, final ids)
must match bit for bit; the float32 stages follow one fixed arithmetic on
both sides, so their results must match bit for bit as well (a stricter bar
than the 1e-5 relative tolerance). Stages that the GPU computes in another
precision than the oracle (the float32 rotation against the float64 one, the
float32 encode against float64) are compared within stated tolerances, and
every later stage is replayed from the GPU's own output of that stage.
"""
import os
import tempfile

import numpy as np
import pytest

import workloads as W
from oracle import philox, rabitq as R
from tests.gpu_helpers import host_index, lib, replay_and_compare, search_dump

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib()


@pytest.fixture(scope="module")
def tiny(rq):
    wl = W.WORKLOADS["tiny"]
    x = wl["mix"].base(wl["n"])
    q = wl["mix"].queries(wl["nq"])
    ix = rq.rq_build(x, wl["nlist"], seed=0, kmeans_iters=wl["iters"])
    return x, q, ix, host_index(ix)


# ---------------------------------------------------------------- build
def test_philox_gaussian_matches_oracle(rq):
    n = 100_001
    g = rq.rq_philox_gaussian(1234, philox.STREAM_ROTATION, n)
    o = philox.gaussian(1234, philox.STREAM_ROTATION, n)
    # identical uniforms; log/cos/sin of two math libraries differ by ulps
    assert np.allclose(g, o, rtol=1e-13, atol=1e-15)


def test_rotation_matches_oracle(tiny):
    _, _, _, h = tiny
    P = h["P"]
    assert np.abs(P.T @ P - np.eye(P.shape[0])).max() <= 1e-12
    Po = R.random_orthogonal(0, P.shape[0])
    assert np.abs(P - Po).max() <= 1e-10


@pytest.mark.parametrize("n,nlist,iters,train", [(3000, 32, 5, 0), (5000, 40, 4, 1500)])
def test_kmeans_bit_exact(rq, n, nlist, iters, train):
    x = W.mixture("tiny").base(n)
    c_gpu = rq.rq_kmeans(x, nlist, seed=7, iters=iters, train_size=train)
    c_cpu = R.kmeans(x, nlist, iters, seed=7, n_train=train)
    assert np.array_equal(c_gpu.view(np.uint32), c_cpu.view(np.uint32))


def test_kmeans_empty_cluster_reseed(rq):
    # Half the rows are one repeated vector: several initial centroids
    # coincide, ties go to the lowest id, and the others start empty.
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1200, 32)).astype(np.float32)
    x[::2] = x[0]
    c_gpu = rq.rq_kmeans(x, 24, seed=1, iters=3)
    c_cpu = R.kmeans(x, 24, 3, seed=1)
    a, _ = R.assign(x, R.kmeans(x, 24, 0, seed=1))
    assert np.bincount(a, minlength=24).min() == 0   # the reseed path is taken
    assert np.array_equal(c_gpu.view(np.uint32), c_cpu.view(np.uint32))


def test_layout_and_encode_match_oracle(tiny):
    x, _, _, h = tiny
    # assignment / list layout: bit-exact given the GPU centroids
    a, _ = R.assign(x, h["centroids"])
    assert np.array_equal(h["assign"], a)
    order = np.lexsort((np.arange(x.shape[0]), a))
    assert np.array_equal(h["ids"], order)
    assert np.array_equal(h["offsets"], np.concatenate([[0], np.cumsum(np.bincount(a, minlength=h["nlist"]))]))
    # encode in float64 from the GPU's P and centroids
    codes, r, alpha, z = R.encode(x[order], h["centroids"], a[order], h["P"])
    zr = np.abs(z) / np.maximum(r, 1e-30)[:, None]
    near = zr < 1e-5          # sign decided below float32 rotation error
    bits_g = R.unpack_bits(h["codes"], h["dp"]).astype(bool)
    bits_o = R.unpack_bits(codes, h["dp"]).astype(bool)
    assert np.array_equal(bits_g[~near], bits_o[~near])
    assert (bits_g != bits_o).sum() <= near.sum()
    assert np.allclose(h["r"], r, rtol=1e-6, atol=0)
    assert np.allclose(h["alpha"], alpha, rtol=2e-5, atol=0)
    r2, f = R.scan_factors(h["r"], h["alpha"], h["dp"])
    assert np.array_equal(h["r2"].view(np.uint32), r2.view(np.uint32))
    assert np.array_equal(h["f"].view(np.uint32), f.view(np.uint32))
    cR = (R.pad(h["centroids"].astype(np.float64), h["dp"]) @ h["P"])
    assert np.allclose(h["cR"], cR, rtol=1e-6, atol=1e-6 * np.abs(cR).max())


def test_build_with_given_centroids_and_rotation(rq):
    x = W.mixture("tiny").base(2000)
    P = R.random_orthogonal(5, 128)
    c = R.kmeans(x, 16, 3, seed=5)
    ix = rq.rq_build_with(x, c, P)
    h = host_index(ix)
    assert np.array_equal(h["P"], P)
    assert np.array_equal(h["centroids"], c)
    o = R.build_index(x, 16, seed=5, centroids=c, P=P)
    assert np.array_equal(h["ids"], o["ids"])
    assert np.array_equal(h["offsets"], o["offsets"])


# ---------------------------------------------------------------- search
@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("prune", [True, False])
def test_search_stages_replay_bit_exact(tiny, mode, prune):
    _, q, ix, h = tiny
    dump = search_dump(ix, q, 8, 10, 100, scan_mode=mode, no_prune=not prune)
    st = replay_and_compare(h, q, dump, prune=prune)
    assert st["pairs"] == q.shape[0] * 8
    # the float32 rotation against the float64 one
    qr = R.rotate(q, h["P"])
    assert np.abs(dump["qrot"] - qr).max() <= 1e-5 * np.abs(qr).max()


def test_probe_ties_between_duplicate_centroids(rq):
    """Centroids repeated exactly: equal centroid distances, so the probe
    order rests on the list id, through the approximate filter and the exact
    selection of the nearest lists."""
    x = W.mixture("tiny").base(3000)
    c = R.kmeans(x, 24, 3, seed=7)
    c = np.concatenate([c, c[:8], c[:8]]).astype(np.float32)   # 40 lists, 16 duplicates
    P = R.random_orthogonal(11, 128)
    ix = rq.rq_build_with(x, c, P)
    h = host_index(ix)
    q = W.mixture("tiny").queries(32)
    q[:4] = c[:4]                                              # queries on a centroid
    for mode in (1, 3):
        dump = search_dump(ix, q, 12, 10, 60, scan_mode=mode)
        replay_and_compare(h, q, dump)


def test_probe_exact_ranking_path_for_large_nlist(rq):
    """nlist above 4096: the probe selection ranks all centroids exactly
    instead of filtering an approximate ranking; replayed bit for bit."""
    mix = W.mixture("tiny")
    x = mix.base(30000)
    q = mix.queries(12)
    ix = rq.rq_build(x, 4500, seed=1, kmeans_iters=2)
    h = host_index(ix)
    for mode in (1, 3):
        dump = search_dump(ix, q, 8, 10, 50, scan_mode=mode)
        replay_and_compare(h, q, dump)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_many_candidates_replay_bit_exact(tiny, mode):
    """No pruning and half of the lists probed: more candidates per query
    than the finalize stages in shared memory at once (2048)."""
    _, q, ix, h = tiny
    dump = search_dump(ix, q[:24], 32, 10, 100, scan_mode=mode, no_prune=True)
    assert dump["n_candidates"].min() > 2048
    replay_and_compare(h, q[:24], dump, prune=False)


def test_recall_target(tiny):
    x, q, ix, _ = tiny
    _, td = R.exact_knn(x, q, 10)
    ids, _ = ix.search(q, 8, 10, 100)
    assert R.recall_at(x, q, ids, td, 10) >= 0.95


def test_modes_graph_and_streams_identical(tiny):
    _, q, ix, _ = tiny
    ref = ix.search(q, 16, 10, 200, scan_mode=1)
    for kw in (dict(scan_mode=2), dict(scan_mode=2, use_graph=True),
               dict(scan_mode=1, use_graph=True), dict(scan_mode=0),
               dict(scan_mode=3), dict(scan_mode=3, use_graph=True)):
        for _ in range(2):
            got = ix.search(q, 16, 10, 200, **kw)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), kw
    s = torch.cuda.Stream()
    qd = torch.from_numpy(q).cuda()
    oi = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ix.search(qd, 16, 10, 200, out_ids=oi, out_dist=od, use_graph=True, stream=s)
    s.synchronize()
    assert np.array_equal(oi.cpu().numpy(), ref[0])


def test_mixed_batch_equals_alone_and_replays(tiny):
    _, q, ix, h = tiny
    nq = 40
    npb, kk = W.per_query_params(nq, 5, (1, 64), (1, 10, 33))
    nr = np.where(np.arange(nq) % 5 == 0, 0, np.maximum(kk, 50)).astype(np.int32)
    for mode in (1, 2, 3):
        dump = search_dump(ix, q[:nq], npb, kk, nr, mixed=True, scan_mode=mode)
        replay_and_compare(h, q[:nq], dump)
    for i in range(0, nq, 7):
        alone = ix.search(q[i:i + 1], int(npb[i]), int(kk[i]), int(nr[i]))
        assert np.array_equal(alone[0][0], dump["ids"][i, :kk[i]])
        assert np.array_equal(alone[1][0], dump["dist"][i, :kk[i]])


def test_short_results_are_padded(rq):
    x = W.mixture("tiny").base(300)
    q = W.mixture("tiny").queries(5)
    ix = rq.rq_build(x, 30, seed=2, kmeans_iters=3)
    h = host_index(ix)
    # one probed list holds ~10 vectors, far fewer than k
    for mode in (1, 2, 3):
        dump = search_dump(ix, q, 1, 50, 60, scan_mode=mode)
        replay_and_compare(h, q, dump)
    assert (dump["ids"] == -1).any() and np.isinf(dump["dist"]).any()
    # n_rerank = 0 returns the estimated top k
    dump = search_dump(ix, q, 3, 7, 0, scan_mode=1)
    replay_and_compare(h, q, dump)


@pytest.mark.parametrize("dim", [96, 200, 960])
def test_padded_dimensions_replay(rq, dim):
    mix = W.mixture("highdim", dim=dim) if dim == 960 else W.mixture("tiny", dim=dim)
    x = mix.base(3000)
    q = mix.queries(12)
    ix = rq.rq_build(x, 24, seed=3, kmeans_iters=3)
    h = host_index(ix)
    assert h["dp"] == R.dim_pad(dim)
    for mode in (1, 2):
        dump = search_dump(ix, q, 6, 10, 80, scan_mode=mode)
        replay_and_compare(h, q, dump)


def test_uint8_base_and_sift_like_data(rq):
    mix = W.mixture("sift1m")
    x = mix.base(20000)
    q = mix.queries(20)
    x8 = x.astype(np.uint8)
    ix = rq.rq_build(x8, 64, seed=4, kmeans_iters=4)
    h = host_index(ix)
    assert h["raw"].dtype == np.float32 and np.array_equal(h["raw"], x)
    for mode in (2, 3):
        dump = search_dump(ix, q, 12, 10, 200, scan_mode=mode)
        replay_and_compare(h, q, dump)
    _, td = R.exact_knn(x, q, 10)
    assert R.recall_at(x, q, dump["ids"], td, 10) >= 0.9


def test_full_size_sift_batch_sampled_replay(rq):
    """The bench's workload at full size (1,000,000 x 128, nlist 1024, a batch
    of 1000 queries, nprobe 16, k 10, n_rerank 200) in the bench's launch
    form (tensor-core scan from a captured graph): identical to the
    uncaptured search with every intermediate dumped, and eight sampled
    queries replayed stage by stage in the oracle, bit for bit."""
    wl = W.WORKLOADS["sift1m"]
    x = torch.from_numpy(wl["mix"].base(wl["n"])).cuda()
    q = wl["mix"].queries(wl["batch"])
    ix = rq.rq_build(x, wl["nlist"], seed=0, kmeans_iters=wl["iters"])
    del x
    qd = torch.from_numpy(q).cuda()
    ids = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    dist = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    for _ in range(2):
        ix.search(qd, 16, 10, 200, out_ids=ids, out_dist=dist, scan_mode=3, use_graph=True)
    torch.cuda.synchronize()
    dump = search_dump(ix, q, 16, 10, 200, scan_mode=3)
    assert np.array_equal(ids.cpu().numpy(), dump["ids"])
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), dump["dist"].view(np.uint32))
    rows = np.random.default_rng(5).choice(q.shape[0], 8, replace=False)
    sub = {kk: (v[rows] if isinstance(v, np.ndarray) and v.shape[:1] == (q.shape[0],) else v)
           for kk, v in dump.items()}
    st = replay_and_compare(host_index(ix), q[rows], sub)
    assert st["pairs"] == 8 * 16


def test_export_import_roundtrip(tiny, tmp_path):
    _, q, ix, _ = tiny
    path = str(tmp_path / "ix.rq")
    ix.export(path)
    rq = lib()
    ix2 = rq.rq_import(path)
    a = ix.search(q, 8, 10, 100)
    b = ix2.search(q, 8, 10, 100)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert ix2.stats() == ix.stats()


def test_server_results_equal_alone(tiny):
    _, q, ix, _ = tiny
    rq = lib()
    srv = rq.Server(ix, slots=3, max_batch=64)
    reqs = []
    rng = np.random.default_rng(11)
    for i in range(30):
        n = int(rng.integers(1, 9))
        lo = int(rng.integers(0, q.shape[0] - n))
        npb = int(rng.integers(1, 40))
        k = int(rng.integers(1, 20))
        nr = int(rng.integers(k, 150)) if i % 4 else 0
        reqs.append((srv.submit(q[lo:lo + n], npb, k, nr), lo, n, npb, k, nr))
    for t, lo, n, npb, k, nr in reqs:
        ids, dist, lat = srv.wait(t, timeout_ms=60000)
        a_ids, a_d = ix.search(q[lo:lo + n], npb, k, nr)
        assert np.array_equal(ids, a_ids) and np.array_equal(dist, a_d)
        assert lat > 0
    srv.close()


def test_invalid_arguments_rejected(tiny):
    _, q, ix, _ = tiny
    rq = lib()
    for args in [(0, 10, 100), (65, 10, 100), (8, 0, 100), (8, 10, 5), (8, 10, 5000)]:
        with pytest.raises(rq.RQError) as e:
            ix.search(q, *args)
        assert e.value.status == rq.RQ_ERR_INVALID_ARG
    for v in (np.nan, np.inf, -np.inf):
        bad = q.copy()
        bad[3, 5] = v
        with pytest.raises(rq.RQError) as e:
            ix.search(bad, 8, 10, 100)
        assert e.value.status == rq.RQ_ERR_INVALID_ARG
    assert ix.device_error() == 0


def test_integer_valued_base_kept_as_bytes_is_lossless(rq):
    mix = W.mixture("sift1m")
    x = mix.base(20000)
    q = mix.queries(30)
    a = rq.rq_build(x, 64, seed=4, kmeans_iters=3)
    b = rq.rq_build(x, 64, seed=4, kmeans_iters=3, keep_float_raw=True)
    assert a.stats()["raw_bytes"] == x.size and b.stats()["raw_bytes"] == 4 * x.size
    for mode in (1, 2, 3):
        ra = a.search(q, 12, 10, 200, scan_mode=mode)
        rb = b.search(q, 12, 10, 200, scan_mode=mode)
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    # a base that is not integer-valued keeps its float copy
    t = rq.rq_build(W.mixture("tiny").base(3000), 16, seed=0, kmeans_iters=2)
    assert t.stats()["raw_bytes"] == 3000 * 128 * 4


# ---------------------------------------------------------------- failure paths
@pytest.mark.parametrize("mode", [2, 3])
def test_scan_wait_runs_out_and_is_reported(tiny, mode):
    """The pipelined scans bound every mbarrier wait. The test hook makes the
    producer hold back its first stage (nothing ever signals it), so the
    consumers' wait (1 ms under the hook) runs out: the kernel flags the
    error word and returns, a synchronous search reports RQ_ERR_TIMEOUT and
    clears the word, an asynchronous one leaves the code for
    rq_device_error, and the context stays usable."""
    _, q, ix, _ = tiny
    rq = lib()
    ref = ix.search(q, 8, 10, 100, scan_mode=mode)
    with pytest.raises(rq.RQError) as e:
        ix.search(q, 8, 10, 100, scan_mode=mode, test_stall=True)
    assert e.value.status == rq.RQ_ERR_TIMEOUT
    assert ix.device_error() == 0            # the synchronous call cleared it
    qd = torch.from_numpy(q).cuda()
    oi = torch.empty((q.shape[0], 10), dtype=torch.int64, device="cuda")
    od = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    ix.search(qd, 8, 10, 100, out_ids=oi, out_dist=od, scan_mode=mode, test_stall=True)
    torch.cuda.synchronize()
    assert ix.device_error() == (4 if mode == 3 else 5)
    assert ix.device_error() == 0            # read and cleared
    for _ in range(2):                       # the context and the index still work
        got = ix.search(q, 8, 10, 100, scan_mode=mode)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_plain_chunks_and_tuned_choices_are_identical(rq, tmp_path):
    """Every form the autotuner can pick (the plain scan at 1024, 2048 and
    4096 vectors per block, the streaming and tensor-core scans) returns the
    same results, bit for bit, on lists longer than a chunk; the tuned choice
    is stored per batch class in the cache file and read back from it."""
    mix = W.mixture("tiny")
    x = mix.base(30000)
    q = mix.queries(40)
    ix = rq.rq_build(x, 8, seed=5, kmeans_iters=3)
    assert ix.stats()["max_list"] > 4096
    ref = ix.search(q, 3, 10, 200, scan_mode=1)
    for kw in (dict(scan_mode=1, plain_chunk=2048), dict(scan_mode=1, plain_chunk=4096),
               dict(scan_mode=1, plain_chunk=4096, use_graph=True), dict(scan_mode=2),
               dict(scan_mode=3)):
        got = ix.search(q, 3, 10, 200, **kw)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), kw
    with pytest.raises(rq.RQError):
        ix.search(q, 3, 10, 200, scan_mode=1, plain_chunk=1500)
    cache = str(tmp_path / "tune.txt")
    ix.autotune(q, 3, 200, cache_path=cache)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and "nq_class=" in lines[0] and " mode=" in lines[0]
    got = ix.search(q, 3, 10, 200)                       # AUTO: the tuned choice
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    ix2 = rq.rq_build(x, 8, seed=5, kmeans_iters=3)
    ix2.autotune(q, 3, 200, cache_path=cache)            # read from the cache file
    assert len(open(cache).read().splitlines()) == 1
    got = ix2.search(q, 3, 10, 200)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


# ---------------------------------------------------------------- FastScan estimator
@pytest.mark.parametrize("prune", [True, False])
def test_fastscan_estimator_replays_bit_exact(tiny, prune):
    """The paper's FastScan form (full-precision residual, float32 tables per
    8 dimensions): per-pair sums, bound, survivors, selection and results
    replayed in the oracle from the GPU's rotated queries, bit for bit."""
    _, q, ix, h = tiny
    rq = lib()
    dump = search_dump(ix, q, 8, 10, 100, estimator=rq.RQ_EST_LUT, no_prune=not prune)
    st = replay_and_compare(h, q, dump, prune=prune, estimator="lut")
    assert st["pairs"] == q.shape[0] * 8
    # the two estimators differ (the 4-bit query is an approximation of it)
    d4 = search_dump(ix, q, 8, 10, 100)
    assert not np.array_equal(d4["selected"], dump["selected"])


def test_fastscan_estimator_mixed_padded_and_unranked(rq):
    """FastScan with mixed per-query nprobe / k / n_rerank (including top-k
    by the estimate), at D_p 256, and refused above 256."""
    mix = W.mixture("tiny", dim=200)
    x = mix.base(4000)
    q = mix.queries(30)
    ix = rq.rq_build(x, 24, seed=6, kmeans_iters=3)
    h = host_index(ix)
    npb, kk = W.per_query_params(30, 8, (1, 24), (1, 10, 20))
    nr = np.where(np.arange(30) % 4 == 0, 0, np.maximum(kk, 60)).astype(np.int32)
    dump = search_dump(ix, q, npb, kk, nr, mixed=True, estimator=rq.RQ_EST_LUT)
    replay_and_compare(h, q, dump, estimator="lut")
    hd = W.mixture("highdim")
    ixh = rq.rq_build(hd.base(2000), 8, seed=1, kmeans_iters=2)
    with pytest.raises(rq.RQError) as e:
        ixh.search(hd.queries(2), 2, 10, 50, estimator=rq.RQ_EST_LUT)
    assert e.value.status == rq.RQ_ERR_NOT_IMPLEMENTED


def test_exact_probe_path_wide_codes_many_lists(rq):
    """D_p above 128 takes the exact centroid ranking, whose selection stages
    all nlist keys in shared memory: 800 lists (6.4 KB of keys) at D_p 256,
    replayed bit for bit in every mode that D_p supports."""
    mix = W.mixture("tiny", dim=200)
    x = mix.base(20000)
    q = mix.queries(10)
    ix = rq.rq_build(x, 800, seed=9, kmeans_iters=2)
    h = host_index(ix)
    for mode in (1, 2):
        dump = search_dump(ix, q, 12, 10, 100, scan_mode=mode)
        replay_and_compare(h, q, dump)


@pytest.mark.parametrize("u8", [False, True])
def test_raw_on_host_rerank_equals_device_copy(u8):
    """With raw_on_host the re-rank reads the caller's page-locked base rows
    in host memory: every result equals the device-copy index's, the index
    exports and imports like any other, and a pageable base is refused."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rq = lib()
    mix = W.mixture("sift1m" if u8 else "tiny")
    x = mix.base(20000)
    if u8:
        x = x.astype(np.uint8)
    q = mix.queries(64).astype(np.float32)
    ref = rq.rq_build(x, 64, seed=3, kmeans_iters=3, keep_float_raw=True)
    pinned = torch.from_numpy(x).pin_memory()
    ix = rq.rq_build(pinned, 64, seed=3, kmeans_iters=3, raw_on_host=True)
    for mode in (1, 3):
        a = ref.search(q, 12, 10, 120, scan_mode=mode)
        b = ix.search(q, 12, 10, 120, scan_mode=mode)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    path = os.path.join(tempfile.mkdtemp(), "host_raw.rqix")
    ix.export(path)
    ix2 = rq.rq_import(path)
    c = ix2.search(q, 12, 10, 120)
    assert np.array_equal(c[0], ref.search(q, 12, 10, 120)[0])
    ix.free()
    assert pinned.numpy().tobytes() == x.tobytes()  # the caller's buffer, untouched
    with pytest.raises(rq.RQError) as e:
        rq.rq_build(x, 64, seed=3, kmeans_iters=3, raw_on_host=True)
    assert e.value.status == rq.RQ_ERR_INVALID_ARG
