"""rq_probe_static: the allocation-free rotation + centroid ranking.

It exists for callers that cannot allocate device memory while they search
(under a framework that owns all device memory, or on a latency-critical
thread that cannot take cudaMalloc's device synchronisation). Its scratch is a fixed
device array shared by all calls, so the test checks it twice in a row --
the second call sees the first call's leftovers -- against the probe stage
of the existing rq_search entry point, bit for bit (the tolerance the other
parity tests use for this stage), and that oversized calls are refused.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import lib, search_dump

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rq = lib()
    mix = W.mixture("tiny")
    x = mix.base(6000)
    q = mix.queries(150)
    ix = rq.rq_build(x, 48, seed=9, kmeans_iters=4)
    return rq, ix, q


@pytest.mark.parametrize("calls", [[(150, 8), (37, 20)], [(64, 48), (150, 8)]])
def test_probe_static_matches_search_probe_twice(setup, calls):
    rq, ix, q = setup
    for nq, nprobe in calls:
        qs = q[:nq]
        ref = search_dump(ix, qs, nprobe, 10, 100)
        qd = torch.from_numpy(np.ascontiguousarray(qs)).cuda()
        ids = torch.full((nq, nprobe), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((nq, nprobe), -7.0, dtype=torch.float32, device="cuda")
        ix.probe_static(qd, nprobe, ids, dist)
        torch.cuda.synchronize()
        assert np.array_equal(ids.cpu().numpy(), ref["probe_ids"])
        assert np.array_equal(dist.cpu().numpy().view(np.uint32),
                              ref["probe_dist"].view(np.uint32))


def test_probe_static_refuses_oversized_and_host_buffers(setup):
    rq, ix, q = setup
    # 48 lists, D_p = 128: each query needs 512 + 384 bytes of the 16 MiB
    big = 20000
    qd = torch.zeros((big, 128), dtype=torch.float32, device="cuda")
    ids = torch.empty((big, 4), dtype=torch.int32, device="cuda")
    dist = torch.empty((big, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rq.RQError) as e:
        ix.probe_static(qd, 4, ids, dist)
    assert e.value.status == rq.RQ_ERR_INVALID_ARG and "scratch" in str(e.value)
    with pytest.raises(ValueError):
        ix.probe_static(q[:4], 4, np.empty((4, 4), np.int32), np.empty((4, 4), np.float32))
    # the C entry point itself refuses host pointers
    import ctypes as C
    qh = np.ascontiguousarray(q[:4])
    oi, od = np.empty((4, 4), np.int32), np.empty((4, 4), np.float32)
    st = rq.lib().rq_probe_static(ix.h, rq._ptr(qh), 4, 4, rq._ptr(oi), rq._ptr(od), None)
    assert st == rq.RQ_ERR_INVALID_ARG


def test_probe_static_wrapper_checks_shapes_and_dtypes(setup):
    """The C entry point sees bare pointers; the binding refuses buffers whose
    shape, dtype or residence would make the kernels read or write out of
    bounds, before anything is launched."""
    rq, ix, q = setup
    dev = "cuda"
    qd = torch.from_numpy(np.ascontiguousarray(q[:8])).to(dev)
    good_i = torch.empty((8, 4), dtype=torch.int32, device=dev)
    good_d = torch.empty((8, 4), dtype=torch.float32, device=dev)
    bad = [
        (qd[:, :64].contiguous(), good_i, good_d),                       # width != dim
        (qd.double(), good_i, good_d),                                   # float64 queries
        (qd, torch.empty((8, 3), dtype=torch.int32, device=dev), good_d),  # too few columns
        (qd, torch.empty((8, 4), dtype=torch.int64, device=dev), good_d),  # int64 ids
        (qd, good_i, torch.empty((8, 4), dtype=torch.float64, device=dev)),
        (qd, good_i, torch.empty((7, 4), dtype=torch.float32, device=dev)),
        (qd.t().contiguous().t(), good_i, good_d),                       # not contiguous
        (qd.cpu(), good_i, good_d),                                      # host queries
    ]
    for a, b, c in bad:
        with pytest.raises(ValueError):
            ix.probe_static(a, 4, b, c)
    ix.probe_static(qd, 4, good_i, good_d)
    torch.cuda.synchronize()
