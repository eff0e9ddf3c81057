"""Failure paths driven from the host, with no GPU fault: a device allocation
made to fail by the library's test hook. Every build and search that meets
the failure returns RQ_ERR_OOM, releases what it had allocated, and the next
call works. (The bounded device waits are exercised by the test_stall hook in
test_gpu_parity.py.)"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SLACK = 64 << 20  # device bytes the driver may move between two readings


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lib()


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_in_build_return_oom_without_leaks(rq):
    x = W.mixture("tiny").base(4000)
    q = W.mixture("tiny").queries(16)
    ix = rq.rq_build(x, 32, seed=1, kmeans_iters=2)
    ref = ix.search(q, 4, 10, 50)
    ix.free()
    base = _free()
    failed = 0
    for k in range(200):
        rq.rq_test_fail_allocations(k)
        try:
            ix = rq.rq_build(x, 32, seed=1, kmeans_iters=2)
        except rq.RQError as e:
            rq.rq_test_fail_allocations(-1)
            assert e.status == rq.RQ_ERR_OOM, (k, str(e))
            assert abs(_free() - base) < SLACK, k
            failed += 1
            continue
        rq.rq_test_fail_allocations(-1)
        got = ix.search(q, 4, 10, 50)       # past the build's allocations: a good index
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        ix.free()
        break
    else:
        pytest.fail("the build never got past the injected failures")
    assert failed >= 5                        # the build makes several allocations
    assert abs(_free() - base) < SLACK


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_injected_allocation_failure_in_search_returns_oom(rq, mode):
    x = W.mixture("tiny").base(4000)
    q = W.mixture("tiny").queries(16)
    ix = rq.rq_build(x, 32, seed=2, kmeans_iters=2)
    ref = rq.rq_build(x, 32, seed=2, kmeans_iters=2).search(q, 6, 10, 60, scan_mode=mode)
    base = _free()
    rq.rq_test_fail_allocations(0)           # the new shape's workspace
    with pytest.raises(rq.RQError) as e:
        ix.search(q, 6, 10, 60, scan_mode=mode)
    rq.rq_test_fail_allocations(-1)
    assert e.value.status == rq.RQ_ERR_OOM
    assert abs(_free() - base) < SLACK
    for _ in range(2):
        got = ix.search(q, 6, 10, 60, scan_mode=mode)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert ix.device_error() == 0
