"""The benchmark's recall is measured against a GPU exact-kNN ground truth
(the full workloads are too large for the CPU oracle inside a timed run).
Here that ground truth and the benchmark's recall function are pinned to the
oracle's brute-force exact kNN and tie-aware recall on sampled data of each
recipe the benchmark uses."""
import numpy as np
import pytest

import bench
import workloads as W
from oracle import rabitq as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["skewed", "sift1m", "highdim"])
def test_bench_ground_truth_is_oracle_exact_knn(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mix = W.mixture(name)
    n = 60_000 if name != "highdim" else 20_000
    x = mix.base(n)
    q = mix.queries(48)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()
    integer = mix.kind == "uint8"
    kth = bench.exact_kth(xd, qd, 10, integer).cpu().numpy()
    ti, td = R.exact_knn(x, q, 10)
    assert np.allclose(kth, td[:, 9], rtol=1e-12, atol=0)
    if integer:
        assert np.array_equal(kth, td[:, 9])
    # recall of a few result sets: the oracle's own answer, one shifted by a
    # rank, one with padded ids
    for ids in (ti, np.roll(ti, 1, axis=1), np.where(np.arange(10) < 7, ti, -1)):
        got = bench.recall_of(xd, qd, ids, torch.from_numpy(td[:, 9]).cuda(), 10)
        assert got == pytest.approx(R.recall_at(x, q, ids, td, 10), abs=1e-12)
