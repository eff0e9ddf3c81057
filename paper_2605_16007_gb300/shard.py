"""List-sharded search across ranks: the host side (Section 3.4).

The paper partitions the inverted lists across devices so that each holds a
balanced share of the vectors. Every device runs the same query batch: it
ranks the global centroids, scans only the probed lists it holds, and
returns its candidates as (estimate, id) keys. The host gathers the keys,
keeps the n_rerank smallest of their union, and re-ranks them exactly.

Keys carry global row ids and rank by (estimate, id), so the merge does not
depend on which rank found a key or in which order the keys arrive. The
n_sel smallest keys of the union equal the n_sel smallest of the
concatenation of every rank's own n_sel smallest. The merged selection is
therefore the single-device selection.

This module holds the partition and the merge (host code, numpy). Every run
here has one GPU, so no multi-GPU data path is built. The merge is tested
with CPU ranks over gloo.
"""
from __future__ import annotations

import numpy as np

U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)


def partition_lists(list_lengths, n_ranks: int) -> np.ndarray:
    """Owner rank of each list. Lists are placed longest first on the rank
    with the fewest vectors so far (ties to the lower rank). This keeps every
    rank's share within one list length of the mean. Deterministic."""
    lens = np.asarray(list_lengths, np.int64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be at least 1")
    owner = np.empty(lens.size, np.int64)
    load = np.zeros(n_ranks, np.int64)
    for l in np.lexsort((np.arange(lens.size), -lens)):     # longest first, ties by id
        r = int(np.argmin(load))
        owner[l] = r
        load[r] += lens[l]
    return owner


def merge_selected(per_rank_keys, n_sel: int) -> np.ndarray:
    """The n_sel smallest (estimate, id) keys of the union of the ranks'
    selections, ascending. Padding keys (all ones) are dropped."""
    keys = [np.asarray(k, np.uint64).ravel() for k in per_rank_keys]
    allk = np.concatenate(keys) if keys else np.zeros(0, np.uint64)
    allk = allk[allk != U64_MAX]
    return np.sort(allk)[:n_sel]
