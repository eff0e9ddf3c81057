"""Seeded synthetic workloads shaped like the paper's datasets (Section 4.1).

This module produces INPUT data only: base vectors and queries drawn from
Gaussian mixtures. It holds none of the search method's arithmetic, so both
the CPU oracle (``oracle/``) and the CUDA path may consume its output.

Every array is generated in row chunks from ``numpy.random.default_rng``
seeded with the tuple ``(seed, stream, chunk)``: any chunk can be
regenerated on its own, so a test can rebuild a sample of a large workload
without generating all of it. Queries come from the same mixture as the base
vectors, with a different seed (``seed + 1``), as the paper draws its query
sets from the same distribution as its corpora.

Workload recipes (the paper's public datasets are not available, so each
recipe stands in for one of them):

* ``tiny``      10,000 x 128 FP32; 64-component isotropic mixture, component
                means ~ N(0, 1), std 0.3.
* ``sift1m``    1,000,000 x 128 integer-valued FP32 in [0, 255]; 256
                components, means |N(0, 40^2)| per dim, std 15, rounded and
                clamped (shaped like SIFT descriptors).
* ``highdim``   1,000,000 x 960 FP32; 512 components, means N(0, 1), per-dim
                std sqrt(U(0.5, 2)) drawn once per dimension.
* ``skewed``    10,000,000 x 96 FP32 unit vectors; 1024 components with Zipf
                (s = 1) weights, means uniform on the sphere, std 0.05 per dim
                before normalisation; IVF list lengths then vary by > 100x.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# Streams of the seed tuple: which random draw a chunk belongs to.
_S_MEANS, _S_SCALE, _S_WEIGHTS, _S_LABELS, _S_NOISE = 0, 1, 2, 3, 4

CHUNK_ROWS = 1 << 16


@dataclasses.dataclass(frozen=True)
class Mixture:
    """A Gaussian mixture: ``n_comp`` means in ``dim`` dims, noise scale."""

    name: str
    dim: int
    n_comp: int
    seed: int
    kind: str  # "gauss", "uint8", "sphere"
    mean_scale: float
    noise_std: float
    zipf: bool = False
    per_dim_var: bool = False

    # -- component parameters (small; generated whole) ---------------------
    def means(self) -> np.ndarray:
        rng = np.random.default_rng([self.seed, _S_MEANS])
        m = rng.standard_normal((self.n_comp, self.dim))
        if self.kind == "uint8":
            m = np.abs(m) * self.mean_scale
        elif self.kind == "sphere":
            m /= np.linalg.norm(m, axis=1, keepdims=True)
        else:
            m *= self.mean_scale
        return m

    def dim_std(self) -> np.ndarray:
        if not self.per_dim_var:
            return np.full(self.dim, self.noise_std)
        rng = np.random.default_rng([self.seed, _S_SCALE])
        return np.sqrt(rng.uniform(0.5, 2.0, self.dim))

    def weights(self) -> np.ndarray:
        if not self.zipf:
            return np.full(self.n_comp, 1.0 / self.n_comp)
        # Zipf with s = 1: weight of the component of rank j is 1/j. The rank
        # order is shuffled so that component id does not encode size.
        rng = np.random.default_rng([self.seed, _S_WEIGHTS])
        w = 1.0 / np.arange(1, self.n_comp + 1)
        w = w[rng.permutation(self.n_comp)]
        return w / w.sum()

    # -- rows ---------------------------------------------------------------
    def chunk(self, stream_seed: int, c: int, rows: int, means, std, cdf):
        rng_l = np.random.default_rng([stream_seed, _S_LABELS, c])
        rng_n = np.random.default_rng([stream_seed, _S_NOISE, c])
        if self.zipf:
            lab = np.searchsorted(cdf, rng_l.random(rows), side="right")
            lab = np.minimum(lab, self.n_comp - 1)
        else:
            lab = rng_l.integers(0, self.n_comp, rows)
        x = means[lab] + rng_n.standard_normal((rows, self.dim)) * std
        if self.kind == "uint8":
            x = np.clip(np.rint(x), 0, 255)
        elif self.kind == "sphere":
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32), lab.astype(np.int32)

    def rows(self, n: int, stream_seed: int, start_chunk: int = 0,
             labels: bool = False):
        """n rows, chunk by chunk; chunks are independent, so they are drawn
        by a thread pool (the result does not depend on the thread count)."""
        means, std = self.means(), self.dim_std()
        cdf = np.cumsum(self.weights())
        out = np.empty((n, self.dim), np.float32)
        lab = np.empty(n, np.int32)

        def fill(job):
            i, r0 = job
            r = min(CHUNK_ROWS, n - r0)
            out[r0:r0 + r], lab[r0:r0 + r] = self.chunk(
                stream_seed, start_chunk + i, r, means, std, cdf)

        jobs = list(enumerate(range(0, n, CHUNK_ROWS)))
        if len(jobs) <= 1:
            for j in jobs:
                fill(j)
        else:
            workers = max(1, min(16, os.cpu_count() or 1, len(jobs)))
            with ThreadPoolExecutor(workers) as ex:
                list(ex.map(fill, jobs))
        return (out, lab) if labels else out

    def base(self, n: int, labels: bool = False):
        return self.rows(n, self.seed, labels=labels)

    def queries(self, n: int, labels: bool = False):
        return self.rows(n, self.seed + 1, labels=labels)


TINY = Mixture("tiny", 128, 64, 0, "gauss", 1.0, 0.3)
SIFT1M = Mixture("sift1m", 128, 256, 0, "uint8", 40.0, 15.0)
HIGHDIM = Mixture("highdim", 960, 512, 0, "gauss", 1.0, 1.0, per_dim_var=True)
SKEWED = Mixture("skewed", 96, 1024, 0, "sphere", 1.0, 0.05, zipf=True)

# Full workload sizes and search parameters of each recipe.
WORKLOADS = {
    "tiny": dict(mix=TINY, n=10_000, nq=100, nlist=64, iters=10,
                 nprobe=8, k=10, n_rerank=100),
    "sift1m": dict(mix=SIFT1M, n=1_000_000, nq=10_000, batch=1000,
                   nlist=1024, iters=10, nprobe=(16, 32, 64, 128), k=10,
                   n_rerank=200),
    "highdim": dict(mix=HIGHDIM, n=1_000_000, nq=1000, nlist=1024, iters=10,
                    nprobe=(32, 128), k=(10, 100), n_rerank=500),
    "skewed": dict(mix=SKEWED, n=10_000_000, nq=4096, nlist=4096, iters=10,
                   nprobe=(8, 256), k=(10, 100), n_rerank=200),
}


def mixture(name: str, dim: int | None = None, seed: int | None = None):
    """A recipe's mixture, optionally with another dimension or seed."""
    m = WORKLOADS[name]["mix"]
    kw = {}
    if dim is not None:
        kw["dim"] = dim
    if seed is not None:
        kw["seed"] = seed
    return dataclasses.replace(m, **kw) if kw else m


def per_query_params(nq: int, seed: int, nprobe_range=(8, 256),
                     k_choices=(10, 100)):
    """Seeded per-query (nprobe, k) mix for uneven serving requests."""
    rng = np.random.default_rng([seed, 99])
    nprobe = rng.integers(nprobe_range[0], nprobe_range[1] + 1, nq)
    k = rng.choice(np.asarray(k_choices), nq)
    return nprobe.astype(np.int32), k.astype(np.int32)
