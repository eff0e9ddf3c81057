"""Plain CPU oracle of IVF-RaBitQ search and index build.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module.
The CUDA library never calls it and shares no code with it.

What the oracle follows, step by step:

* Section 2.1.2 (IVF): k-means centroids, each vector in the list of its
  nearest centroid; a query scans the lists of its nProbe nearest centroids.
* Section 2.2.1, Eqs. 1-3: normalised residuals, a random orthogonal P,
  sign codes b = sign(P^T u), the residual norm and alpha = ||P^T u||_1/sqrt(D).
* Section 2.2.2, Eqs. 4-5: the inner-product estimator and the distance
  decomposition.
* Section 3.3.2: the transformed query is scalar-quantised (B_q = 4 bits) and
  the estimator is evaluated with bitwise AND + popcount over bit-planes.
* Section 3.3.3: top-k with an upper bound, lists visited in centroid order.
* Section 3.3.4: exact re-rank of the candidates on the raw vectors.

Precision: the build (P, residual norms, alpha) runs in float64. Where the
paper leaves the arithmetic open, the search stages use a fixed float32
arithmetic (each operation rounded once, no fused multiply-add, a fixed
summation order), written out in the functions below. Given the same inputs to
a stage, any implementation that follows these readings gets the same bits.

Readings where the paper is silent (each also listed with the design notes):

* D is zero-padded to D_p = ceil(D/128)*128 and sqrt(D) becomes sqrt(D_p).
* sign(0) = +1: code bit = [z_d >= 0]; bit d lives in byte d//8, bit d%8.
* r_x = 0: code all ones, alpha = 1 (then f_x = 0 and the estimate is exact).
* Query quantisation: deterministic round-half-up to 4 bits over [vl, vr].
* k-means: initial centroids are the nlist rows of smallest Philox rank key;
  a fixed number of iterations; assignment ties to the lower centroid id; an
  empty cluster takes the member farthest from the centroid of the largest
  cluster (ties: lowest ids).
* Every ranking breaks ties by (distance, id).
"""
from __future__ import annotations

import numpy as np

from . import philox

F32 = np.float32
F64 = np.float64
BQ = 4                    # query bits (B_q)
QMAX = (1 << BQ) - 1      # 15
LANES = 32                # width of the fixed lane-sum order
BOUND_MIN = 1024          # the first bound sees at least this many candidates,
BOUND_FACTOR = 16         # and 16 n_sel of them,
BOUND_MAX = 32768         # but no more than this (or n_sel, when larger)
U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)
U32_MAX = 0xFFFFFFFF

_POP8 = np.array([bin(i).count("1") for i in range(256)], np.int64)


def dim_pad(d: int) -> int:
    """D_p: the input dimension rounded up to a multiple of 128."""
    return ((d + 127) // 128) * 128


def pad(x: np.ndarray, dp: int) -> np.ndarray:
    out = np.zeros(x.shape[:-1] + (dp,), x.dtype)
    out[..., : x.shape[-1]] = x
    return out


def popcount8(a: np.ndarray) -> np.ndarray:
    """Per-row popcount of a uint8 array summed over its last axis."""
    return _POP8[a].sum(axis=-1)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Bit d -> byte d//8, bit position d%8 (least significant bit first)."""
    return np.packbits(bits.astype(np.uint8), axis=-1, bitorder="little")


def unpack_bits(codes: np.ndarray, dp: int) -> np.ndarray:
    return np.unpackbits(codes, axis=-1, bitorder="little", count=dp)


def orderable(d: np.ndarray) -> np.ndarray:
    """Monotone map of float32 to uint32: a < b  <=>  key(a) < key(b)."""
    u = np.asarray(d, F32).view(np.uint32).astype(np.uint64)
    neg = (u >> np.uint64(31)) != 0
    return np.where(neg, u ^ np.uint64(0xFFFFFFFF), u ^ np.uint64(0x80000000))


def from_orderable(o: np.ndarray) -> np.ndarray:
    o = np.asarray(o, np.uint64)
    pos = (o >> np.uint64(31)) != 0
    u = np.where(pos, o ^ np.uint64(0x80000000), o ^ np.uint64(0xFFFFFFFF))
    return u.astype(np.uint32).view(F32)


def make_keys(d: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """(distance, id) packed so that integer order is (distance, id) order."""
    return (orderable(d) << np.uint64(32)) | np.asarray(ids, np.uint64)


def key_dist(keys):
    return from_orderable(np.asarray(keys, np.uint64) >> np.uint64(32))


def key_id(keys):
    return (np.asarray(keys, np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.int64)


# --------------------------------------------------------------------------
# Fixed float32 reductions
# --------------------------------------------------------------------------
def lane_sum(v: np.ndarray) -> np.ndarray:
    """Sum over the last axis in the 32-lane order (float32).

    Lane l accumulates the terms d = l, l+32, l+64, ... in increasing d,
    starting from 0; the 32 lane sums are then combined pairwise with
    strides 16, 8, 4, 2, 1 (lane l adds lane l+stride).
    """
    v = np.asarray(v, F32)
    acc = np.zeros(v.shape[:-1] + (LANES,), F32)
    for j in range(0, v.shape[-1], LANES):
        blk = v[..., j:j + LANES]
        w = blk.shape[-1]
        acc[..., :w] = acc[..., :w] + blk
    for s in (16, 8, 4, 2, 1):
        acc = acc[..., :s] + acc[..., s:2 * s]
    return acc[..., 0]


def seq_sqdist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """||a_i - b_j||^2 for all pairs, float32, summed over d = 0, 1, ... in order.

    a: (n, d), b: (m, d) -> (n, m). Each term is (a - b) rounded, squared and
    rounded, then added and rounded (no fused multiply-add).
    """
    a = np.asarray(a, F32)
    b = np.asarray(b, F32)
    acc = np.zeros((a.shape[0], b.shape[0]), F32)
    for d in range(a.shape[1]):
        diff = a[:, d, None] - b[None, :, d]
        acc = acc + diff * diff
    return acc


# --------------------------------------------------------------------------
# Build: P (Section 2.2.1, Eq. 3)
# --------------------------------------------------------------------------
def gaussian_matrix(seed: int, dp: int) -> np.ndarray:
    return philox.gaussian(seed, philox.STREAM_ROTATION, dp * dp).reshape(dp, dp)


def random_orthogonal(seed: int, dp: int) -> np.ndarray:
    """P = Q diag(sign(diag R)) for G = QR, G a D_p x D_p Gaussian matrix.

    With the sign fix the factor is unique, and P is distributed uniformly
    (Haar) over the orthogonal group.
    """
    g = gaussian_matrix(seed, dp)
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


# --------------------------------------------------------------------------
# Build: k-means (Section 2.1.2; Section 3.1.1 Phases 1-2)
# --------------------------------------------------------------------------
def train_rows(seed: int, n: int, n_train: int) -> np.ndarray:
    """Training subset: all rows, or the n_train rows of smallest rank key."""
    if n_train <= 0 or n_train >= n:
        return np.arange(n, dtype=np.int64)
    keys = philox.row_keys(seed, philox.STREAM_TRAIN_SAMPLE, n)
    return np.sort(np.argsort(keys)[:n_train]).astype(np.int64)


def kmeans_init(seed: int, n: int, rows: np.ndarray, nlist: int) -> np.ndarray:
    """Initial centroid rows: the nlist training rows with the smallest rank
    keys, in ascending key order (a uniform sample without replacement)."""
    keys = philox.row_keys(seed, philox.STREAM_KMEANS_INIT, n)[rows]
    return rows[np.argsort(keys)[:nlist]]


def assign(x: np.ndarray, c: np.ndarray, chunk: int = 4096):
    """Nearest centroid of each row; ties go to the lower centroid id.

    Distances: float32, summed over dimensions in order (``seq_sqdist``).
    Returns (assignment, its distance).
    """
    n = x.shape[0]
    a = np.empty(n, np.int64)
    dist = np.empty(n, F32)
    for i in range(0, n, chunk):
        d = seq_sqdist(x[i:i + chunk], c)
        a[i:i + chunk] = np.argmin(d, axis=1)
        dist[i:i + chunk] = d[np.arange(d.shape[0]), a[i:i + chunk]]
    return a, dist


def sqdist_f64(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """||a_i - b_j||^2 for all pairs in float64 as ||a||^2 - 2 <a, b> + ||b||^2
    (one matrix product). For float32 inputs every product is exact in
    float64 and the result is within a few float64 ulps of ||a||^2 + ||b||^2
    of the exact value; used where the float64 independent build needs the
    plain distance, not the fixed float32 order."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    d = (a * a).sum(axis=1)[:, None] - 2.0 * (a @ b.T) + (b * b).sum(axis=1)[None, :]
    return np.maximum(d, 0.0)


def _nearest_f64(job):
    """(rows, centroids) -> nearest centroid of each row and its distance."""
    x, c = job
    d = sqdist_f64(x, c)
    a = np.argmin(d, axis=1)
    return a, d[np.arange(d.shape[0]), a]


def assign_f64(x: np.ndarray, c: np.ndarray, chunk: int = 8192, map_fn=map):
    """Nearest centroid of each row (Section 2.1.2) by float64 distance
    (``sqdist_f64``), ties to the lower centroid id. Returns (assignment, its
    distance). Row chunks are independent; ``map_fn`` (default: the builtin
    map) may spread them over worker processes."""
    n = x.shape[0]
    a = np.empty(n, np.int64)
    dist = np.empty(n, F64)
    starts = range(0, n, chunk)
    for i, (ai, di) in zip(starts, map_fn(_nearest_f64, ((x[i:i + chunk], c) for i in starts))):
        a[i:i + chunk] = ai
        dist[i:i + chunk] = di
    return a, dist


def update(x: np.ndarray, a: np.ndarray, nlist: int, dist=None) -> np.ndarray:
    """New centroids: mean of the members, summed in float64 in ascending row
    order, divided in float64, rounded to float32. Empty clusters are then
    re-seeded in ascending id: each takes, from the currently largest cluster
    (ties: lowest id), its member farthest from that cluster's new centroid
    (ties: lowest row), which moves to the empty cluster. ``dist`` is the
    distance used for that (default: the fixed float32 order).
    """
    dist = seq_sqdist if dist is None else dist
    n, d = x.shape
    c = np.zeros((nlist, d), F32)
    counts = np.bincount(a, minlength=nlist)
    order = np.argsort(a, kind="stable")
    starts = np.concatenate([[0], np.cumsum(counts)])
    for j in range(nlist):
        if counts[j] == 0:
            continue
        mem = order[starts[j]:starts[j + 1]]
        s = np.cumsum(x[mem].astype(F64), axis=0)[-1]
        c[j] = (s / F64(counts[j])).astype(F32)
    a = a.copy()
    for j in np.flatnonzero(counts == 0):
        donor = int(np.argmax(counts))
        mem = np.flatnonzero(a == donor)
        dd = dist(x[mem], c[donor:donor + 1])[:, 0]
        far = mem[int(np.argmax(dd))]
        c[j] = x[far]
        a[far] = j
        counts[donor] -= 1
        counts[j] += 1
    return c


def kmeans(x: np.ndarray, nlist: int, iters: int, seed: int,
           n_train: int = 0, return_history: bool = False, f64: bool = False,
           map_fn=map):
    """Lloyd iterations from the seeded initial rows (fixed iteration count).
    Distances in the fixed float32 order, or in float64 with ``f64`` (the
    independent build; ``map_fn`` may spread its row chunks over workers)."""
    n = x.shape[0]
    rows = train_rows(seed, n, n_train)
    xt = x[rows]
    c = x[kmeans_init(seed, n, rows, nlist)].astype(F32)
    nearest = (lambda xx, cc: assign_f64(xx, cc, map_fn=map_fn)) if f64 else assign
    hist = []
    for _ in range(iters):
        a, dist = nearest(xt, c)
        hist.append(float(dist.astype(F64).sum()))
        c = update(xt, a, nlist, sqdist_f64 if f64 else None)
    if return_history:
        a, dist = nearest(xt, c)
        hist.append(float(dist.astype(F64).sum()))
        return c, hist
    return c


# --------------------------------------------------------------------------
# Build: encode (Eqs. 1-3; Section 3.2.2)
# --------------------------------------------------------------------------
def encode(x: np.ndarray, c: np.ndarray, a: np.ndarray, P: np.ndarray):
    """Sign codes and factors of each row against its centroid, in float64.

    u = x - c (unnormalised), r = ||u||, z = P^T [u; 0], bit_d = [z_d >= 0],
    alpha = ||z||_1 / (sqrt(D_p) r), which is <P b / sqrt(D_p), u / r> for
    b = sign(z) (Eq. 3). r = 0 gives all-ones codes and alpha = 1.
    Returns codes (n, D_p/8) uint8, r (n,) f64, alpha (n,) f64, z (n, D_p).
    """
    dp = P.shape[0]
    u = x.astype(F64) - c[a].astype(F64)
    r = np.sqrt((u * u).sum(axis=1))
    z = pad(u, dp) @ P
    bits = z >= 0
    alpha = np.abs(z).sum(axis=1) / (np.sqrt(F64(dp)) * np.where(r > 0, r, 1.0))
    alpha = np.where(r > 0, alpha, 1.0)
    return pack_bits(bits), r, alpha, z


def _encode_rows(job):
    """(rows, their centroids, P) -> codes, r, alpha of ``encode``."""
    x, c, P = job
    codes, r, alpha, _ = encode(x, c, np.arange(x.shape[0]), P)
    return codes, r, alpha


def scan_factors(r32: np.ndarray, alpha32: np.ndarray, dp: int):
    """Per-vector float32 constants of the estimator: r^2 and
    f = r / (sqrt(D_p) * alpha), each a single float32 operation."""
    r32 = np.asarray(r32, F32)
    alpha32 = np.asarray(alpha32, F32)
    sq = F32(np.sqrt(F32(dp)))
    return r32 * r32, r32 / (sq * alpha32)


def build_index(x: np.ndarray, nlist: int, seed: int, iters: int = 10,
                n_train: int = 0, centroids: np.ndarray | None = None,
                P: np.ndarray | None = None, f64: bool = False, map_fn=map,
                chunk: int = 1 << 16):
    """Index build (k-means, P, encode, list layout); P, the residual norms
    and alpha are always float64.

    ``centroids`` and ``P`` may be given to rebuild an index from another
    build's centroids and rotation (replay of the encode step). With ``f64``
    the k-means and list assignments use float64 distances (the independent
    build of the benchmark's CPU baseline); otherwise the fixed float32 order
    that the GPU build follows. The assignment and the encode work on
    independent row chunks; ``map_fn`` (default: the builtin map) may spread
    them over worker processes.
    """
    x = np.asarray(x, F32)
    n, d = x.shape
    dp = dim_pad(d)
    if P is None:
        P = random_orthogonal(seed, dp)
    if centroids is None:
        centroids = kmeans(x, nlist, iters, seed, n_train, f64=f64, map_fn=map_fn)
    a, _ = assign_f64(x, centroids, map_fn=map_fn) if f64 else assign(x, centroids)
    order = np.lexsort((np.arange(n), a))          # list order, then row id
    counts = np.bincount(a, minlength=nlist)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    starts = range(0, n, chunk)
    jobs = ((x[order[i:i + chunk]], centroids[a[order[i:i + chunk]]], P) for i in starts)
    parts = list(map_fn(_encode_rows, jobs))
    codes = np.concatenate([p[0] for p in parts]) if parts else np.zeros((0, dp // 8), np.uint8)
    r = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0)
    alpha = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0)
    r32, al32 = r.astype(F32), alpha.astype(F32)
    r2, f = scan_factors(r32, al32, dp)
    cR = (pad(centroids.astype(F64), dp) @ P).astype(F32)
    return dict(n=n, dim=d, dp=dp, nlist=nlist, P=P, centroids=centroids,
                cR=cR, offsets=offsets, ids=order.astype(np.int64),
                assign=a, codes=codes, r=r32, alpha=al32, r2=r2, f=f,
                raw=x)


# --------------------------------------------------------------------------
# Search (Section 2.1.2 query processing; Sections 2.2.2, 3.3)
# --------------------------------------------------------------------------
def rotate(q: np.ndarray, P: np.ndarray) -> np.ndarray:
    """q' = P^T [q; 0] in float64, rounded to float32 (done once per query;
    P^T (q - c) = q' - P^T c because P is linear)."""
    return (pad(np.asarray(q, F64), P.shape[0]) @ P).astype(F32)


def probe(qrot: np.ndarray, cR: np.ndarray, nprobe: int):
    """The nprobe nearest centroids of each rotated query, by (distance, id).

    Distance ||q' - P^T c||^2 (= ||q - c||^2 by orthogonality) in float32,
    summed over d in order. Returns ids (nq, nprobe) and distances.
    """
    dist = seq_sqdist(qrot, cR)
    ids = np.arange(cR.shape[0])
    out_i = np.empty((qrot.shape[0], nprobe), np.int64)
    out_d = np.empty((qrot.shape[0], nprobe), F32)
    for i in range(qrot.shape[0]):
        keys = np.sort(make_keys(dist[i], ids))[:nprobe]
        out_i[i], out_d[i] = key_id(keys), key_dist(keys)
    return out_i, out_d


def quantize(res: np.ndarray):
    """B_q = 4 scalar quantisation of rotated residuals (rows of ``res``).

    vl = min, vr = max, delta = (vr - vl)/15, inv = 15/(vr - vl),
    q_u = min(15, floor((r - vl)*inv + 0.5)); all zero when vr == vl.
    nq2 = ||res||^2 in the 32-lane order. Sq = sum q_u. plane j holds bit j
    of every q_u, packed like the codes.
    """
    res = np.asarray(res, F32)
    vl = res.min(axis=-1)
    vr = res.max(axis=-1)
    width = vr - vl
    same = width == 0
    safe = np.where(same, F32(1), width)
    delta = np.where(same, F32(0), width / F32(QMAX)).astype(F32)
    inv = np.where(same, F32(0), F32(QMAX) / safe).astype(F32)
    y = (res - vl[..., None]) * inv[..., None] + F32(0.5)
    qu = np.minimum(np.floor(y).astype(np.int64), QMAX)
    qu[same] = 0
    sq = qu.sum(axis=-1)
    nq2 = lane_sum(res * res)
    planes = np.stack([pack_bits((qu >> j) & 1) for j in range(BQ)], axis=-2)
    return dict(qu=qu, vl=vl, delta=delta, nq2=nq2, sq=sq, planes=planes)


def ip_planes(codes: np.ndarray, planes: np.ndarray) -> np.ndarray:
    """sum_d bit_d * q_u,d as sum_j 2^j popcount(code AND plane_j)."""
    return sum((1 << j) * popcount8(codes & planes[j]) for j in range(BQ))


def estimate(codes, r2, f, quant: dict, dp: int, qi=None) -> np.ndarray:
    """Estimated squared distance (Eqs. 4-5) with the quantised query, float32.

    With ip = sum bit*q_u and pc = popcount(code):
      t  = delta*(2 ip - Sq) + vl*(2 pc - D_p)   (= sum_d b_d * r_d, dequantised)
      d2 = (nq2 + r^2) - 2*(f*t),   f = r/(sqrt(D_p)*alpha),
    then + 0 to turn -0 into +0. ``qi`` picks one quantised residual.
    """
    g = (lambda k: quant[k]) if qi is None else (lambda k: quant[k][qi])
    ip = ip_planes(codes, g("planes"))
    pc = popcount8(codes)
    a = (2 * ip - g("sq")).astype(F32)
    b = (2 * pc - dp).astype(F32)
    t = g("delta") * a + g("vl") * b
    d2 = (g("nq2") + np.asarray(r2, F32)) - F32(2) * (np.asarray(f, F32) * t)
    return (d2 + F32(0)).astype(F32)


def lut_tables(res: np.ndarray) -> np.ndarray:
    """FastScan tables of one rotated residual (Section 3.3.2, the paper's
    estimator: the query is not quantised). For group g of eight dimensions
    and byte value v, T[g, v] is the float32 sum of res[8 g + i] over the set
    bits i of v, added in increasing i from 0. res: (D_p,) -> (D_p/8, 256).
    """
    res = np.asarray(res, F32)
    groups = res.shape[-1] // 8
    out = np.zeros((groups, 256), F32)
    for v in range(256):
        acc = np.zeros(groups, F32)
        for i in range(8):
            if (v >> i) & 1:
                acc = acc + res[i::8]       # res[8 g + i] for every group g
        out[:, v] = acc
    return out


def estimate_lut(codes, r2, f, res) -> np.ndarray:
    """Estimated squared distance (Eqs. 4-5) with the full-precision rotated
    residual, in the FastScan form (float32): s = sum over groups g, in
    increasing g, of T[g, code byte g] (so s = sum_d bit_d res_d);
    t = 2 s - S, S = sum_d res_d in the 32-lane order (so t = sum_d b_d res_d,
    b_d = 2 bit_d - 1); d2 = (nq2 + r^2) - 2 (f t), nq2 = ||res||^2 in the
    32-lane order; then + 0."""
    res = np.asarray(res, F32)
    T = lut_tables(res)
    codes = np.asarray(codes, np.uint8)
    s = np.zeros(codes.shape[0], F32)
    for g in range(T.shape[0]):
        s = s + T[g][codes[:, g]]
    t = F32(2) * s - lane_sum(res)
    nq2 = lane_sum(res * res)
    d2 = (nq2 + np.asarray(r2, F32)) - F32(2) * (np.asarray(f, F32) * t)
    return (d2 + F32(0)).astype(F32)


def list_candidates(index: dict, qrot_i: np.ndarray, probe_ids: np.ndarray,
                    estimator: str = "bq4"):
    """Estimated distances of every vector in the probed lists of one query,
    in probe order and list order. Returns (d2, ids, quantisations); with
    ``estimator="lut"`` the unquantised FastScan form is used and the
    quantisations list holds the residuals."""
    off = index["offsets"]
    ds, ids, qs = [], [], []
    for c in probe_ids:
        lo, hi = int(off[c]), int(off[c + 1])
        res = (qrot_i - index["cR"][c])
        if estimator == "lut":
            qs.append(res)
            ds.append(estimate_lut(index["codes"][lo:hi], index["r2"][lo:hi],
                                   index["f"][lo:hi], res))
        else:
            q = quantize(res[None, :])
            qs.append(q)
            ds.append(estimate(index["codes"][lo:hi], index["r2"][lo:hi],
                               index["f"][lo:hi], q, index["dp"], qi=0))
        ids.append(index["ids"][lo:hi])
    if not ds:
        return np.zeros(0, F32), np.zeros(0, np.int64), qs
    return np.concatenate(ds), np.concatenate(ids), qs


def bound_window(n_sel: int) -> int:
    """How many candidates, in probe order, set a query's first bound:
    max(1024, n_sel, min(16 n_sel, 32768))."""
    return max(BOUND_MIN, n_sel, min(BOUND_FACTOR * n_sel, BOUND_MAX))


def first_bound(d2: np.ndarray, n_sel: int, window: int | None = None):
    """Upper bound for pruning (Section 3.3.3): the n_sel-th smallest
    orderable distance among the first ``bound_window(n_sel)`` candidates in
    probe order (lists by ascending centroid distance, so the prefix holds
    the most promising candidates); no bound (all ones) when the query has
    fewer than n_sel candidates. The n_sel-th smallest of any prefix is at or
    above the n_sel-th smallest of all candidates, so nothing the selection
    keeps is pruned; a longer prefix gives a tighter bound.
    """
    if d2.size < n_sel or n_sel == 0:
        return U32_MAX
    m = min(d2.size, bound_window(n_sel) if window is None else window)
    return int(np.sort(orderable(d2[:m]))[n_sel - 1])


def select_running_bound(d2, ids, n_sel: int):
    """The paper's Top-k with a running upper bound (Section 3.3.3), written
    out one candidate at a time: candidates arrive in probe order (lists by
    ascending centroid distance); once n_sel keys are held, the bound is the
    largest held key, a candidate above it is pruned, and one below it
    replaces the held maximum. Returns the held keys ascending and how many
    candidates were pruned.

    The first-bound form used by ``select_candidates`` (one bound fixed from
    the first candidates) is a different schedule of the same idea; both
    return the n_sel smallest keys.
    """
    keys = make_keys(d2, ids)
    held: list[int] = []
    pruned = 0
    for key in (int(v) for v in keys):
        if len(held) < n_sel:
            held.append(key)
            continue
        top = max(held)
        if key > top:
            pruned += 1
            continue
        held.remove(top)
        held.append(key)
    return np.array(sorted(held), np.uint64), pruned


def select_candidates(d2, ids, n_sel: int, prune: bool = True):
    """The n_sel smallest (distance, id) keys, ascending.

    With ``prune``, candidates above the first bound are dropped before the
    selection; the result is the same since the bound is never below the
    n_sel-th key.
    """
    keys = make_keys(d2, ids)
    if prune:
        tau = first_bound(d2, n_sel)
        keys = keys[orderable(d2) <= np.uint64(tau)]
    return np.sort(keys)[:n_sel]


def rerank(raw: np.ndarray, q: np.ndarray, cand_ids: np.ndarray, k: int):
    """Exact float32 squared distances (32-lane order) of the candidates,
    top k by (distance, id). Pads with id -1 and +inf."""
    out_i = np.full(k, -1, np.int64)
    out_d = np.full(k, np.inf, F32)
    if cand_ids.size:
        diff = np.asarray(raw, F32)[cand_ids] - np.asarray(q, F32)[None, :]
        d = lane_sum(diff * diff)
        keys = np.sort(make_keys(d, cand_ids))[:k]
        out_i[:keys.size], out_d[:keys.size] = key_id(keys), key_dist(keys)
    return out_i, out_d


def search(index: dict, q: np.ndarray, nprobe, k, n_rerank, qrot=None,
           prune: bool = True, return_stages: bool = False, estimator: str = "bq4"):
    """Full search of a batch. ``nprobe``, ``k``, ``n_rerank`` are scalars or
    per-query arrays. ``qrot`` replaces the float64 rotation (replay of a
    rotation computed elsewhere). n_rerank = 0 returns the top k by the
    estimate, without re-rank. ``estimator``: "bq4" (4-bit query, bit-plane
    popcounts) or "lut" (full-precision query, FastScan tables).
    """
    q = np.asarray(q, F32)
    nq = q.shape[0]
    as_arr = lambda v: np.broadcast_to(np.asarray(v, np.int64), (nq,))
    npb, kk, nrr = as_arr(nprobe), as_arr(k), as_arr(n_rerank)
    if qrot is None:
        qrot = rotate(q, index["P"])
    pid, pd = probe(qrot, index["cR"], int(npb.max()) if nq else 0)
    kmax = int(kk.max()) if nq else 0
    ids = np.full((nq, kmax), -1, np.int64)
    dist = np.full((nq, kmax), np.inf, F32)
    stages = []
    for i in range(nq):
        d2, cid, qs = list_candidates(index, qrot[i], pid[i, :npb[i]], estimator)
        n_sel = int(nrr[i]) if nrr[i] > 0 else int(kk[i])
        sel = select_candidates(d2, cid, n_sel, prune)
        if nrr[i] > 0:
            oi, od = rerank(index["raw"], q[i], key_id(sel), int(kk[i]))
        else:
            oi = np.full(kk[i], -1, np.int64)
            od = np.full(kk[i], np.inf, F32)
            oi[:sel.size], od[:sel.size] = key_id(sel), key_dist(sel)
        ids[i, :kk[i]], dist[i, :kk[i]] = oi, od
        if return_stages:
            stages.append(dict(d2=d2, ids=cid, quant=qs, sel=sel,
                               tau=first_bound(d2, n_sel)))
    if return_stages:
        return ids, dist, dict(qrot=qrot, probe_ids=pid, probe_d=pd,
                               per_query=stages)
    return ids, dist


# --------------------------------------------------------------------------
# Ground truth
# --------------------------------------------------------------------------
def exact_knn(x: np.ndarray, q: np.ndarray, k: int, chunk: int = 256):
    """Brute-force exact kNN in float64, ties by (distance, id)."""
    x64 = np.asarray(x, F64)
    xn = (x64 * x64).sum(axis=1)
    ids = np.empty((q.shape[0], k), np.int64)
    dist = np.empty((q.shape[0], k), F64)
    for i in range(0, q.shape[0], chunk):
        qq = np.asarray(q[i:i + chunk], F64)
        d = xn[None, :] - 2.0 * qq @ x64.T + (qq * qq).sum(axis=1)[:, None]
        part = np.argpartition(d, min(k + 8, d.shape[1] - 1), axis=1)[:, :k + 8]
        for j in range(qq.shape[0]):
            cand = part[j]
            dd = ((x64[cand] - qq[j]) ** 2).sum(axis=1)
            o = np.lexsort((cand, dd))[:k]
            ids[i + j], dist[i + j] = cand[o], dd[o]
    return ids, dist


def exact_dist(x: np.ndarray, q: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """float64 squared distances of q[i] to x[ids[i, j]] (nan for id -1)."""
    out = np.full(ids.shape, np.nan)
    for i in range(ids.shape[0]):
        ok = ids[i] >= 0
        diff = np.asarray(x, F64)[ids[i, ok]] - np.asarray(q[i], F64)
        out[i, ok] = (diff * diff).sum(axis=1)
    return out


def recall_at(x, q, ids, true_dist, k: int) -> float:
    """Tie-aware recall@k: a returned id is a hit if its exact distance is at
    most the k-th true distance."""
    d = exact_dist(x, q, ids[:, :k])
    kth = true_dist[:, k - 1][:, None]
    hits = np.nan_to_num(d, nan=np.inf) <= kth * (1 + 1e-12)
    return float(hits.sum()) / (ids.shape[0] * k)
