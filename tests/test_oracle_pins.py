"""Pins of the CPU oracle against what the paper and mathematics fix.

Each oracle function is checked against something other than itself:
published known-answer vectors, a hand-derived worked example, closed forms,
invariants (orthogonality, the alpha identity of Eq. 3, the integer identity
behind the bit-plane estimator), unbiasedness of Eq. 4 over random rotations,
error bounds against float64, and brute force on tiny inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import philox, rabitq as R
from tests.conftest import read_golden

F32, F64 = np.float32, np.float64


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    _, lines = read_golden("philox4x32_10_kat.txt")
    for row in lines:
        v = [int(t, 16) for t in row]
        out = philox.philox4x32_10([v[0:4]], v[4:6])[0]
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_moments_and_unit_map():
    g = philox.gaussian(7, philox.STREAM_ROTATION, 400_000)
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    # kurtosis of a normal is 3
    assert abs((g ** 4).mean() / g.var() ** 2 - 3.0) < 0.05
    a = np.array([0, 2**64 - 1, 2**63], dtype=np.uint64)
    u = philox.unit_open(a)
    assert u[0] == 0.5 * 2.0**-52 and u[1] == 1.0 - 0.5 * 2.0**-52 and u[2] == 0.5 + 0.5 * 2.0**-52


# ---------------------------------------------------------------- P
@pytest.mark.parametrize("dp", [128, 1024])
def test_rotation_orthogonal(dp):
    P = R.random_orthogonal(3, dp)
    err = np.abs(P.T @ P - np.eye(dp)).max()
    assert err <= 1e-12
    v = np.random.default_rng(0).standard_normal(dp)
    assert abs(np.linalg.norm(P.T @ v) - np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(v)


def test_rotation_is_signed_qr_of_gaussian():
    # G = P R' must hold with R' = P^T G upper triangular, positive diagonal.
    dp = 128
    G = R.gaussian_matrix(11, dp)
    P = R.random_orthogonal(11, dp)
    Rp = P.T @ G
    assert np.abs(np.tril(Rp, -1)).max() < 1e-11
    assert (np.diag(Rp) > 0).all()
    # Haar sanity: entries have variance 1/D_p
    assert abs(P.var() * dp - 1.0) < 0.05


# ---------------------------------------------------------------- keys
def test_orderable_is_monotone_and_invertible():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(5000).astype(F32) * 1e3,
                        np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45], F32)])
    o = R.orderable(v)
    for i in range(0, v.size - 1):
        a, b = v[i], v[i + 1]
        if a < b:
            assert o[i] < o[i + 1]
        elif a > b:
            assert o[i] > o[i + 1]
    back = R.from_orderable(o)
    same = (back == v)
    assert same.all()
    keys = R.make_keys(v, np.arange(v.size))
    srt = np.sort(keys)
    ref = sorted(range(v.size), key=lambda i: (float(v[i]), i))
    # -0 and +0 are equal floats (keys order -0 first); == treats them equal
    assert np.array_equal(R.key_dist(srt), v[ref])
    assert np.all(np.diff(R.key_dist(srt).astype(F64)) >= 0)


# ---------------------------------------------------------------- sums
def test_lane_sum_error_bound_and_small_cases():
    rng = np.random.default_rng(2)
    for n in (1, 7, 31, 32, 33, 96, 128, 960, 1024):
        v = rng.standard_normal((20, n)).astype(F32)
        s = R.lane_sum(v * v)
        ex = (v.astype(F64) ** 2).sum(axis=1)
        # |err| <= (n/32 + 5) * eps * sum|terms| (sequential then tree depth 5)
        bound = (n / 32 + 6) * 2.0**-24 * ex
        assert np.all(np.abs(s - ex) <= bound + 1e-30)
    # exact on integers: the result is an exact sum when all partial sums fit
    v = rng.integers(-100, 100, (10, 128)).astype(F32)
    assert np.array_equal(R.lane_sum(v), v.astype(F64).sum(axis=1))


def test_lane_sum_order_by_hand():
    # 2^24 sits where float32 spacing is 2, so 2^24 + 1 rounds back to 2^24
    # (ties to even) while 2^24 + 2 is exact. Terms 1 at d = 1 and d = 17
    # meet first at the stride-16 step (lane 1 + lane 17 = 2), then join lane
    # 0 at stride 1: 2^24 + 2. Summed in d order (or with adjacent lanes
    # paired first) each 1 is lost against 2^24: 2^24.
    v = np.zeros((1, 64), F32)
    v[0, 0], v[0, 1], v[0, 17] = 2.0**24, 1.0, 1.0
    assert R.lane_sum(v)[0] == 2.0**24 + 2
    # terms of one lane (d = 1 and 33) add in increasing d before the tree
    w = np.zeros((1, 64), F32)
    w[0, 1], w[0, 33], w[0, 0] = 2.0**24, 1.0, 1.0
    assert R.lane_sum(w)[0] == 2.0**24      # lane 1: 2^24 + 1 -> 2^24; + lane 0's 1 -> 2^24


def test_seq_sqdist_order_by_hand():
    # squares 2^24, 1, 1 added in d order: each 1 is lost (2^24 + 1 -> 2^24);
    # any order that adds the two ones first gives 2^24 + 2
    a = np.array([[4096.0, 1.0, 1.0]], F32)
    assert R.seq_sqdist(a, np.zeros((1, 3), F32))[0, 0] == 2.0**24
    b = np.array([[1.0, 1.0, 4096.0]], F32)
    assert R.seq_sqdist(b, np.zeros((1, 3), F32))[0, 0] == 2.0**24 + 2


def test_seq_sqdist_error_bound():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((17, 128)).astype(F32)
    b = rng.standard_normal((9, 128)).astype(F32)
    d = R.seq_sqdist(a, b)
    ex = ((a.astype(F64)[:, None, :] - b.astype(F64)[None]) ** 2).sum(-1)
    assert np.all(np.abs(d - ex) <= (128 + 4) * 2.0**-24 * ex)


# ---------------------------------------------------------------- k-means
def test_kmeans_init_is_smallest_keys():
    n, nlist, seed = 300, 17, 5
    rows = np.arange(n)
    got = R.kmeans_init(seed, n, rows, nlist)
    keys = philox.row_keys(seed, philox.STREAM_KMEANS_INIT, n)
    w0 = philox.stream_block(seed, philox.STREAM_KMEANS_INIT, np.arange(n))[:, 0]
    ref = sorted(range(n), key=lambda i: (int(w0[i]), i))[:nlist]
    assert list(got) == ref
    assert np.array_equal(keys >> np.uint64(32), w0.astype(np.uint64))
    assert len(set(got.tolist())) == nlist


def test_train_subset():
    rows = R.train_rows(9, 1000, 100)
    assert rows.size == 100 and np.all(np.diff(rows) > 0)
    assert np.array_equal(R.train_rows(9, 1000, 0), np.arange(1000))


def test_train_rows_are_smallest_keys():
    """The training subset is the n_train rows whose Philox word (stream 3)
    is smallest, ties by row, returned in ascending row order -- checked by
    ranking the rows here one by one from the raw generator output."""
    n, n_train, seed = 257, 40, 21
    w0 = philox.stream_block(seed, philox.STREAM_TRAIN_SAMPLE, np.arange(n))[:, 0]
    ranked = sorted(range(n), key=lambda i: (int(w0[i]), i))
    assert list(R.train_rows(seed, n, n_train)) == sorted(ranked[:n_train])
    # the largest keys, or another stream's keys, give another subset
    assert sorted(ranked[-n_train:]) != sorted(ranked[:n_train])
    w_init = philox.stream_block(seed, philox.STREAM_KMEANS_INIT, np.arange(n))[:, 0]
    other = sorted(sorted(range(n), key=lambda i: (int(w_init[i]), i))[:n_train])
    assert list(R.train_rows(seed, n, n_train)) != other


def test_float64_assignment_is_nearest_exactly():
    """The float64 assignment of the independent build: on integer-valued
    rows (every float64 operation exact) it is the brute-force nearest
    centroid by exact squared distance, ties (duplicate centroids) to the
    lower id; on real-valued rows its distances are within float64 rounding
    of the exact ones."""
    rng = np.random.default_rng(19)
    x = rng.integers(0, 256, (300, 16)).astype(F32)
    c = rng.integers(0, 256, (24, 16)).astype(F32)
    c[20:] = c[3:7]                        # duplicates: ties go to 3..6
    d = R.sqdist_f64(x, c)
    ex = np.array([[sum((int(a) - int(b)) ** 2 for a, b in zip(xi, cj)) for cj in c] for xi in x])
    assert np.array_equal(d, ex.astype(F64))
    a, dist = R.assign_f64(x, c, chunk=64)
    ref = [min(range(24), key=lambda j: (ex[i, j], j)) for i in range(300)]
    assert list(a) == ref and np.array_equal(dist, ex[np.arange(300), ref].astype(F64))
    xr = rng.standard_normal((50, 96)).astype(F32)
    cr = rng.standard_normal((30, 96)).astype(F32)
    exr = ((xr.astype(F64)[:, None] - cr.astype(F64)[None]) ** 2).sum(-1)
    assert np.allclose(R.sqdist_f64(xr, cr), exr, rtol=1e-13, atol=1e-12)


def test_update_is_mean_and_reseeds_empty():
    # 1-D example worked by hand: centroids 0, 0 (duplicate), 10.
    x = np.array([[-1.0], [1.0], [2.0], [9.0], [11.0], [30.0]], F32)
    c0 = np.array([[0.0], [0.0], [10.0]], F32)
    a, _ = R.assign(x, c0)
    assert list(a) == [0, 0, 0, 2, 2, 2]      # tie 0 vs 1 goes to 0
    c1 = R.update(x, a, 3)
    # cluster 0 mean = 2/3, cluster 2 mean = 50/3; cluster 1 is empty. The
    # largest clusters are 0 and 2 (3 members each) -> 0 (lowest id). Its
    # members lie at distances 5/3, 1/3, 4/3 from 2/3, so -1.0 moves.
    assert c1[0, 0] == F32(2.0 / 3.0) and c1[2, 0] == F32(50.0 / 3.0)
    assert c1[1, 0] == -1.0


def test_kmeans_objective_nonincreasing_and_recovers_mixture():
    mix = W.mixture("tiny")
    x, lab = mix.base(3000, labels=True)
    c, hist = R.kmeans(x, 64, 8, seed=0, return_history=True)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-6) for i in range(len(hist) - 1))
    assert hist[-1] < 0.5 * hist[0]
    # Started from the true component means of a well separated mixture, one
    # assignment recovers the labels exactly and the update gives the mean of
    # each component's rows.
    means = mix.means().astype(F32)
    a, _ = R.assign(x, means)
    assert np.array_equal(a, lab)
    c1 = R.update(x, a, 64)
    for j in range(64):
        m = x[lab == j].astype(F64).mean(axis=0)
        assert np.allclose(c1[j], m, rtol=0, atol=1e-6 * (1 + np.abs(m).max()))


# ---------------------------------------------------------------- encode
def test_alpha_identity_and_codes():
    mix = W.mixture("tiny")
    x = mix.base(500)
    c = x[:4].copy()
    a, _ = R.assign(x, c)
    P = R.random_orthogonal(1, 128)
    codes, r, alpha, z = R.encode(x, c, a, P)
    u = x.astype(F64) - c[a].astype(F64)
    assert np.allclose(np.linalg.norm(z, axis=1), r, rtol=1e-12)
    bits = R.unpack_bits(codes, 128).astype(F64)
    b = 2 * bits - 1
    ok = r > 0
    # <P b / sqrt(D), u / r> = ||P^T u||_1 / (sqrt(D) r)   (Eq. 3)
    lhs = ((b @ P.T) * u).sum(axis=1) / (math.sqrt(128) * np.where(ok, r, 1))
    assert np.allclose(lhs[ok], alpha[ok], rtol=1e-12, atol=0)
    assert np.all((alpha > 0) & (alpha <= 1 + 1e-12))
    # sign convention: bit = [z >= 0]
    assert np.array_equal(bits.astype(bool), z >= 0)


def test_build_layout_and_chunked_encode():
    """build_index lays the rows out list by list (ascending row id inside a
    list) and encodes each against its own list's centroid: its codes and
    factors equal Eqs. 1-3 applied to every row directly, whatever the
    chunking of the rows and whether the chunks are mapped by a pool."""
    mix = W.mixture("tiny")
    x = mix.base(1500)
    P = R.random_orthogonal(4, 128)
    c = R.kmeans(x, 12, 2, seed=4)
    ref = R.build_index(x, 12, seed=4, centroids=c, P=P, chunk=1 << 20)
    for chunk in (1, 97, 512):
        got = R.build_index(x, 12, seed=4, centroids=c, P=P, chunk=chunk)
        for key in ("ids", "offsets", "codes", "r", "alpha", "r2", "f"):
            assert np.array_equal(got[key], ref[key]), (chunk, key)
    a, _ = R.assign(x, c)
    order = ref["ids"]
    assert np.all(np.diff(a[order]) >= 0)
    for l in range(12):
        rows = order[ref["offsets"][l]:ref["offsets"][l + 1]]
        assert np.all(a[rows] == l) and np.all(np.diff(rows) > 0)
    codes, r, alpha, _ = R.encode(x[order], c, a[order], P)
    assert np.array_equal(ref["codes"], codes)
    assert np.array_equal(ref["r"], r.astype(F32)) and np.array_equal(ref["alpha"], alpha.astype(F32))


def test_alpha_mean_and_zero_residual():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2000, 1024)).astype(F32)
    P = R.random_orthogonal(2, 1024)
    c = np.zeros((1, 1024), F32)
    _, _, alpha, _ = R.encode(x, c, np.zeros(2000, np.int64), P)
    # mean of ||z||_1 / (sqrt(D) ||z||) for a uniform unit vector -> sqrt(2/pi)
    assert abs(alpha.mean() - math.sqrt(2 / math.pi)) < 2e-3
    codes, r, alpha, _ = R.encode(c, c, np.zeros(1, np.int64), P)
    assert r[0] == 0 and alpha[0] == 1.0 and (codes == 255).all()


# ---------------------------------------------------------------- quantize
def test_quantize_error_bound_and_degenerate():
    rng = np.random.default_rng(5)
    res = (rng.standard_normal((200, 128)) * rng.uniform(0.01, 100, (200, 1))).astype(F32)
    qz = R.quantize(res)
    qu = qz["qu"]
    assert qu.min() >= 0 and qu.max() <= 15
    recon = qu * qz["delta"][:, None].astype(F64) + qz["vl"][:, None]
    err = np.abs(recon - res)
    assert np.all(err <= qz["delta"][:, None] * (0.5 + 1e-5))
    assert np.array_equal(qz["sq"], qu.sum(axis=1))
    # bit-planes reassemble q_u
    back = sum((1 << j) * R.unpack_bits(qz["planes"][:, j], 128).astype(np.int64)
               for j in range(4))
    assert np.array_equal(back, qu)
    ex = (res.astype(F64) ** 2).sum(axis=1)
    assert np.all(np.abs(qz["nq2"] - ex) <= 10 * 2.0**-24 * ex)
    # vr == vl: all zeros
    flat = np.full((1, 128), 3.5, F32)
    q1 = R.quantize(flat)
    assert (q1["qu"] == 0).all() and q1["delta"][0] == 0 and q1["sq"][0] == 0


# ---------------------------------------------------------------- estimator
def _lut_ip(codes, qu):
    """FastScan form (Section 3.3.2): per 8-dim chunk, a 256-entry table of
    sum of q_u over the set bits, indexed by the code byte."""
    total = np.zeros(codes.shape[0], np.int64)
    for j in range(codes.shape[1]):
        table = np.array([sum(qu[8 * j + b] for b in range(8) if (v >> b) & 1)
                          for v in range(256)])
        total += table[codes[:, j]]
    return total


def test_integer_estimator_forms_agree_exactly():
    rng = np.random.default_rng(6)
    dp = 128
    codes = rng.integers(0, 256, (300, dp // 8), dtype=np.uint8)
    res = rng.standard_normal((1, dp)).astype(F32)
    qz = R.quantize(res)
    qu = qz["qu"][0]
    bits = R.unpack_bits(codes, dp).astype(np.int64)
    ip = R.ip_planes(codes, qz["planes"][0])
    assert np.array_equal(ip, bits @ qu)                       # brute force
    assert np.array_equal(ip, _lut_ip(codes, qu))              # gather / LUT
    sel = np.where(bits.astype(bool), qu[None, :], 0).sum(1)   # select / mask
    assert np.array_equal(ip, sel)
    b = 2 * bits - 1                                           # +-1 form
    assert np.array_equal(2 * ip - qz["sq"][0], b @ qu)
    assert np.array_equal(2 * R.popcount8(codes) - dp, b.sum(1))


def test_estimator_worked_example_by_hand():
    g, _ = read_golden("estimator_by_hand.txt")
    x = np.array([g["x"]], F32).astype(F32)
    q = np.array([g["q"]], F32).astype(F32)
    dp = 8
    P = np.eye(dp)
    c = np.zeros((1, dp), F32)
    codes, r, alpha, _ = R.encode(x, c, np.zeros(1, np.int64), P)
    assert int(codes[0, 0]) == int(g["code_byte"][0])
    assert R.popcount8(codes)[0] == int(g["popcount"][0])
    assert r[0] ** 2 == pytest.approx(float(g["r2"][0]), rel=1e-15)
    assert alpha[0] == pytest.approx(int(g["alpha_num"][0]) / math.sqrt(int(g["alpha_den_sq"][0])), rel=1e-15)
    qz = R.quantize(q - c)
    assert list(qz["qu"][0]) == [int(v) for v in g["qu"]]
    assert qz["sq"][0] == int(g["sq"][0])
    assert R.ip_planes(codes, qz["planes"][0])[0] == int(g["ip"][0])
    assert qz["nq2"][0] == int(g["nq2"][0])
    r2, f = R.scan_factors(r.astype(F32), alpha.astype(F32), dp)
    assert f[0] == pytest.approx(int(g["f_num"][0]) / int(g["f_den"][0]), rel=1e-6)
    d2 = R.estimate(codes, r2, f, qz, dp, qi=0)[0]
    want = Fraction(int(g["d2_num"][0]), int(g["d2_den"][0]))
    assert d2 == pytest.approx(float(want), rel=1e-6)
    assert ((x - q) ** 2).sum() == int(g["exact"][0])


def test_t_form_matches_eq5_with_dequantised_query():
    # Eq. 4-5 evaluated directly in float64 from the dequantised residual must
    # match the float32 t-form up to float32 rounding.
    rng = np.random.default_rng(8)
    dp = 128
    P = R.random_orthogonal(4, dp)
    x = rng.standard_normal((400, dp)).astype(F32)
    c = (rng.standard_normal((1, dp)) * 0.5).astype(F32)
    q = rng.standard_normal((1, dp)).astype(F32)
    codes, r, alpha, z = R.encode(x, c, np.zeros(400, np.int64), P)
    r2, f = R.scan_factors(r.astype(F32), alpha.astype(F32), dp)
    res = R.rotate(q, P) - (c.astype(F64) @ P).astype(F32)
    qz = R.quantize(res)
    d2 = R.estimate(codes, r2, f, qz, dp, qi=0)
    zq = qz["qu"][0] * F64(qz["delta"][0]) + F64(qz["vl"][0])   # dequantised
    nq = math.sqrt(F64(qz["nq2"][0]))
    b = 2.0 * R.unpack_bits(codes, dp) - 1
    s_hat = (b @ (zq / nq)) / (math.sqrt(dp) * alpha)                # Eq. 4
    ref = F64(qz["nq2"][0]) + r ** 2 - 2 * nq * r * s_hat             # Eq. 5
    assert np.allclose(d2, ref, rtol=2e-5, atol=2e-5 * ref.mean())


def test_eq5_with_exact_inner_product_is_exact_distance():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((50, 16))
    q = rng.standard_normal(16)
    c = rng.standard_normal(16)
    ux = (x - c) / np.linalg.norm(x - c, axis=1, keepdims=True)
    uq = (q - c) / np.linalg.norm(q - c)
    d2 = (np.linalg.norm(q - c) ** 2 + np.linalg.norm(x - c, axis=1) ** 2
          - 2 * np.linalg.norm(q - c) * np.linalg.norm(x - c, axis=1) * (ux @ uq))
    assert np.allclose(d2, ((x - q) ** 2).sum(axis=1), rtol=1e-12)


def test_lut_tables_by_brute_force_order():
    """Each FastScan entry is the float32 sum of the residual entries of the
    entry's set bits, added in increasing bit order from 0 (checked one entry
    at a time), LSB-first like the codes."""
    rng = np.random.default_rng(41)
    res = (rng.standard_normal(128) * np.float32(1e3)).astype(F32)
    res[::7] *= np.float32(1e-6)                     # mixed magnitudes: order matters
    T = R.lut_tables(res)
    assert T.shape == (16, 256)
    for g in (0, 5, 15):
        for v in range(256):
            acc = np.float32(0)
            for i in range(8):
                if (v >> i) & 1:
                    acc = np.float32(acc + res[8 * g + i])
            assert T[g, v] == acc, (g, v)
    # the byte of a code addresses its own group: one set bit picks one entry
    code = np.zeros((1, 16), np.uint8)
    code[0, 3] = 1 << 5
    assert R.lut_tables(res)[3, code[0, 3]] == res[8 * 3 + 5]


def test_lut_estimator_is_eq4_with_full_precision_query():
    """The FastScan form evaluates Eq. 4 with the unquantised residual: on
    integer-valued residuals (every float32 sum exact) t = sum_d b_d res_d
    exactly and d2 equals the t-form evaluated in float64 then rounded by the
    same float32 steps; on real residuals t is within the float32 rounding of
    the float64 dot product; and the 4-bit quantised estimate differs from it
    by at most D_p delta / 2 in t (the per-dimension quantisation error)."""
    rng = np.random.default_rng(43)
    dp = 128
    codes = rng.integers(0, 256, (300, dp // 8)).astype(np.uint8)
    bits = R.unpack_bits(codes, dp).astype(np.int64)
    b = 2 * bits - 1
    r2 = rng.uniform(0.5, 2.0, 300).astype(F32)
    f = rng.uniform(0.01, 0.2, 300).astype(F32)
    res_i = rng.integers(-20, 21, dp).astype(F32)
    d = R.estimate_lut(codes, r2, f, res_i)
    t = (b * res_i.astype(np.int64)).sum(axis=1)
    nq2 = np.float32((res_i.astype(np.int64) ** 2).sum())
    ref = (nq2 + r2) - np.float32(2) * (f * t.astype(F32))
    assert np.array_equal(d, (ref + np.float32(0)).astype(F32))
    res = rng.standard_normal(dp).astype(F32)
    T = R.lut_tables(res)
    s = np.zeros(300, F32)
    for g in range(dp // 8):
        s = s + T[g][codes[:, g]]
    t32 = np.float32(2) * s - R.lane_sum(res)
    t64 = (b * res.astype(F64)).sum(axis=1)
    assert np.all(np.abs(t32 - t64) <= 3 * dp * 2.0 ** -24 * np.abs(res).sum())
    qz = R.quantize(res[None, :])
    ip = R.ip_planes(codes, qz["planes"][0])
    pc = R.popcount8(codes)
    tq = qz["delta"][0] * (2 * ip - qz["sq"][0]).astype(F64) + qz["vl"][0] * (2 * pc - dp)
    assert np.all(np.abs(tq - t64) <= dp * qz["delta"][0] / 2 + 1e-4)


def test_lut_search_limit_is_exact_knn(tiny):
    """With every list probed and every candidate re-ranked the FastScan
    search is the exact kNN; with the tiny workload's settings its recall is
    at least the 4-bit form's."""
    x, q, ix = tiny
    ti, td = R.exact_knn(x, q, 10)
    ids, dist = R.search(ix, q, 32, 10, x.shape[0], estimator="lut")
    assert np.array_equal(ids, ti)
    a, _ = R.search(ix, q, 4, 10, 40, estimator="lut")
    b4, _ = R.search(ix, q, 4, 10, 40)
    assert R.recall_at(x, q, a, td, 10) >= R.recall_at(x, q, b4, td, 10) - 0.02


def test_estimator_unbiased_over_rotations():
    # E_P[s_hat] = <u_x, u_q> for Haar P (the RaBitQ estimator property).
    rng = np.random.default_rng(10)
    d, n = 16, 20000
    ux = rng.standard_normal(d); ux /= np.linalg.norm(ux)
    uq = rng.standard_normal(d); uq = uq - 0.6 * ux; uq /= np.linalg.norm(uq)
    G = rng.standard_normal((n, d, d))
    Q, Rr = np.linalg.qr(G)
    s = np.sign(np.einsum("nii->ni", Rr))
    P = Q * s[:, None, :]
    zx = np.einsum("nij,i->nj", P, ux)
    zq = np.einsum("nij,i->nj", P, uq)
    alpha = np.abs(zx).sum(1) / math.sqrt(d)
    b = np.where(zx >= 0, 1.0, -1.0)
    s_hat = (b * zq).sum(1) / (math.sqrt(d) * alpha)
    diff = s_hat - ux @ uq
    assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(n)


# ---------------------------------------------------------------- search
@pytest.fixture(scope="module")
def tiny():
    mix = W.mixture("tiny")
    x = mix.base(4000)
    q = mix.queries(40)
    ix = R.build_index(x, 32, seed=0, iters=6)
    return x, q, ix


def test_probe_all_lists_and_fp64_order(tiny):
    x, q, ix = tiny
    qr = R.rotate(q, ix["P"])
    ids, d = R.probe(qr, ix["cR"], 32)
    assert all(sorted(r) == list(range(32)) for r in ids.tolist())
    ex = ((q.astype(F64)[:, None] - ix["centroids"].astype(F64)[None]) ** 2).sum(-1)
    ref = np.argsort(ex, axis=1, kind="stable")
    gap_ok = np.diff(np.sort(ex, axis=1), axis=1).min(axis=1) > 1e-3 * ex.max()
    assert np.array_equal(ids[gap_ok], ref[gap_ok])


def test_probe_ties_go_to_lower_id():
    # duplicate centroids: equal distances, the lower id is taken first
    cR = np.array([[1.0, 0.0], [0.0, 0.0], [1.0, 0.0], [0.0, 0.0], [3.0, 0.0]], F32)
    ids, d = R.probe(np.zeros((1, 2), F32), cR, 4)
    assert list(ids[0]) == [1, 3, 0, 2] and list(d[0]) == [0.0, 0.0, 1.0, 1.0]


def test_prune_is_lossless_including_ties():
    rng = np.random.default_rng(12)
    d = rng.integers(0, 50, 5000).astype(F32)   # many exact ties
    ids = rng.permutation(5000)
    for n_sel in (1, 10, 200, 1024, 3000, 6000):
        a = R.select_candidates(d, ids, n_sel, prune=True)
        b = R.select_candidates(d, ids, n_sel, prune=False)
        assert np.array_equal(a, b)
        full = sorted(zip(d.tolist(), ids.tolist()))[:n_sel]
        assert [int(i) for i in R.key_id(a)] == [i for _, i in full]
    # distinct estimates, nearest first (the probe order puts the closest
    # lists first): the first candidates hold the n_sel smallest, so a bound
    # one rank too low would drop the n_sel-th
    d = np.arange(5000).astype(F32)
    for n_sel in (1, 2, 10, 1024, 1025, 3000):
        a = R.select_candidates(d, ids, n_sel, prune=True)
        assert np.array_equal(a, R.select_candidates(d, ids, n_sel, prune=False))
        assert np.array_equal(R.key_id(a), ids[:n_sel])


def test_first_bound_window_and_tightness():
    """The first bound looks at max(1024, n_sel, min(16 n_sel, 32768))
    candidates in probe order (values by hand), is the n_sel-th smallest of
    them exactly, never falls below the n_sel-th smallest of all candidates,
    and tightens as the window grows."""
    assert [R.bound_window(v) for v in (1, 10, 64, 100, 2000, 2048, 4096, 40000)] == \
        [1024, 1024, 1024, 1600, 32000, 32768, 32768, 40000]
    rng = np.random.default_rng(21)
    d = rng.standard_normal(50000).astype(F32)
    d[:5000] -= np.float32(1.0)            # the nearest lists come first
    for n_sel in (10, 100, 2000):
        m = R.bound_window(n_sel)
        dd = d.copy()
        dd[m - 1] = np.float32(-100.0)     # the window's last candidate is the best one
        tau = R.first_bound(dd, n_sel)
        assert tau == int(np.sort(R.orderable(dd[:m]))[n_sel - 1])
        assert tau < int(np.sort(R.orderable(dd[:m - 1]))[n_sel - 1])
        assert tau >= int(np.sort(R.orderable(dd))[n_sel - 1])
        looser = R.first_bound(dd, n_sel, window=max(1024, n_sel))
        assert looser >= tau
    assert R.first_bound(d[:5], 10) == R.U32_MAX


def test_running_bound_form_equals_first_bound_form():
    """Section 3.3.3 keeps a running bound (the largest of the current top
    n_sel) while candidates arrive in probe order; the search fixes one bound
    from the first candidates instead. Both schedules, and no pruning at
    all, select the same n_sel smallest (distance, id) keys, ties included;
    the running bound prunes a candidate only when it exceeds the held
    maximum."""
    rng = np.random.default_rng(31)
    for trial in range(6):
        m = int(rng.integers(1, 3000))
        if trial % 2:
            d = rng.integers(0, 40, m).astype(F32)          # many ties
        else:
            d = np.sort(rng.standard_normal(m).astype(F32))  # nearest first
            d += rng.standard_normal(m).astype(F32)
        ids = rng.permutation(m)
        for n_sel in (1, 7, 100, 1500):
            run, pruned = R.select_running_bound(d, ids, n_sel)
            assert np.array_equal(run, R.select_candidates(d, ids, n_sel, prune=True))
            assert np.array_equal(run, R.select_candidates(d, ids, n_sel, prune=False))
            assert 0 <= pruned <= max(0, m - n_sel)
    # by hand: keys arrive 5, 3, 9, 1, 9, 2 (ids 0..5); n_sel 2 holds {5, 3},
    # then 9 > 5 is pruned, 1 replaces 5, the second 9 > 3 is pruned, 2
    # replaces 3
    run, pruned = R.select_running_bound(np.array([5, 3, 9, 1, 9, 2], F32), np.arange(6), 2)
    assert R.key_id(run).tolist() == [3, 5] and pruned == 2


def test_rerank_matches_fp64_and_pads():
    rng = np.random.default_rng(13)
    raw = rng.integers(0, 256, (100, 128)).astype(F32)
    q = rng.integers(0, 256, 128).astype(F32)
    cand = rng.choice(100, 30, replace=False)
    oi, od = R.rerank(raw, q, cand, 10)
    ex = ((raw[cand].astype(F64) - q) ** 2).sum(1)
    ref = cand[np.lexsort((cand, ex))][:10]
    assert np.array_equal(oi, ref) and np.array_equal(od, np.sort(ex)[:10])
    oi, od = R.rerank(raw, q, cand[:3], 5)
    assert list(oi[3:]) == [-1, -1] and np.isinf(od[3:]).all()


def test_search_limit_is_exact_knn(tiny):
    x, q, ix = tiny
    ti, td = R.exact_knn(x, q, 10)
    ids, dist = R.search(ix, q, 32, 10, x.shape[0])
    assert np.array_equal(ids, ti)
    assert np.allclose(dist, td, rtol=1e-5)


def test_exact_knn_brute_force():
    rng = np.random.default_rng(14)
    x = rng.integers(0, 4, (200, 8)).astype(F32)   # heavy ties
    q = rng.integers(0, 4, (5, 8)).astype(F32)
    ids, dist = R.exact_knn(x, q, 7)
    for i in range(5):
        d = ((x.astype(F64) - q[i]) ** 2).sum(1)
        ref = sorted(range(200), key=lambda j: (d[j], j))[:7]
        assert list(ids[i]) == ref


def test_exact_dist_and_recall_by_hand():
    """Tie-aware recall@k worked by hand. Query 0 at 0 against rows
    0, 1, 2, 2, 3, 5 has squared distances 0, 1, 4, 4, 9, 25: its true top 3
    are rows 0, 1, 2 and the 3rd true distance is 4, which row 3 ties.
    Query 1 at 5: distances 25, 16, 9, 9, 4, 0, 3rd true distance 9."""
    x = np.array([[0.0], [1.0], [2.0], [2.0], [3.0], [5.0]], F32)
    q = np.array([[0.0], [5.0]], F32)
    ti, td = R.exact_knn(x, q, 3)
    assert ti.tolist() == [[0, 1, 2], [5, 4, 2]] and td[:, 2].tolist() == [4.0, 9.0]
    d = R.exact_dist(x, q, np.array([[0, 1, 2, -1], [5, 4, 3, 0]]))
    assert d[0, :3].tolist() == [0.0, 1.0, 4.0] and np.isnan(d[0, 3])
    assert d[1].tolist() == [0.0, 4.0, 9.0, 25.0]
    cases = [
        ([[0, 1, 3], [5, 4, 3]], 1.0),      # row 3 ties the 3rd distance: a hit
        ([[3, 2, 1], [5, 4, 2]], 1.0),      # at the 3rd distance counts (<=, not <)
        ([[0, 1, 4], [5, 4, 2]], 5 / 6),    # row 4 (9 > 4) misses
        ([[0, -1, 2], [5, 4, 2]], 5 / 6),   # a padded id misses
        ([[0, 1, 2], [5, 4, 0]], 5 / 6),    # row 0 for query 1 (25 > 9) misses
        ([[-1, -1, -1], [-1, -1, -1]], 0.0),
    ]
    for ids, want in cases:
        assert R.recall_at(x, q, np.array(ids), td, 3) == pytest.approx(want), ids


def test_recall_target_on_tiny_workload():
    wl = W.WORKLOADS["tiny"]
    x = wl["mix"].base(wl["n"])
    q = wl["mix"].queries(wl["nq"])
    ix = R.build_index(x, wl["nlist"], seed=0, iters=wl["iters"])
    _, td = R.exact_knn(x, q, 10)
    ids, _ = R.search(ix, q, wl["nprobe"], wl["k"], wl["n_rerank"])
    assert R.recall_at(x, q, ids, td, 10) >= 0.95


def test_per_query_params_and_no_rerank(tiny):
    x, q, ix = tiny
    npb = np.array([1, 4, 32, 2] * 10)
    kk = np.array([1, 10, 5, 3] * 10)
    ids, dist = R.search(ix, q, npb, kk, 50)
    for i in range(8):
        one, _ = R.search(ix, q[i:i + 1], int(npb[i]), int(kk[i]), 50)
        assert np.array_equal(ids[i, :kk[i]], one[0])
    ids0, d0 = R.search(ix, q[:4], 4, 5, 0)
    assert np.all(np.diff(d0, axis=1) >= 0)


def _fma32(x, y, z):
    """float32 fused multiply-add, correctly rounded: the product is exact in
    float64 and the sum's float64 rounding error is recovered (TwoSum) to
    break float32 rounding ties the right way."""
    x, y, z = (np.asarray(v, np.float64) for v in (x, y, z))
    p = x * y                      # exact: 24 + 24 bits
    s = p + z
    bp = s - z
    e = (p - bp) + (z - (s - bp))  # s + e == p + z exactly
    r = s.astype(np.float32)
    back = r.astype(np.float64)
    # where s is a float32 midpoint, the sign of e decides the rounding
    up = np.nextafter(r, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(r, np.float32(-np.inf)).astype(np.float64)
    tie_hi = (s - back) == (up - back) / 2
    tie_lo = (back - s) == (back - dn) / 2
    r = np.where(tie_hi & (e > 0), np.float32(up), r)
    r = np.where(tie_lo & (e < 0), np.float32(dn), r)
    return r.astype(np.float32)


def test_certified_probe_filter_bound():
    """The centroid filter of the search keeps c unless its approximate
    distance a = ||q||^2 + (||c||^2 - 2 <q, c>), computed in float32 with
    fused multiply-adds in any order, is more than
    e = 16 D_p 2^-24 (||q||^2 + ||c||^2) above a smaller bound; that needs
    |a - exact| <= e, exact being the fixed-order float32 distance. Checked
    with sequential and reversed FMA orders on random rows, rows almost equal
    to the query (cancellation) and large, mixed-sign magnitudes."""
    rng = np.random.default_rng(17)
    dp = 128
    esc = np.float32(16.0 * dp * 2.0 ** -24)
    cases = []
    q = rng.normal(0, 1, (8, dp)).astype(np.float32)
    cases.append((q, rng.normal(0, 1, (64, dp)).astype(np.float32)))
    cases.append((q, (q[:1] + rng.normal(0, 1e-3, (64, dp))).astype(np.float32)))
    big = (rng.normal(0, 1, (8, dp)) * 1e6).astype(np.float32)
    cases.append((big, (big[:1] * rng.uniform(0.999, 1.001, (64, dp))).astype(np.float32)))
    cases.append((q * 300, rng.normal(0, 300, (64, dp)).astype(np.float32)))
    for qq, cc in cases:
        exact = R.seq_sqdist(qq, cc)
        for order in (range(dp), range(dp - 1, -1, -1)):
            qn = np.zeros(qq.shape[0], np.float32)
            cn = np.zeros(cc.shape[0], np.float32)
            dot = np.zeros((qq.shape[0], cc.shape[0]), np.float32)
            for d in order:
                qn = _fma32(qq[:, d], qq[:, d], qn)
                cn = _fma32(cc[:, d], cc[:, d], cn)
                dot = _fma32(qq[:, d, None], cc[None, :, d], dot)
            g = _fma32(np.float32(-2.0), dot, cn[None, :])
            a = (qn[:, None] + g).astype(np.float32)
            e = esc * (qn[:, None] + cn[None, :])
            gap = np.abs(a.astype(np.float64) - exact.astype(np.float64))
            assert np.all(gap <= e), (gap / e).max()


def _tf32(x):
    """float32 values with the low 13 mantissa bits dropped (what the tensor
    core's TF32 operands keep)."""
    return (np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _add32(a, b, mode):
    """float32 addition, rounded to nearest (numpy) or toward zero."""
    if mode == "rn":
        return (a + b).astype(np.float32)
    s = a.astype(np.float64) + b.astype(np.float64)
    r = s.astype(np.float32)
    over = np.abs(r.astype(np.float64)) > np.abs(s)
    return np.where(over, np.nextafter(r, np.float32(0.0)), r).astype(np.float32)


def test_tensor_core_probe_filter_bound():
    """The certified centroid filter with the tensor-core ranking: inner
    products of TF32-truncated inputs (products exact in float32), summed in
    float32 in groups of 8 then across groups, in either direction, rounded
    to nearest or toward zero; g = fma(-2, dot, ||c||^2) and
    a = ||q||^2 + g in float32. |a - exact| must stay within
    2^-8 (||q||^2 + ||c||^2), exact being the fixed-order float32 distance."""
    rng = np.random.default_rng(23)
    dp = 128
    esc = np.float32(2.0 ** -8)
    q = rng.normal(0, 1, (8, dp)).astype(np.float32)
    cases = [(q, rng.normal(0, 1, (64, dp)).astype(np.float32)),
             (q, (q[:1] + rng.normal(0, 1e-3, (64, dp))).astype(np.float32))]
    big = (rng.normal(0, 1, (8, dp)) * 1e6).astype(np.float32)
    cases.append((big, (big[:1] * rng.uniform(0.999, 1.001, (64, dp))).astype(np.float32)))
    cases.append((q * 300, rng.normal(0, 300, (64, dp)).astype(np.float32)))
    unit = rng.normal(0, 1, (8, dp)).astype(np.float32)
    unit /= np.linalg.norm(unit, axis=1, keepdims=True)
    cases.append((unit, (unit[:1] + rng.normal(0, 0.05, (64, dp))).astype(np.float32)))
    worst = 0.0
    for qq, cc in cases:
        exact = R.seq_sqdist(qq, cc)
        qt, ct = _tf32(qq), _tf32(cc)
        prod = (qt[:, None, :].astype(np.float64) * ct[None, :, :].astype(np.float64)).astype(np.float32)
        for mode in ("rn", "rz"):
            for rev in (False, True):
                order = list(range(dp))[::-1] if rev else list(range(dp))
                dot = np.zeros((qq.shape[0], cc.shape[0]), np.float32)
                for g0 in range(0, dp, 8):
                    part = np.zeros_like(dot)
                    for d in order[g0:g0 + 8]:
                        part = _add32(part, prod[:, :, d], mode)
                    dot = _add32(dot, part, mode)
                qn = np.zeros(qq.shape[0], np.float32)
                cn = np.zeros(cc.shape[0], np.float32)
                for d in order:
                    qn = _fma32(qq[:, d], qq[:, d], qn)
                    cn = _fma32(cc[:, d], cc[:, d], cn)
                g = _fma32(np.float32(-2.0), dot, cn[None, :])
                a = (qn[:, None] + g).astype(np.float32)
                e = esc * (qn[:, None] + cn[None, :])
                gap = np.abs(a.astype(np.float64) - exact.astype(np.float64))
                assert np.all(gap <= e), (gap / e).max()
                worst = max(worst, float((gap / e).max()))
    assert worst > 0.01  # the truncation does show: the bound is not vacuous


def test_fma32_helper_is_correctly_rounded():
    """The helper of the bound pin: against exact rationals on random and
    tie-making inputs."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, 300).astype(np.float32)
    y = rng.normal(0, 1, 300).astype(np.float32)
    z = rng.normal(0, 1e-3, 300).astype(np.float32)
    # ties: z chosen so that x*y + z lands halfway between two float32 values
    x[:20] = np.float32(1.0) + np.float32(2.0 ** -23)
    y[:20] = np.float32(1.0) + np.float32(2.0 ** -23)
    z[:20] = np.float32(0.0)
    r = _fma32(x, y, z)
    for i in range(300):
        ex = Fraction(float(x[i])) * Fraction(float(y[i])) + Fraction(float(z[i]))
        cands = [np.float32(float(ex)), np.nextafter(np.float32(float(ex)), np.float32(np.inf)),
                 np.nextafter(np.float32(float(ex)), np.float32(-np.inf))]
        best = min(cands, key=lambda c: (abs(Fraction(float(c)) - ex),
                                         int(np.float32(c).view(np.uint32)) & 1))
        assert r[i] == best, (i, r[i], best)
