"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of an oracle function's source (a
dropped term, a wrong sign, a transposed operand, a wrong index, tie or
rounding rule), swaps the copy into the oracle module for the duration of
the case, and runs the pins that should notice. A case passes when at least
one of those pins fails under the mutant. CPU only; nothing here touches the
CUDA path.
"""
import inspect
import textwrap

import pytest

import workloads as W
from oracle import philox, rabitq as R
from tests import test_oracle_pins as P


def _mutant(module, name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, f"{name}: pattern must occur exactly once"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), ns)
    return ns[name]


def _tiny():
    mix = W.mixture("tiny")
    x = mix.base(4000)
    q = mix.queries(40)
    return x, q, R.build_index(x, 32, seed=0, iters=6)


def _fails(pin):
    params = inspect.signature(pin).parameters
    args = []
    for p in params:
        if p == "tiny":
            args.append(_tiny())
        elif p == "dp":
            args.append(128)
        else:
            raise AssertionError(f"no value for {p}")
    try:
        pin(*args)
    except Exception:
        return True
    return False


EST = [P.test_estimator_worked_example_by_hand, P.test_t_form_matches_eq5_with_dequantised_query]

# (module, function, text, replacement, pins that must notice)
CASES = {
    # estimator (Eqs. 4-5, t-form)
    "estimate: vl term dropped": (R, "estimate", 't = g("delta") * a + g("vl") * b', 't = g("delta") * a', EST),
    "estimate: sign of the cross term": (R, "estimate", "- F32(2) * (", "+ F32(2) * (", EST),
    "estimate: sign of Sq": (R, "estimate", '(2 * ip - g("sq"))', '(2 * ip + g("sq"))', EST),
    "estimate: r^2 dropped": (R, "estimate", '(g("nq2") + np.asarray(r2, F32))', '(g("nq2") + F32(0))', EST),
    "estimate: D_p instead of 2 pc - D_p": (R, "estimate", "(2 * pc - dp)", "(pc - dp)", EST),
    "ip_planes: plane weight j + 1": (R, "ip_planes", "(1 << j)", "(j + 1)",
                                      [P.test_integer_estimator_forms_agree_exactly] + EST),
    "scan_factors: sqrt(D_p) dropped": (R, "scan_factors", "r32 / (sq * alpha32)", "r32 / alpha32", EST),
    # FastScan form (unquantised query)
    "lut_tables: most significant bit first": (R, "lut_tables", "acc = acc + res[i::8]",
                                               "acc = acc + res[7 - i::8]",
                                               [P.test_lut_tables_by_brute_force_order]),
    "estimate_lut: s instead of 2 s": (R, "estimate_lut", "t = F32(2) * s - lane_sum(res)",
                                       "t = s - lane_sum(res)",
                                       [P.test_lut_estimator_is_eq4_with_full_precision_query]),
    "estimate_lut: sum of the residual dropped": (R, "estimate_lut", "t = F32(2) * s - lane_sum(res)",
                                                  "t = F32(2) * s",
                                                  [P.test_lut_estimator_is_eq4_with_full_precision_query]),
    # query quantisation
    "quantize: rounds down": (R, "quantize", "* inv[..., None] + F32(0.5)", "* inv[..., None]",
                              [P.test_quantize_error_bound_and_degenerate] + EST),
    "quantize: 16 levels": (R, "quantize", "width / F32(QMAX)", "width / F32(16)",
                            [P.test_quantize_error_bound_and_degenerate] + EST),
    "quantize: norm without the square": (R, "quantize", "nq2 = lane_sum(res * res)", "nq2 = lane_sum(np.abs(res))",
                                          [P.test_quantize_error_bound_and_degenerate] + EST),
    # rotation and encode (Eqs. 1-3)
    "random_orthogonal: sign fix dropped": (R, "random_orthogonal", "return q * s[None, :]", "return q",
                                            [P.test_rotation_is_signed_qr_of_gaussian]),
    "random_orthogonal: transposed": (R, "random_orthogonal", "return q * s[None, :]", "return (q * s[None, :]).T",
                                      [P.test_rotation_is_signed_qr_of_gaussian]),
    "_encode_rows: every row against the first centroid": (
        R, "_encode_rows", "np.arange(x.shape[0])", "np.zeros(x.shape[0], np.int64)",
        [P.test_build_layout_and_chunked_encode]),
    "build_index: lists in descending row order": (
        R, "build_index", "np.lexsort((np.arange(n), a))", "np.lexsort((-np.arange(n), a))",
        [P.test_build_layout_and_chunked_encode]),
    "encode: P instead of P^T": (R, "encode", "z = pad(u, dp) @ P", "z = pad(u, dp) @ P.T",
                                 [P.test_alpha_identity_and_codes]),
    "encode: sign(0) -> 0 bit": (R, "encode", "bits = z >= 0", "bits = z > 0",
                                 [P.test_alpha_identity_and_codes, P.test_alpha_mean_and_zero_residual]),
    "encode: alpha without sqrt(D_p)": (R, "encode", "(np.sqrt(F64(dp)) * np.where(r > 0, r, 1.0))",
                                        "np.where(r > 0, r, 1.0)", [P.test_alpha_identity_and_codes]),
    "pack_bits: most significant bit first": (R, "pack_bits", 'bitorder="little"', 'bitorder="big"',
                                              [P.test_estimator_worked_example_by_hand]),
    "rotate: P instead of P^T": (R, "rotate", "@ P).astype(F32)", "@ P.T).astype(F32)",
                                 [P.test_probe_all_lists_and_fp64_order]),
    # fixed-order sums
    "lane_sum: adjacent lanes paired": (R, "lane_sum", "acc = acc[..., :s] + acc[..., s:2 * s]",
                                        "acc = acc[..., 0:2 * s:2] + acc[..., 1:2 * s:2]",
                                        [P.test_lane_sum_order_by_hand]),
    "seq_sqdist: reversed order": (R, "seq_sqdist", "for d in range(a.shape[1]):",
                                   "for d in reversed(range(a.shape[1])):", [P.test_seq_sqdist_order_by_hand]),
    # k-means
    "assign: ties to the higher id": (R, "assign", "a[i:i + chunk] = np.argmin(d, axis=1)",
                                      "a[i:i + chunk] = d.shape[1] - 1 - np.argmin(d[:, ::-1], axis=1)",
                                      [P.test_update_is_mean_and_reseeds_empty]),
    "update: mean over count + 1": (R, "update", "(s / F64(counts[j]))", "(s / F64(counts[j] + 1))",
                                    [P.test_update_is_mean_and_reseeds_empty]),
    "update: reseed from the nearest member": (R, "update", "far = mem[int(np.argmax(dd))]",
                                               "far = mem[int(np.argmin(dd))]",
                                               [P.test_update_is_mean_and_reseeds_empty]),
    "sqdist_f64: sign of the cross term": (R, "sqdist_f64", "- 2.0 * (a @ b.T)", "+ 2.0 * (a @ b.T)",
                                           [P.test_float64_assignment_is_nearest_exactly]),
    "assign_f64: ties to the higher id": (R, "_nearest_f64", "a = np.argmin(d, axis=1)",
                                          "a = d.shape[1] - 1 - np.argmin(d[:, ::-1], axis=1)",
                                          [P.test_float64_assignment_is_nearest_exactly]),
    "kmeans_init: largest keys": (R, "kmeans_init", "rows[np.argsort(keys)[:nlist]]",
                                  "rows[np.argsort(keys)[::-1][:nlist]]", [P.test_kmeans_init_is_smallest_keys]),
    "train_rows: largest keys": (R, "train_rows", "np.argsort(keys)[:n_train]",
                                 "np.argsort(keys)[::-1][:n_train]", [P.test_train_rows_are_smallest_keys]),
    "train_rows: k-means init stream": (R, "train_rows", "philox.STREAM_TRAIN_SAMPLE",
                                        "philox.STREAM_KMEANS_INIT", [P.test_train_rows_are_smallest_keys]),
    # ground truth and recall
    "recall_at: strict comparison": (R, "recall_at", "<= kth * (1 + 1e-12)", "< kth * (1 - 1e-12)",
                                     [P.test_exact_dist_and_recall_by_hand]),
    "recall_at: padded ids count as hits": (R, "recall_at", "nan=np.inf", "nan=0.0",
                                            [P.test_exact_dist_and_recall_by_hand]),
    "recall_at: first true distance": (R, "recall_at", "true_dist[:, k - 1]", "true_dist[:, 0]",
                                          [P.test_exact_dist_and_recall_by_hand]),
    "exact_dist: absolute instead of squared": (R, "exact_dist", "(diff * diff).sum(axis=1)",
                                                "np.abs(diff).sum(axis=1)",
                                                [P.test_exact_dist_and_recall_by_hand]),
    # keys, probe, pruning, selection, re-rank
    "orderable: negatives not inverted": (R, "orderable", "np.where(neg, u ^ np.uint64(0xFFFFFFFF)",
                                          "np.where(neg, u ^ np.uint64(0x80000000)",
                                          [P.test_orderable_is_monotone_and_invertible]),
    "probe: ties by descending id": (R, "probe", "keys = np.sort(make_keys(dist[i], ids))[:nprobe]",
                                     "keys = np.sort(make_keys(dist[i], ids[::-1]))[:nprobe]",
                                     [P.test_probe_ties_go_to_lower_id]),
    "select_candidates: strict bound": (R, "select_candidates", "orderable(d2) <= np.uint64(tau)",
                                        "orderable(d2) < np.uint64(tau)",
                                        [P.test_prune_is_lossless_including_ties]),
    "first_bound: one rank early": (R, "first_bound", "[n_sel - 1])", "[max(0, n_sel - 2)])",
                                    [P.test_prune_is_lossless_including_ties]),
    "bound_window: no 16 n_sel term": (R, "bound_window", "min(BOUND_FACTOR * n_sel, BOUND_MAX)",
                                       "BOUND_MIN", [P.test_first_bound_window_and_tightness]),
    "first_bound: window one short": (R, "first_bound", "bound_window(n_sel) if window is None else window",
                                      "bound_window(n_sel) - 1 if window is None else window",
                                      [P.test_first_bound_window_and_tightness]),
    "select_running_bound: bound is the held minimum": (R, "select_running_bound", "top = max(held)",
                                                        "top = min(held)",
                                                  [P.test_running_bound_form_equals_first_bound_form]),
    "select_running_bound: keeps the maximum": (R, "select_running_bound", "held.remove(top)",
                                                "held.remove(min(held))",
                                                [P.test_running_bound_form_equals_first_bound_form]),
    "rerank: absolute instead of squared": (R, "rerank", "d = lane_sum(diff * diff)", "d = lane_sum(np.abs(diff))",
                                            [P.test_rerank_matches_fp64_and_pads]),
    "list_candidates: residual sign": (R, "list_candidates", 'res = (qrot_i - index["cR"][c])',
                                       'res = (index["cR"][c] - qrot_i)',
                                       [P.test_recall_target_on_tiny_workload]),
    "search: selects k instead of n_rerank": (R, "search", "n_sel = int(nrr[i]) if nrr[i] > 0 else int(kk[i])",
                                              "n_sel = int(kk[i])", [P.test_search_limit_is_exact_knn]),
    "exact_knn: ties by descending id": (R, "exact_knn", "o = np.lexsort((cand, dd))[:k]",
                                         "o = np.lexsort((-cand, dd))[:k]", [P.test_exact_knn_brute_force]),
    # Philox
    "philox: nine rounds": (philox, "philox4x32_10", "for _ in range(10):", "for _ in range(9):",
                            [P.test_philox_known_answers]),
    "philox: Weyl constant": (philox, "philox4x32_10", "k1 = (k1 + W1) & MASK32", "k1 = (k1 + W0) & MASK32",
                              [P.test_philox_known_answers]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pins_catch_planted_mistake(case, monkeypatch):
    module, name, old, new, pins = CASES[case]
    for pin in pins:              # the unmutated oracle passes these pins
        assert not _fails(pin), f"{pin.__name__} fails without the mutation"
    monkeypatch.setattr(module, name, _mutant(module, name, old, new))
    caught = [pin.__name__ for pin in pins if _fails(pin)]
    assert caught, f"no pin noticed: {case}"
