"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle -- a dropped term, a wrong sign,
index or normalisation, a swapped case, a missing tie rule -- by replacing
one of its functions for the duration of the case (CPU only), then runs the
pins that should notice it and requires at least one of them to fail.  A
mistake that no pin notices would leave that part of the oracle unpinned."""
import math

import numpy as np
import pytest

import test_oracle_knn as pk
import test_oracle_mlp as pm
import test_oracle_sfa as ps
from oracle import sofa_oracle as orc

ORIG = {name: getattr(orc, name) for name in
        ("znorm", "dft", "dft_values", "selected_values", "weight", "value_table", "sample_stride",
         "select_values", "learn_bins", "learn_summary", "symbols", "mind", "lb2", "sqdist", "tie_order", "knn",
         "gemini_knn", "mlp_forward", "gelu", "softmax_xent", "mlp_loss_grad", "adam_step")}


# ------------------------------------------------------------------ the mistakes
def znorm_sample_sigma(x):
    z, mu, sg = ORIG["znorm"](x)
    n = np.asarray(x).shape[1]
    f = math.sqrt(n / (n - 1.0))
    return (z * np.float32(f)).astype(np.float32), mu, sg / f


def dft_unnormalised(z):
    re, im = ORIG["dft"](z)
    s = math.sqrt(np.asarray(z).shape[1])
    return re * s, im * s


def dft_imag_sign(z):
    re, im = ORIG["dft"](z)
    return re, -im


def dft_index_shift(z):
    re, im = ORIG["dft"](z)
    return np.roll(re, -1, axis=1), np.roll(im, -1, axis=1)


def weight_nyquist_two(n, k):
    return 2.0


def weight_all_one(n, k):
    return 1.0


def value_table_keeps_nyquist_imag(n, pool=0):
    K = n // 2 if pool <= 0 else min(pool, n // 2)
    return [(k, p) for k in range(1, K + 1) for p in (0, 1)]


def bins_equi_depth_off_by_one(v, alpha, mode="equi-depth"):
    if mode != "equi-depth":
        return ORIG["learn_bins"](v, alpha, mode)
    sv = np.sort(v, kind="stable")
    S = v.shape[0]
    beta = np.empty(alpha + 1, np.float64)
    beta[0], beta[alpha] = -np.inf, np.inf
    for a in range(1, alpha):
        beta[a] = sv[min(S - 1, (a * S) // alpha + 1)]
    return beta.astype(np.float32)


def bins_equi_width_alpha_minus_one(v, alpha, mode="equi-depth"):
    if mode != "equi-width":
        return ORIG["learn_bins"](v, alpha, mode)
    lo, hi = float(np.min(v)), float(np.max(v))
    beta = np.empty(alpha + 1, np.float64)
    beta[0], beta[alpha] = -np.inf, np.inf
    for a in range(1, alpha):
        beta[a] = lo + a * (hi - lo) / (alpha - 1)
    return beta.astype(np.float32)


def symbols_breakpoint_goes_down(v, beta_j):
    return np.searchsorted(beta_j[1:-1].astype(np.float64), v, side="left").astype(np.uint8)


def mind_below_to_upper_edge(b, lo, hi):
    b, lo, hi = (np.asarray(a, np.float64) for a in (b, lo, hi))
    return np.where(b < lo, hi - b, np.where(b > hi, b - hi, 0.0))


def lb2_without_weights(qv, wds, summ):
    s = dict(summ)
    s["w"] = np.ones_like(np.asarray(summ["w"], np.float64))
    return ORIG["lb2"](qv, wds, s)


def _select_variant(vals, n, l, mode, pool, tie_sign, move_nyquist):
    """select_values with its tie rule or its Nyquist move changed."""
    tab = orc.value_table(n, pool)
    var = ((vals - vals.mean(axis=0)) ** 2).mean(axis=0)
    ids = np.arange(len(tab))
    order = list(np.lexsort((tie_sign * ids, -var))) if mode == "variance" else list(ids)
    m = min(2 * l, len(tab))
    top = order[:m]
    word = top[:l]
    nyq = [c for c in word if 2 * tab[c][0] == n] if move_nyquist else []
    word = nyq + [c for c in word if c not in nyq]
    chosen = word + top[l:m]
    ks = np.array([tab[c][0] for c in chosen], np.int32)
    return dict(ids=np.array(chosen, np.int32), ks=ks, parts=np.array([tab[c][1] for c in chosen], np.int32),
                w=np.array([orc.weight(n, int(k)) for k in ks]), var=var[chosen], all_var=var)


def select_ties_by_descending_id(vals, n, l, mode="variance", pool=0):
    return _select_variant(vals, n, l, mode, pool, -1, True)


def select_nyquist_not_moved(vals, n, l, mode="variance", pool=0):
    return _select_variant(vals, n, l, mode, pool, 1, False)


def select_lowest_variance_first(vals, n, l, mode="variance", pool=0):
    # each column scaled to variance 1/var: the ranking turns upside down
    return ORIG["select_values"]((vals - vals.mean(axis=0)) / np.maximum(vals.var(axis=0), 1e-300), n, l, mode, pool)


def stride_floor(ratio):
    return max(1, int(math.floor(1.0 / ratio)))


def tie_order_no_runs(d2, ids):
    d = np.sqrt(d2)
    o = np.lexsort((ids, d))
    return ids[o].astype(np.int64), d[o]


def tie_order_wide_window(d2, ids):
    d = np.sqrt(d2)
    o = np.lexsort((ids, d))
    d, ids = d[o], ids[o]
    out_i, out_d, i = [], [], 0
    while i < len(d):
        j = i
        while j + 1 < len(d) and d[j + 1] <= d[i] * (1 + 1e-5):
            j += 1
        seg = np.argsort(ids[i:j + 1], kind="stable")
        out_i.extend(ids[i:j + 1][seg])
        out_d.extend(d[i:j + 1][seg])
        i = j + 1
    return np.array(out_i, np.int64), np.array(out_d)


def sqdist_drops_last_value(Z, zq):
    return ORIG["sqdist"](np.ascontiguousarray(np.asarray(Z)[:, :-1]), np.ascontiguousarray(np.asarray(zq)[:-1]))


def knn_window_not_widened(Z, Zq, k):
    idx = np.empty((Zq.shape[0], k), np.int64)
    dist = np.empty((Zq.shape[0], k), np.float64)
    for q in range(Zq.shape[0]):
        d2 = orc.sqdist(Z, Zq[q])
        d = np.sqrt(d2)
        keep = np.nonzero(d <= np.partition(d, k - 1)[k - 1])[0]
        oi, od = orc.tie_order(d2[keep], keep.astype(np.int64))
        idx[q], dist[q] = oi[:k], od[:k]
    return idx, dist


def gemini_stop_without_tie_window(Z, W, Zq, summ, k):
    idx = np.empty((Zq.shape[0], k), np.int64)
    dist = np.empty((Zq.shape[0], k), np.float64)
    refined = np.zeros(Zq.shape[0], np.int64)
    qv_all = orc.selected_values(Zq, summ)
    for q in range(Zq.shape[0]):
        lb = orc.lb2(qv_all[q][: summ["l"]], W, summ)
        best_d2, best_i = [], []
        for i in np.argsort(lb, kind="stable"):
            if len(best_d2) >= k and math.sqrt(max(lb[i], 0.0)) > math.sqrt(sorted(best_d2)[k - 1]):
                break
            best_d2.append(float(orc.sqdist(Z[i:i + 1], Zq[q])[0]))
            best_i.append(int(i))
            refined[q] += 1
        oi, od = orc.tie_order(np.array(best_d2), np.array(best_i, np.int64))
        idx[q], dist[q] = oi[:k], od[:k]
    return idx, dist, refined


def summary_from_every_row(x, l, alpha, ratio=0.1, binning="equi-depth", select="variance", pool=0):
    return ORIG["learn_summary"](x, l, alpha, 1.0, binning, select, pool)


def summary_sample_shifted(x, l, alpha, ratio=0.1, binning="equi-depth", select="variance", pool=0):
    return ORIG["learn_summary"](x[1:], l, alpha, ratio, binning, select, pool)


def dft_values_parts_swapped(z, pool=0):
    re, im = orc.dft(z)
    tab = orc.value_table(np.asarray(z).shape[1], pool)
    return np.stack([im[:, k] if p == 0 else re[:, k] for k, p in tab], axis=1)


def selected_values_parts_swapped(z, summ):
    re, im = orc.dft(z)
    return np.stack([im[:, k] if p == 0 else re[:, k] for k, p in zip(summ["ks"], summ["parts"])], axis=1)


def lb2_interval_one_bin_down(qv, wds, summ):
    beta = summ["beta"].astype(np.float64)
    out = np.zeros(wds.shape[0], np.float64)
    for j in range(summ["l"]):
        s = wds[:, j].astype(np.int64)
        m = orc.mind(qv[j], beta[j][np.maximum(s - 1, 0)], beta[j][s])
        out += summ["w"][j] * m * m
    return out


def forward_w2_transposed(params, x):
    p = dict(params)
    p["W2"] = params["W2"].T
    return ORIG["mlp_forward"](p, x)


def gelu_tanh(x):
    return 0.5 * x * (1.0 + np.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))


def softmax_grad_not_mean(logits, y):
    loss, g = ORIG["softmax_xent"](logits, y)
    return loss, g * logits.shape[0]


def grads_drop_b1(params, x, y):
    loss, g = ORIG["mlp_loss_grad"](params, x, y)
    g = dict(g)
    g["b1"] = np.zeros_like(g["b1"])
    return loss, g


def adam_no_bias_correction(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    out = {}
    for key in params:
        m[key] = b1 * m[key] + (1 - b1) * grads[key]
        v[key] = b2 * v[key] + (1 - b2) * grads[key] ** 2
        out[key] = params[key] - lr * m[key] / (np.sqrt(v[key]) + eps)
    return out


# ------------------------------------------------------------------ cases
CASES = [
    ("population sigma replaced by sample sigma", {"znorm": znorm_sample_sigma},
     [ps.test_znorm_closed_form, ps.test_znorm_population_sigma_and_constant_row]),
    ("DFT without the n^-1/2 normalisation", {"dft": dft_unnormalised},
     [ps.test_dft_sinusoid_closed_form, lambda: ps.test_dft_matches_numpy_fft(8)]),
    ("DFT with the imaginary sign flipped", {"dft": dft_imag_sign},
     [ps.test_dft_sinusoid_closed_form, lambda: ps.test_dft_matches_numpy_fft(8)]),
    ("DFT coefficient index shifted by one", {"dft": dft_index_shift}, [ps.test_dft_sinusoid_closed_form]),
    ("Nyquist value weighted 2", {"weight": weight_nyquist_two},
     [lambda: ps.test_parseval_weights(8), ps.test_value_table]),
    ("every value weighted 1", {"weight": weight_all_one},
     [lambda: ps.test_parseval_weights(9), ps.test_full_pool_dft_lb_equals_ed]),
    ("Nyquist imaginary part kept as a candidate", {"value_table": value_table_keeps_nyquist_imag},
     [ps.test_value_table]),
    ("equi-depth breakpoint index off by one", {"learn_bins": bins_equi_depth_off_by_one},
     [lambda: ps.test_equi_depth_counts(1000, 4), lambda: ps.test_equi_depth_counts(300, 256)]),
    ("equi-width spacing over alpha - 1", {"learn_bins": bins_equi_width_alpha_minus_one},
     [ps.test_equi_width_spacing]),
    ("a value on a breakpoint goes down", {"symbols": symbols_breakpoint_goes_down},
     [ps.test_symbols_bruteforce]),
    ("below the bin measured to its upper edge", {"mind": mind_below_to_upper_edge}, [ps.test_mind_three_cases]),
    ("real and imaginary candidate values swapped", {"dft_values": dft_values_parts_swapped},
     [ps.test_full_pool_dft_lb_equals_ed, ps.test_selection_finds_planted_frequencies]),
    ("selected values read from the wrong part", {"selected_values": selected_values_parts_swapped},
     [ps.test_selected_values_closed_form, pk.test_gemini_refines_a_near_tie_beyond_the_kth]),
    ("bound taken against the bin below the symbol's", {"lb2": lb2_interval_one_bin_down},
     [ps.test_lb2_tiny_closed_form, lambda: ps.test_lb_le_dftlb_le_ed("rw", 256, "equi-depth")]),
    ("Eq. (1) weight dropped from the SFA bound", {"lb2": lb2_without_weights}, [ps.test_lb2_tiny_closed_form]),
    ("variance ties broken by descending id", {"select_values": select_ties_by_descending_id},
     [ps.test_selection_ties_and_nyquist_first]),
    ("selected Nyquist value not moved to word position 0", {"select_values": select_nyquist_not_moved},
     [ps.test_selection_ties_and_nyquist_first]),
    ("values ranked by inverse variance", {"select_values": select_lowest_variance_first},
     [ps.test_selection_finds_planted_frequencies]),
    ("sample stride rounded down", {"sample_stride": stride_floor}, [ps.test_sample_stride]),
    ("tie runs not reordered by index", {"tie_order": tie_order_no_runs},
     [pk.test_tie_window_is_one_millionth_relative, pk.test_run_is_anchored_at_first_element]),
    ("tie window 1e-5 instead of 1e-6", {"tie_order": tie_order_wide_window},
     [pk.test_tie_window_is_one_millionth_relative]),
    ("k-NN window not widened by the tie window", {"knn": knn_window_not_widened},
     [pk.test_window_keeps_a_near_tie_beyond_the_kth]),
    ("GEMINI stops without the tie window", {"gemini_knn": gemini_stop_without_tie_window},
     [pk.test_gemini_refines_a_near_tie_beyond_the_kth]),
    ("summary learned from every row instead of the sample", {"learn_summary": summary_from_every_row},
     [ps.test_learn_summary_uses_the_strided_sample]),
    ("summary sample shifted by one row", {"learn_summary": summary_sample_shifted},
     [ps.test_learn_summary_uses_the_strided_sample]),
    ("squared distance drops the last value", {"sqdist": sqdist_drops_last_value}, [pk.test_sqdist_matches_numpy]),
    ("middle layer applied transposed", {"mlp_forward": forward_w2_transposed},
     [pm.test_forward_orientation_closed_form, pm.test_finite_differences]),
    ("GELU by the tanh approximation", {"gelu": gelu_tanh}, [pm.test_gelu_closed_values]),
    ("cross-entropy gradient not averaged over the batch", {"softmax_xent": softmax_grad_not_mean},
     [pm.test_zero_weights_uniform_softmax, pm.test_finite_differences]),
    ("first-layer bias gradient dropped", {"mlp_loss_grad": grads_drop_b1}, [pm.test_finite_differences]),
    ("Adam without bias correction", {"adam_step": adam_no_bias_correction}, [pm.test_adam_first_step_is_lr_sign]),
]


@pytest.mark.parametrize("name,patch,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_the_planted_mistake(monkeypatch, name, patch, pins):
    for attr, fn in patch.items():
        monkeypatch.setattr(orc, attr, fn)
    caught = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught.append(pin)
    assert caught, f"no pin noticed: {name}"


def test_pins_pass_on_the_oracle_itself():
    """The same pins pass without a planted mistake (so a failure above is the
    mistake's doing)."""
    for _, _, pins in CASES:
        for pin in pins:
            pin()
