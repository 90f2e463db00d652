"""CPU oracle for SOFA's exact k-NN hot path (Schaefer et al., arXiv 2411.17483).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code,
table or constant with the CUDA library and never calls it.

Plain, slow FP64 restatements of the paper, each function citing its passage:

* z-normalisation / z-ED ........ Sec. II, Definition (z-ED)          -> C: orc_znorm
* DFT ........................... Alg. 1 step 1, Alg. 2 step 1, Eq. 1 -> C: orc_dft
* variance feature selection .... Sec. IV "Novel Feature Selection", Alg. 1 step 2
* MCB bins (equi-depth / width) . Sec. IV "Transformation and Learned Quantization", Alg. 1 step 3
* SFA words ..................... Alg. 2 step 2 (half-open bins [beta(a-1), beta(a)))
* SFA lower bound ............... Eq. 1, SFA LBD, Eq. dist_i
* exact k-NN, tie rule .......... Sec. II NN problem, k-NN extension (Sec. IV, Table III)
* GEMINI filter-and-refine ...... Sec. II-A
* proposal MLP (fwd / bwd) ...... not in the paper: a learned seed for the best-so-far

Readings where the paper is silent or ambiguous:
population sigma; Z rounded to fp32 after an FP64 multiply by 1/sigma; an
orthonormal DFT with weight 2 for 0<k<n/2 and 1 for the Nyquist value; strided
sampling; equi-depth breakpoint a = sorted[floor(a*S/alpha)]; breakpoints
stored as fp32 with -inf / +inf ends; variance ties broken by candidate id;
ties in distance (within 1e-6 relative of a run's first element) ordered by
ascending index.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsofa_oracle.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                "oracle library missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(_LIB_PATH)
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.orc_znorm.argtypes = [f32p, ctypes.c_int64, ctypes.c_int32, f32p, f64p, f64p]
        lib.orc_dft_rows.argtypes = [f32p, ctypes.c_int64, ctypes.c_int32, f64p, f64p]
        lib.orc_sqdist.argtypes = [f32p, ctypes.c_int64, ctypes.c_int32, f32p, f64p]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- z-norm
def znorm(x: np.ndarray):
    """Canonical z-normalised fp32 series (Sec. II, Def. z-ED).

    mu and sigma (population) are FP64 left-to-right sums; Z = fp32((x-mu)*(1/sigma)).
    Returns (Z, mu, sigma)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    N, n = x.shape
    z = np.empty_like(x)
    mu = np.empty(N, np.float64)
    sg = np.empty(N, np.float64)
    _load().orc_znorm(x, N, n, z, mu, sg)
    return z, mu, sg


# ---------------------------------------------------------------- DFT values
def value_table(n: int, pool: int = 0):
    """Candidate Fourier values (Sec. IV "Feature Selection": individual real or
    imaginary parts).  Coefficients k = 1..floor(n/2) (k=0 is the mean, 0 after
    z-normalisation, Eq. 1 remark), restricted to k <= pool when pool > 0.
    Order (= candidate id): k ascending, real part before imaginary part.  The
    imaginary part of the Nyquist coefficient (n even, k = n/2) is identically
    zero and is not a candidate.  Returns list of (k, part) with part 0=re, 1=im."""
    K = n // 2 if pool <= 0 else min(pool, n // 2)
    out = []
    for k in range(1, K + 1):
        out.append((k, 0))
        if not (n % 2 == 0 and 2 * k == n):
            out.append((k, 1))
    return out


def weight(n: int, k: int) -> float:
    """Weight of a value of coefficient k in Eq. (1): each 0<k<n/2 stands for the
    conjugate pair k, n-k (weight 2); the Nyquist coefficient (2k == n) is its
    own pair (weight 1).  Parseval with these weights gives the exact ED^2."""
    return 1.0 if 2 * k == n else 2.0


def dft(z: np.ndarray):
    """Orthonormal DFT X_k = n^{-1/2} sum_t Z_t e^{-2 pi i k t/n}, k=0..floor(n/2),
    direct FP64 sums (Alg. 1/2 step 1).  Returns (re, im), each N x (n/2+1)."""
    z = np.ascontiguousarray(z, dtype=np.float32)
    N, n = z.shape
    K = n // 2 + 1
    re = np.empty((N, K), np.float64)
    im = np.empty((N, K), np.float64)
    _load().orc_dft_rows(z, N, n, re, im)
    return re, im


def dft_values(z: np.ndarray, pool: int = 0):
    """All candidate values (value_table order) of each z row, FP64: N x ncand."""
    re, im = dft(z)
    n = z.shape[1]
    tab = value_table(n, pool)
    out = np.empty((z.shape[0], len(tab)), np.float64)
    for c, (k, p) in enumerate(tab):
        out[:, c] = re[:, k] if p == 0 else im[:, k]
    return out


# ---------------------------------------------------------------- sampling
def sample_stride(ratio: float) -> int:
    """Alg. 1 line 2 'sample(X, r)': the paper does not say how.  Reading: a
    deterministic strided sample, every s-th series from row 0, with
    s = ceil(1/r - 1e-9) (so r = 0.1 gives exactly every 10th series)."""
    if not (0.0 < ratio <= 1.0):
        raise ValueError("sample ratio must lie in (0, 1]")
    return max(1, int(math.ceil(1.0 / ratio - 1e-9)))


def sample_rows(N: int, ratio: float) -> np.ndarray:
    s = sample_stride(ratio)
    return np.arange(0, N, s, dtype=np.int64)


# ---------------------------------------------------------------- selection
def select_values(vals: np.ndarray, n: int, l: int, mode: str = "variance", pool: int = 0):
    """Feature selection (Sec. IV "Novel Feature Selection"; Alg. 1 step 2):
    best = k-argmax of the per-value variance over the sample.

    vals: S x ncand FP64 candidate values of the sampled series.  Variance is the
    FP64 population variance.  Ranking: variance descending, ties by candidate id
    ascending ('first' mode: by id only, the classical low-pass SFA).  The top
    min(2l, ncand) values are taken; the first l form the SFA word and all of them
    are the proposal network's inputs.  Word order: rank order, except that a
    selected Nyquist value is moved to word position 0 (its weight differs).

    Returns dict(ids, ks, parts, w, var, ranked) for the selected values."""
    tab = value_table(n, pool)
    ncand = len(tab)
    if vals.shape[1] != ncand:
        raise ValueError("candidate count mismatch")
    mean = vals.mean(axis=0)
    var = ((vals - mean) ** 2).mean(axis=0)
    ids = np.arange(ncand)
    if mode == "variance":
        order = list(np.lexsort((ids, -var)))          # primary: -var, secondary: id
    elif mode == "first":
        order = list(ids)
    else:
        raise ValueError(mode)
    m = min(2 * l, ncand)
    top = order[:m]
    word = top[:l]
    nyq = [c for c in word if 2 * tab[c][0] == n]
    if nyq:
        word = nyq + [c for c in word if c not in nyq]
    chosen = word + top[l:m]
    ks = np.array([tab[c][0] for c in chosen], np.int32)
    parts = np.array([tab[c][1] for c in chosen], np.int32)
    w = np.array([weight(n, int(k)) for k in ks], np.float64)
    return dict(ids=np.array(chosen, np.int32), ks=ks, parts=parts, w=w,
                var=var[chosen], all_var=var)


# ---------------------------------------------------------------- bins (MCB)
def learn_bins(v: np.ndarray, alpha: int, mode: str = "equi-depth") -> np.ndarray:
    """MCB bins for one selected value (Sec. IV "Transformation and Learned
    Quantization"; Alg. 1 step 3).  v: the S sample values of that Fourier value.

    alpha bins [beta(a-1), beta(a)), a = 1..alpha, with beta(0) = -inf and
    beta(alpha) = +inf (the outer bins are open).
    equi-depth: beta(a) = sorted(v)[floor(a*S/alpha)]
    equi-width: beta(a) = min + a*(max-min)/alpha   (FP64)
    Breakpoints are stored as fp32 (the stored model); returned as float32."""
    S = v.shape[0]
    beta = np.empty(alpha + 1, np.float64)
    beta[0] = -np.inf
    beta[alpha] = np.inf
    if mode == "equi-depth":
        sv = np.sort(v, kind="stable")
        for a in range(1, alpha):
            beta[a] = sv[(a * S) // alpha]
    elif mode == "equi-width":
        lo = float(np.min(v))
        hi = float(np.max(v))
        for a in range(1, alpha):
            beta[a] = lo + a * (hi - lo) / alpha
    else:
        raise ValueError(mode)
    return beta.astype(np.float32)


def learn_summary(x: np.ndarray, l: int, alpha: int, ratio: float = 0.1,
                  binning: str = "equi-depth", select: str = "variance", pool: int = 0):
    """Alg. 1 (MCB) end to end: sample, DFT, select, learn bins."""
    N, n = x.shape
    rows = sample_rows(N, ratio)
    z, _, _ = znorm(x[rows])
    vals = dft_values(z, pool)
    sel = select_values(vals, n, l, select, pool)
    lw = min(l, len(sel["ids"]))
    beta = np.stack([learn_bins(vals[:, sel["ids"][j]], alpha, binning) for j in range(lw)])
    sel["beta"] = beta
    sel["n"] = n
    sel["l"] = lw
    sel["alpha"] = alpha
    return sel


# ---------------------------------------------------------------- SFA words
def selected_values(z: np.ndarray, summ) -> np.ndarray:
    """FP64 values of the selected Fourier values (word order then extras)."""
    re, im = dft(z)
    cols = []
    for k, p in zip(summ["ks"], summ["parts"]):
        cols.append(re[:, k] if p == 0 else im[:, k])
    return np.stack(cols, axis=1)


def symbols(v: np.ndarray, beta_j: np.ndarray) -> np.ndarray:
    """Symbol of value(s) v under bins beta_j (Alg. 2 step 2): the a with
    v in [beta(a), beta(a+1)), i.e. the count of finite breakpoints <= v."""
    inner = beta_j[1:-1].astype(np.float64)
    return np.searchsorted(inner, v, side="right").astype(np.uint8)


def words(z: np.ndarray, summ) -> np.ndarray:
    """SFA words (Alg. 2), N x l uint8."""
    v = selected_values(z, summ)
    l = summ["l"]
    return np.stack([symbols(v[:, j], summ["beta"][j]) for j in range(l)], axis=1)


# ---------------------------------------------------------------- lower bound
def mind(b, lo, hi):
    """Eq. dist_i: distance from value b to the interval [lo, hi):
    lo - b below it, b - hi above it, 0 inside."""
    b = np.asarray(b, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return np.where(b < lo, lo - b, np.where(b > hi, b - hi, 0.0))


def lb2(qv: np.ndarray, wds: np.ndarray, summ) -> np.ndarray:
    """Squared SFA lower bound between a query's numeric Fourier values qv (its
    first l selected values) and N words (SFA LBD of Sec. IV, with Eq. 1's
    weights): sum_j w_j * mind_j(word_j, qv_j)^2.  FP64."""
    l = summ["l"]
    beta = summ["beta"].astype(np.float64)
    out = np.zeros(wds.shape[0], np.float64)
    for j in range(l):
        s = wds[:, j].astype(np.int64)
        lo = beta[j][s]
        hi = beta[j][s + 1]
        m = mind(qv[j], lo, hi)
        out += summ["w"][j] * m * m
    return out


def dft_lb2(qv: np.ndarray, xv: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Eq. (1) restricted to the selected values: sum_j w_j (q_j - x_j)^2."""
    return ((qv[None, :] - xv) ** 2 * w[None, :]).sum(axis=1)


# ---------------------------------------------------------------- exact k-NN
def sqdist(Z: np.ndarray, zq: np.ndarray) -> np.ndarray:
    """FP64 squared z-ED of one canonical query to every canonical series."""
    Z = np.ascontiguousarray(Z, dtype=np.float32)
    zq = np.ascontiguousarray(zq, dtype=np.float32)
    out = np.empty(Z.shape[0], np.float64)
    _load().orc_sqdist(Z, Z.shape[0], Z.shape[1], zq, out)
    return out


def tie_order(d2: np.ndarray, ids: np.ndarray):
    """Final ordering: sort by FP64 distance (then id); a run of consecutive
    results whose distance d satisfies d <= d0 + 1e-6*d0 (d0 = the run's first
    distance) is reordered by ascending index.  Returns (ids, dist)."""
    d = np.sqrt(d2)
    o = np.lexsort((ids, d))
    d = d[o]
    ids = ids[o]
    out_i = []
    out_d = []
    i = 0
    m = len(d)
    while i < m:
        d0 = d[i]
        lim = d0 + 1e-6 * d0
        j = i
        while j + 1 < m and d[j + 1] <= lim:
            j += 1
        seg = np.argsort(ids[i:j + 1], kind="stable")
        out_i.extend(ids[i:j + 1][seg])
        out_d.extend(d[i:j + 1][seg])
        i = j + 1
    return np.array(out_i, np.int64), np.array(out_d, np.float64)


def knn_full(Z: np.ndarray, Zq: np.ndarray, k: int):
    """Exact k-NN by brute force (Sec. II NN problem, k-NN extension): every
    distance, fully sorted, tie runs reordered, first k.  Definition form."""
    Q = Zq.shape[0]
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)
    ids = np.arange(Z.shape[0], dtype=np.int64)
    for q in range(Q):
        d2 = sqdist(Z, Zq[q])
        oi, od = tie_order(d2, ids)
        idx[q] = oi[:k]
        dist[q] = od[:k]
    return idx, dist


def knn(Z: np.ndarray, Zq: np.ndarray, k: int):
    """Same result as knn_full, restricted before sorting to the distances that
    can reach the first k places: d <= D_k + 1e-6*D_k with D_k the k-th smallest.
    Runs that touch the first k places start at or before place k, so all their
    members satisfy that bound (the bound is monotone in the run's start)."""
    Q = Zq.shape[0]
    N = Z.shape[0]
    if k > N:
        raise ValueError("k > N")
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)
    for q in range(Q):
        d2 = sqdist(Z, Zq[q])
        d = np.sqrt(d2)
        Dk = np.partition(d, k - 1)[k - 1]
        lim = Dk + 1e-6 * Dk
        keep = np.nonzero(d <= lim)[0]
        oi, od = tie_order(d2[keep], keep.astype(np.int64))
        idx[q] = oi[:k]
        dist[q] = od[:k]
    return idx, dist


def knn_chunked(chunks, Zq: np.ndarray, k: int, keep: int = 64):
    """Same result as knn_full over a dataset too large to hold at once.
    `chunks` yields (row0, Z_chunk) with the canonical rows row0.. of the
    dataset, in any order, covering every row once.  Per query, each chunk
    contributes its k + keep smallest squared distances; the merged set is then
    cut by the rule of `knn` (d <= D_k + 1e-6 D_k) and ordered by tie_order.
    A chunk whose (k + keep)-th distance lies inside the final window could
    have dropped a member of it: that raises instead of returning a guess."""
    Q = Zq.shape[0]
    m = k + keep
    best_d2 = [np.empty(0, np.float64) for _ in range(Q)]
    best_id = [np.empty(0, np.int64) for _ in range(Q)]
    cuts = [[] for _ in range(Q)]  # squared distance of the last kept row of a truncated chunk
    total = 0
    for row0, Zc in chunks:
        rows = Zc.shape[0]
        total += rows
        for q in range(Q):
            d2 = sqdist(Zc, Zq[q])
            if rows > m:
                sel = np.argpartition(d2, m - 1)[:m]
                cuts[q].append(float(d2[sel].max()))
            else:
                sel = np.arange(rows)
            best_d2[q] = np.concatenate([best_d2[q], d2[sel]])
            best_id[q] = np.concatenate([best_id[q], sel.astype(np.int64) + int(row0)])
    if k > total:
        raise ValueError("k > N")
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)
    for q in range(Q):
        d = np.sqrt(best_d2[q])
        Dk = np.partition(d, k - 1)[k - 1]
        lim = Dk + 1e-6 * Dk
        if cuts[q] and np.sqrt(min(cuts[q])) <= lim:
            raise RuntimeError("a chunk's kept distances do not cover the tie window: raise `keep`")
        sel = np.nonzero(d <= lim)[0]
        oi, od = tie_order(best_d2[q][sel], best_id[q][sel])
        idx[q] = oi[:k]
        dist[q] = od[:k]
    return idx, dist


def gemini_knn(Z: np.ndarray, W: np.ndarray, Zq: np.ndarray, summ, k: int):
    """GEMINI filter-and-refine (Sec. II-A, Sec. IV "Exact Similarity Search"):
    visit series in ascending SFA lower bound, compute the exact distance only
    while the lower bound does not exceed the k-th best distance so far (widened
    by the 1e-6 tie window).  Returns (idx, dist, refined_count)."""
    Q = Zq.shape[0]
    qv_all = selected_values(Zq, summ)
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)
    refined = np.zeros(Q, np.int64)
    for q in range(Q):
        lb = lb2(qv_all[q][: summ["l"]], W, summ)
        order = np.argsort(lb, kind="stable")
        best_d2 = []
        best_i = []
        for i in order:
            if len(best_d2) >= k:
                kth = sorted(best_d2)[k - 1]
                dk = math.sqrt(kth)
                lim = dk + 1e-6 * dk
                if math.sqrt(max(lb[i], 0.0)) > lim * (1 + 1e-9):
                    break
            d2 = float(sqdist(Z[i:i + 1], Zq[q])[0])
            best_d2.append(d2)
            best_i.append(int(i))
            refined[q] += 1
        oi, od = tie_order(np.array(best_d2), np.array(best_i, np.int64))
        idx[q] = oi[:k]
        dist[q] = od[:k]
    return idx, dist, refined


# ---------------------------------------------------------------- proposal MLP
def gelu(x):
    """Exact GELU, x * Phi(x), Phi via erf."""
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def mlp_forward(params, x):
    """Proposal network 32 -> 256 -> 256 -> C (GELU hidden layers, softmax out).
    params: dict W1 [d_in,h], b1 [h], W2 [h,h], b2 [h], W3 [h,C], b3 [C] (FP64).
    Returns logits and the cache for the backward pass."""
    a1 = x @ params["W1"] + params["b1"]
    h1 = gelu(a1)
    a2 = h1 @ params["W2"] + params["b2"]
    h2 = gelu(a2)
    logits = h2 @ params["W3"] + params["b3"]
    return logits, (x, a1, h1, a2, h2)


def softmax_xent(logits, y):
    """Mean softmax cross-entropy and its gradient w.r.t. the logits."""
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    B = logits.shape[0]
    loss = float(-np.log(p[np.arange(B), y]).mean())
    g = p.copy()
    g[np.arange(B), y] -= 1.0
    return loss, g / B


def mlp_loss_grad(params, x, y):
    """Loss and gradients of every parameter (FP64 backward pass)."""
    logits, (x, a1, h1, a2, h2) = mlp_forward(params, x)
    loss, g3 = softmax_xent(logits, y)
    grads = {}
    grads["W3"] = h2.T @ g3
    grads["b3"] = g3.sum(axis=0)
    gh2 = g3 @ params["W3"].T
    ga2 = gh2 * gelu_grad(a2)
    grads["W2"] = h1.T @ ga2
    grads["b2"] = ga2.sum(axis=0)
    gh1 = ga2 @ params["W2"].T
    ga1 = gh1 * gelu_grad(a1)
    grads["W1"] = x.T @ ga1
    grads["b1"] = ga1.sum(axis=0)
    return loss, grads


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; t counts from 1."""
    out = {}
    for key in params:
        m[key] = b1 * m[key] + (1 - b1) * grads[key]
        v[key] = b2 * v[key] + (1 - b2) * grads[key] ** 2
        mh = m[key] / (1 - b1 ** t)
        vh = v[key] / (1 - b2 ** t)
        out[key] = params[key] - lr * mh / (np.sqrt(vh) + eps)
    return out
