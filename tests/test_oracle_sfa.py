"""Pins of the oracle's SFA parts against facts the paper and mathematics fix.

None of these re-types an oracle formula: each compares with a closed form, an
invariant, a library routine or a brute-force count."""
import math
import os

import numpy as np
import pytest

from oracle import sofa_oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rw(N, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal((N, n)), axis=1).astype(np.float32)


# ------------------------------------------------------------------ z-norm
def test_znorm_closed_form():
    # x = 1..8: mean 4.5, population variance (8^2-1)/12 = 5.25
    x = np.arange(1, 9, dtype=np.float32)[None, :]
    z, mu, sg = orc.znorm(x)
    assert mu[0] == 4.5
    assert sg[0] == math.sqrt(5.25)
    expect = (np.arange(1, 9) - 4.5) / math.sqrt(5.25)
    assert np.allclose(z[0], expect, rtol=0, atol=1e-6)


def test_znorm_population_sigma_and_constant_row():
    x = rw(50, 64, 0)
    x[3] = 7.0
    z, mu, sg = orc.znorm(x)
    assert np.all(z[3] == 0)
    zz = np.delete(z, 3, axis=0).astype(np.float64)
    assert np.allclose(zz.mean(axis=1), 0, atol=1e-6)
    # population sigma => sum z^2 = n (a sample sigma would give n-1)
    assert np.allclose((zz ** 2).sum(axis=1), 64, rtol=1e-6)
    ok = np.arange(50) != 3
    xs = x[ok].astype(np.float64)
    ref = (xs - xs.mean(axis=1, keepdims=True)) / xs.std(axis=1, keepdims=True)
    assert np.allclose(z[ok], ref, atol=2e-6)


# ------------------------------------------------------------------ DFT
def test_dft_sinusoid_closed_form():
    """x_t = A cos(2 pi f t/n + phi), integer 0 < f < n/2:
    orthonormal DFT gives X_f = (A sqrt(n)/2) e^{i phi}, X_k = 0 otherwise."""
    with open(os.path.join(GOLDEN, "sinusoid_dft.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for n, f, A, phi, ere, eim in rows:
        n, f = int(n), int(f)
        A, phi, ere, eim = float(A), float(phi), float(ere), float(eim)
        t = np.arange(n)
        x = (A * np.cos(2 * np.pi * f * t / n + phi)).astype(np.float32)[None, :]
        re, im = orc.dft(x)
        assert abs(re[0, f] - ere) < 1e-5 * A * math.sqrt(n)
        assert abs(im[0, f] - eim) < 1e-5 * A * math.sqrt(n)
        other = [k for k in range(n // 2 + 1) if k != f]
        assert np.abs(re[0, other]).max() < 1e-5 * A * math.sqrt(n)
        assert np.abs(im[0, other]).max() < 1e-5 * A * math.sqrt(n)


@pytest.mark.parametrize("n", [8, 15, 64, 256])
def test_dft_matches_numpy_fft(n):
    x = rw(20, n, 1)
    re, im = orc.dft(x)
    F = np.fft.rfft(x.astype(np.float64), axis=1) / math.sqrt(n)
    assert np.allclose(re, F.real, atol=1e-9)
    assert np.allclose(im, F.imag, atol=1e-9)


@pytest.mark.parametrize("n", [8, 9, 64, 256])
def test_parseval_weights(n):
    """Eq. (1) over every value with weights 1 (k=0), 2 (0<k<n/2), 1 (Nyquist)
    equals the squared ED exactly (up to FP64 rounding)."""
    a = rw(30, n, 2)
    b = rw(30, n, 3)
    za, _, _ = orc.znorm(a)
    zb, _, _ = orc.znorm(b)
    ra, ia = orc.dft(za)
    rb, ib = orc.dft(zb)
    ed2 = ((za.astype(np.float64) - zb.astype(np.float64)) ** 2).sum(axis=1)
    tot = (ra[:, 0] - rb[:, 0]) ** 2
    for k in range(1, n // 2 + 1):
        w = orc.weight(n, k)
        tot += w * ((ra[:, k] - rb[:, k]) ** 2 + (ia[:, k] - ib[:, k]) ** 2)
    assert np.allclose(tot, ed2, rtol=1e-11)


def test_value_table():
    assert orc.value_table(8) == [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1), (4, 0)]
    assert orc.value_table(7) == [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)]
    assert orc.value_table(256, pool=16) == [(k, p) for k in range(1, 17) for p in (0, 1)]
    assert orc.weight(8, 4) == 1.0 and orc.weight(8, 3) == 2.0 and orc.weight(7, 3) == 2.0


def test_full_pool_dft_lb_equals_ed():
    """All candidate values with Eq. (1) weights: the DFT bound is the ED^2."""
    n = 32
    z, _, _ = orc.znorm(rw(40, n, 4))
    v = orc.dft_values(z)
    w = np.array([orc.weight(n, k) for k, _ in orc.value_table(n)])
    for i in range(1, 40):
        lb = orc.dft_lb2(v[0], v[i:i + 1], w)[0]
        ed2 = ((z[0].astype(np.float64) - z[i]) ** 2).sum()
        assert abs(lb - ed2) <= 1e-10 * ed2


# ------------------------------------------------------------------ sampling
def test_sample_stride():
    assert orc.sample_stride(0.1) == 10
    assert orc.sample_stride(0.01) == 100
    assert orc.sample_stride(1.0) == 1
    assert orc.sample_stride(0.3) == 4
    assert list(orc.sample_rows(25, 0.1)) == [0, 10, 20]


# ------------------------------------------------------------------ selection
def test_selection_finds_planted_frequencies():
    """Sinusoids with energy at k=5 (cos) and k=11 (sin): the top variance values
    are Re X_5 and Im X_11 (high-variance selection, Sec. IV)."""
    rng = np.random.default_rng(5)
    n, S = 64, 400
    t = np.arange(n)
    a = rng.standard_normal(S)[:, None] * 3
    b = rng.standard_normal(S)[:, None] * 2
    x = a * np.cos(2 * np.pi * 5 * t / n) + b * np.sin(2 * np.pi * 11 * t / n)
    x = x + 0.05 * rng.standard_normal((S, n))
    z, _, _ = orc.znorm(x.astype(np.float32))
    v = orc.dft_values(z)
    sel = orc.select_values(v, n, l=2)
    tab = orc.value_table(n)
    got = {tab[c] for c in sel["ids"][:2]}
    assert got == {(5, 0), (11, 1)}


def test_selection_ties_and_nyquist_first():
    n = 8
    tab = orc.value_table(n)            # 7 candidates, id 6 = Nyquist real part
    rng = np.random.default_rng(0)
    S = 100
    vals = np.zeros((S, len(tab)))
    base = rng.standard_normal(S)
    # ids 1 and 3 tie exactly at the top variance; id 6 (Nyquist) third
    vals[:, 1] = 3 * base
    vals[:, 3] = -3 * base
    vals[:, 6] = 2 * base
    vals[:, 0] = 1 * base
    sel = orc.select_values(vals, n, l=3)
    # brute force ranking with the tie rule: var desc, then id
    var = vals.var(axis=0)
    brute = sorted(range(len(tab)), key=lambda c: (-var[c], c))
    assert brute[:3] == [1, 3, 6]
    assert list(sel["ids"][:3]) == [6, 1, 3]      # Nyquist moved to word position 0
    assert sel["w"][0] == 1.0 and sel["w"][1] == 2.0
    first = orc.select_values(vals, n, l=3, mode="first")
    assert list(first["ids"][:3]) == [0, 1, 2]


# ------------------------------------------------------------------ bins
@pytest.mark.parametrize("S,alpha", [(1000, 4), (997, 16), (5000, 256), (300, 256)])
def test_equi_depth_counts(S, alpha):
    rng = np.random.default_rng(S)
    v = rng.standard_normal(S)                  # distinct values
    beta = orc.learn_bins(v, alpha, "equi-depth")
    # breakpoints are stored fp32: compare the fp32-rounded sample
    v32 = v.astype(np.float32).astype(np.float64)
    s = orc.symbols(v32, beta)
    counts = np.bincount(s, minlength=alpha)
    lo, hi = S // alpha, -(-S // alpha)
    if S >= alpha:
        assert counts.min() >= lo and counts.max() <= hi
    assert counts.sum() == S


def test_equi_depth_ties_only_shift_by_multiplicity():
    v = np.repeat(np.arange(10, dtype=np.float64), 30)      # each value 30 times
    beta = orc.learn_bins(v, 4, "equi-depth")
    s = orc.symbols(v, beta)
    counts = np.bincount(s, minlength=4)
    assert counts.sum() == 300
    assert np.all(np.abs(counts - 75) <= 30)


def test_equi_width_spacing():
    rng = np.random.default_rng(1)
    v = rng.uniform(-3, 5, 2000)
    beta = orc.learn_bins(v, 64, "equi-width").astype(np.float64)
    assert beta[0] == -np.inf and beta[-1] == np.inf
    d = np.diff(beta[1:-1])
    w = (v.max() - v.min()) / 64
    assert np.allclose(d, w, rtol=0, atol=4 * np.spacing(np.float32(5.0)))
    assert abs(beta[1] - (v.min() + w)) < 1e-6


def test_symbols_bruteforce():
    rng = np.random.default_rng(2)
    beta = np.concatenate([[-np.inf], np.sort(rng.standard_normal(7)), [np.inf]]).astype(np.float32)
    vals = np.concatenate([rng.standard_normal(200), beta[1:-1].astype(np.float64)])
    s = orc.symbols(vals, beta)
    for v, got in zip(vals, s):
        count = sum(1 for a in range(1, 8) if float(beta[a]) <= v)
        assert got == count
        assert float(beta[got]) <= v < float(beta[got + 1])      # half-open bins


def test_mind_three_cases():
    assert orc.mind(0.0, 1.0, 2.0) == 1.0        # below the bin
    assert orc.mind(3.5, 1.0, 2.0) == 1.5        # above the bin
    assert orc.mind(1.5, 1.0, 2.0) == 0.0        # inside
    assert orc.mind(1.0, 1.0, 2.0) == 0.0


# ------------------------------------------------------------------ LB <= ED
@pytest.mark.parametrize("gen", ["rw", "noisy", "sin"])
@pytest.mark.parametrize("alpha,binning", [(256, "equi-depth"), (4, "equi-depth"), (16, "equi-width")])
def test_lb_le_dftlb_le_ed(gen, alpha, binning):
    rng = np.random.default_rng(11)
    n, N = 64, 3000
    if gen == "rw":
        x = rw(N, n, 7)
    elif gen == "noisy":
        x = rw(N, n, 8) + 0.5 * rng.standard_normal((N, n)).astype(np.float32)
    else:
        t = np.arange(n)
        f = rng.uniform(0, n / 2, (N, 8, 1))
        ph = rng.uniform(0, 2 * np.pi, (N, 8, 1))
        A = np.exp(rng.standard_normal((N, 8, 1)))
        x = (A * np.sin(2 * np.pi * f * t / n + ph)).sum(axis=1) + 0.3 * rng.standard_normal((N, n))
        x = x.astype(np.float32)
    summ = orc.learn_summary(x, l=8, alpha=alpha, ratio=0.1, binning=binning)
    z, _, _ = orc.znorm(x)
    W = orc.words(z, summ)
    V = orc.selected_values(z, summ)[:, :8]
    for qi in range(0, 40):
        lb = orc.lb2(V[qi], W, summ)
        dl = orc.dft_lb2(V[qi], V, summ["w"][:8])
        ed2 = orc.sqdist(z, z[qi])
        assert np.all(lb <= dl * (1 + 1e-12) + 1e-12)
        assert np.all(dl <= ed2 * (1 + 1e-9) + 1e-9)
        assert lb[qi] == 0.0


def test_lb2_tiny_closed_form():
    """Eq. dist_i with Eq. (1)'s weights on a hand-worked case: two values,
    the first a Nyquist value (weight 1), the second weight 2; bins
    [-inf, 0, 1, inf) and [-inf, -1, 2, inf); query values (3, 0.5).
    Word (1, 0): intervals [0, 1) and [-inf, -1) -> 1*(3-1)^2 + 2*(0.5+1)^2 = 8.5.
    Word (0, 2): [-inf, 0) and [2, inf) -> 1*(3-0)^2 + 2*(2-0.5)^2 = 13.5.
    Word (2, 1): [1, inf) and [-1, 2) hold both values -> 0."""
    inf = np.inf
    summ = {"l": 2, "w": np.array([1.0, 2.0]),
            "beta": np.array([[-inf, 0.0, 1.0, inf], [-inf, -1.0, 2.0, inf]], np.float32)}
    wds = np.array([[1, 0], [0, 2], [2, 1]], np.uint8)
    lb = orc.lb2(np.array([3.0, 0.5]), wds, summ)
    assert list(lb) == [8.5, 13.5, 0.0]


def test_learn_summary_uses_the_strided_sample():
    """Alg. 1 learns from sample(X, r): with r = 0.1 the rows 0, 10, 20, ...
    Those rows are cosines at k = 9 (random amplitude and sign), every other
    row a cosine at k = 3, so only the strided sample ranks Re X_9 first; the
    whole collection, or a sample shifted by one row, ranks Re X_3 first."""
    rng = np.random.default_rng(21)
    N, n = 1000, 64
    t = np.arange(n)
    amp = rng.standard_normal((N, 1)) * 3
    f = np.where(np.arange(N)[:, None] % 10 == 0, 9, 3)
    x = (amp * np.cos(2 * np.pi * f * t / n) + 0.01 * rng.standard_normal((N, n))).astype(np.float32)
    summ = orc.learn_summary(x, l=1, alpha=16, ratio=0.1)
    assert (int(summ["ks"][0]), int(summ["parts"][0])) == (9, 0)
    # the bins come from the same sample: the k = 9 values of rows 0, 10, ...
    z, _, _ = orc.znorm(x[::10])
    v = orc.dft_values(z)[:, orc.value_table(n).index((9, 0))]
    assert np.array_equal(summ["beta"][0], orc.learn_bins(v, 16, "equi-depth"))


def test_selected_values_closed_form():
    """A selected value is the real or imaginary part its (k, part) names:
    for x_t = 2 cos(2 pi 5 t/n) + 3 sin(2 pi 7 t/n), n = 32, the orthonormal
    DFT gives Re X_5 = sqrt(n), Im X_7 = -1.5 sqrt(n), Im X_5 = Re X_7 = 0."""
    n = 32
    t = np.arange(n)
    x = (2 * np.cos(2 * np.pi * 5 * t / n) + 3 * np.sin(2 * np.pi * 7 * t / n)).astype(np.float32)[None, :]
    summ = {"ks": np.array([5, 7, 5, 7]), "parts": np.array([0, 1, 1, 0])}
    v = orc.selected_values(x, summ)[0]
    expect = [math.sqrt(n), -1.5 * math.sqrt(n), 0.0, 0.0]
    assert np.allclose(v, expect, rtol=0, atol=1e-5)
