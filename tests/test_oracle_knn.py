"""Pins of the oracle's exact k-NN, tie rule and GEMINI search."""
import math

import numpy as np
import pytest

from oracle import sofa_oracle as orc


def rw(N, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal((N, n)), axis=1).astype(np.float32)


def test_sqdist_matches_numpy():
    z, _, _ = orc.znorm(rw(300, 48, 0))
    d = orc.sqdist(z, z[5])
    ref = ((z.astype(np.float64) - z[5].astype(np.float64)) ** 2).sum(axis=1)
    assert np.allclose(d, ref, rtol=1e-13)
    assert d[5] == 0.0


def test_query_equal_to_member_is_its_own_nn():
    z, _, _ = orc.znorm(rw(500, 32, 1))
    idx, dist = orc.knn(z, z[[7, 100, 499]], 1)
    assert list(idx[:, 0]) == [7, 100, 499]
    assert np.all(dist == 0)


def test_tie_rule_duplicates_and_near_ties():
    rng = np.random.default_rng(3)
    n = 16
    z = rng.standard_normal((40, n)).astype(np.float32)
    q = rng.standard_normal(n).astype(np.float32)
    # exact duplicates of a near point at rows 30, 4, 17: the lowest index first
    near = q + np.float32(0.01)
    for r in (30, 4, 17):
        z[r] = near
    idx, dist = orc.knn_full(z, q[None, :], 3)
    assert list(idx[0]) == [4, 17, 30]
    assert dist[0, 0] == dist[0, 1] == dist[0, 2]


def test_tie_window_is_one_millionth_relative():
    """Distances d0 < d1 with d1/d0 - 1 = 5e-7 form one run (index order);
    with 5e-6 they stay in distance order."""
    d0 = 2.0
    for rel, expect in ((5e-7, [3, 9]), (5e-6, [9, 3])):
        d2 = np.array([d0 ** 2, (d0 * (1 + rel)) ** 2])
        ids = np.array([9, 3])
        oi, od = orc.tie_order(d2, ids)
        assert list(oi) == expect


def test_run_is_anchored_at_first_element():
    # 1.0, 1.0+0.8e-6 (in run), 1.0+1.6e-6 (outside: > 1e-6 from the run's first)
    d = np.array([1.0, 1.0 + 0.8e-6, 1.0 + 1.6e-6])
    ids = np.array([5, 1, 0])
    oi, _ = orc.tie_order(d ** 2, ids)
    assert list(oi) == [1, 5, 0]


@pytest.mark.parametrize("k", [1, 5, 50])
def test_window_knn_equals_full_sort(k):
    rng = np.random.default_rng(k)
    z, _, _ = orc.znorm(rw(2000, 32, 5))
    q = z[:10].copy()
    q += 1e-3 * rng.standard_normal(q.shape).astype(np.float32)
    # plant near ties
    z[1500] = z[1]
    z[1501] = z[2] * np.float32(1 + 1e-8)
    a = orc.knn_full(z, q, k)
    b = orc.knn(z, q, k)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("k,chunk,keep", [(1, 97, 4), (5, 250, 8), (50, 700, 64), (3, 5000, 1)])
def test_chunked_knn_equals_full_sort(k, chunk, keep):
    rng = np.random.default_rng(10 + k)
    z, _, _ = orc.znorm(rw(2000, 32, 6))
    q = z[:8].copy()
    q += 1e-3 * rng.standard_normal(q.shape).astype(np.float32)
    z[1700] = z[1]                          # exact duplicate across chunks
    z[1701] = z[2] * np.float32(1 + 1e-8)   # near tie across chunks
    order = list(range(0, 2000, chunk))[::-1]   # chunks in reverse order
    a = orc.knn_full(z, q, k)
    b = orc.knn_chunked(((r, z[r:r + chunk]) for r in order), q, k, keep=keep)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_chunked_knn_refuses_a_truncated_window():
    z, _, _ = orc.znorm(rw(400, 16, 7))
    z[:] = z[0]                              # every row ties with every other
    with pytest.raises(RuntimeError):
        orc.knn_chunked(((r, z[r:r + 100]) for r in range(0, 400, 100)), z[:1], 1, keep=4)


@pytest.mark.parametrize("n,alpha,k", [(8, 2, 1), (16, 4, 5), (64, 256, 50), (64, 4, 1), (16, 256, 5)])
def test_gemini_equals_bruteforce(n, alpha, k):
    """GEMINI (Sec. II-A) with the SFA bound returns exactly the brute-force
    answer: a failure here means some LB exceeded a true distance."""
    N = 1500
    x = rw(N, n, n + alpha)
    x[700] = x[3]                                   # a duplicate pair
    summ = orc.learn_summary(x, l=min(8, n - 1), alpha=alpha, ratio=0.1)
    z, _, _ = orc.znorm(x)
    W = orc.words(z, summ)
    qx = rw(6, n, 99)
    qx[0] = x[3]
    zq, _, _ = orc.znorm(qx)
    gi, gd, refined = orc.gemini_knn(z, W, zq, summ, k)
    bi, bd = orc.knn_full(z, zq, k)
    assert np.array_equal(gi, bi)
    assert np.array_equal(gd, bd)
    assert refined.min() >= k


def test_window_keeps_a_near_tie_beyond_the_kth():
    """Row 10 at distance 1 and row 3 at distance 1 + 4.77e-7 (one fp32 step
    count away): one tie run, so the 1-NN is row 3 (lowest index), although
    row 10 alone is the nearest.  The restricted forms must widen their window
    by the 1e-6 tie window to see row 3."""
    n = 4
    Z = np.full((20, n), 2.0, np.float32)           # every other row at distance 4
    Z[10] = [1.0, 0.0, 0.0, 0.0]
    Z[3] = [np.float32(1.0 + 5e-7), 0.0, 0.0, 0.0]
    q = np.zeros((1, n), np.float32)
    d3 = float(np.float32(1.0 + 5e-7))
    assert 1.0 < d3 < 1.0 + 1e-6                     # within the tie window of row 10
    for fn in (orc.knn_full, orc.knn,
               lambda Z_, q_, k: orc.knn_chunked(((r, Z_[r:r + 7]) for r in range(0, 20, 7)), q_, k, keep=2)):
        idx, dist = fn(Z, q, 1)
        assert idx[0, 0] == 3 and dist[0, 0] == d3


def test_gemini_refines_a_near_tie_beyond_the_kth():
    """GEMINI's stopping rule must keep the 1e-6 tie window: row 10 is at
    distance exactly 1 with bound 0; row 3 is at distance 2b = 1 + 4.77e-7
    and its bound is 2*beta^2 with beta the bin edge just below its value, so
    1 < bound <= its distance^2.  Stopping at bound > (the best distance)^2
    would never refine row 3, whose lower index puts it first in the tie run.
    n = 8; the selected value is Re X_2 (weight 2); every other row is far
    (6 cos) but shares row 3's bin, hence its bound."""
    n = 8
    cos2 = np.array([1, 0, -1, 0, 1, 0, -1, 0], np.float32)   # cos(2 pi 2 t / 8)
    sin2 = np.array([0, 1, 0, -1, 0, 1, 0, -1], np.float32)   # sin(2 pi 2 t / 8)
    b = np.float32(0.5 * (1 + 5e-7))
    Z = np.tile(3.0 * cos2, (20, 1)).astype(np.float32)
    Z[10] = 0.5 * sin2                                         # distance^2 = 4 * 0.25 = 1, Re X_2 = 0
    Z[3] = b * cos2                                            # distance^2 = 4 b^2, Re X_2 = b sqrt(2)
    q = np.zeros((1, n), np.float32)
    vb = float(b) * math.sqrt(2.0)
    edge = np.float32(vb)
    if float(edge) > vb:                                       # the bin edge at or just below row 3's value
        edge = np.nextafter(edge, np.float32(0))
    summ = {"l": 1, "ks": np.array([2]), "parts": np.array([0]), "w": np.array([2.0]),
            "beta": np.array([[-np.inf, 0.35, float(edge), np.inf]], np.float32)}
    assert 1.0 < 2 * float(edge) ** 2 <= 4 * float(b) ** 2 < (1 + 1e-6) ** 2
    W = orc.words(Z, summ)
    assert W[3, 0] == 2 and W[10, 0] == 0
    bi, bd = orc.knn_full(Z, q, 1)
    assert bi[0, 0] == 3
    gi, gd, _ = orc.gemini_knn(Z, W, q, summ, 1)
    assert gi[0, 0] == 3 and gd[0, 0] == bd[0, 0]
