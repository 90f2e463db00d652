"""Build options and the Nyquist word value, CUDA path vs the CPU oracle.

* Equi-width bins, first-l selection and the paper's restricted coefficient
  pool (Sec. IV "Transformation and Learned Quantization", "Novel Feature
  Selection"; Sec. V sets the pool to the first 16 coefficients).  The learned
  summary, the words, the lower bounds and the exact k-NN are each compared
  with the oracle.
* A planted Nyquist case.  Every series carries a random-amplitude (-1)^t
  component, so the variance-ranked selection takes Re X_{n/2} into the word.
  Eq. (1) gives that value weight 1, not 2, and the library moves it to word
  position 0.  This drives the NYQ specialisations of the seed, envelope and
  series-bound kernels through exact k-NN.
"""
import numpy as np
import pytest
import torch

from oracle import sofa_oracle as orc
from paper_2411_17483_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def sofa():
    from paper_2411_17483_gb300 import sofa as s
    s.load()
    return s


def oracle_knn(x, q, k):
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    return orc.knn(z, zq, k)


def assert_knn_equal(gi, gd, oi, od):
    gi = gi.cpu().numpy()
    gd = gd.cpu().numpy().astype(np.float64)
    bad = np.nonzero(np.any(gi != oi, axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} queries differ, first {bad[:5]}: gpu {gi[bad[0]]} oracle {oi[bad[0]]}"
    rel = np.abs(gd - od) / np.maximum(od, 1e-30)
    assert rel.max() <= 1e-4
    assert np.array_equal(gd.astype(np.float32), od.astype(np.float32))


def summary_from_gpu(ix, n, l, alpha, pool):
    """The oracle's summary record for the GPU's exported selection and bins
    (sel ids in word order, word values first), so that oracle words and
    bounds can be computed under the GPU's own summary."""
    sel, var, beta = ix.summary()
    tab = orc.value_table(n, pool)
    ids = sel.numpy().astype(np.int32)
    ks = np.array([tab[c][0] for c in ids], np.int32)
    parts = np.array([tab[c][1] for c in ids], np.int32)
    w = np.array([orc.weight(n, int(kk)) for kk in ks], np.float64)
    return dict(ids=ids, ks=ks, parts=parts, w=w, var=var.numpy(), beta=beta.numpy(), n=n, l=l, alpha=alpha)


def check_words(ix, z, summ, delta):
    """GPU words equal the oracle's words under the same summary, except for
    values within the projection margin of a breakpoint (off by one there)."""
    gw = ix.words().numpy()
    ow = orc.words(z, summ)
    v = orc.selected_values(z, summ)[:, :summ["l"]]
    diff = gw != ow
    for r, j in zip(*np.nonzero(diff)):
        b = summ["beta"][j].astype(np.float64)
        near = np.min(np.abs(b[1:-1] - v[r, j]))
        assert near <= delta, (r, j, near)
        assert abs(int(gw[r, j]) - int(ow[r, j])) == 1
    return gw, ow


def check_bounds(ix, z, zq, q, summ, words_equal):
    """GPU lower bounds never exceed the FP64 distance, and on rows whose words
    agree they are the oracle's SFA bound up to the widening by the margins."""
    lb = ix.lower_bounds(q).cpu().numpy().astype(np.float64)
    qv = orc.selected_values(zq, summ)[:, :summ["l"]]
    W = orc.words(z, summ)
    for i in range(q.shape[0]):
        ed2 = orc.sqdist(z, zq[i])
        assert np.all(lb[i] <= ed2 * (1 + 1e-5)), "GPU bound above the true distance"
        olb = orc.lb2(qv[i], W, summ)
        assert np.all(lb[i][words_equal] <= olb[words_equal] * (1 + 1e-5) + 1e-6)
        assert np.mean(lb[i][words_equal] >= 0.98 * olb[words_equal] - 0.05) > 0.99


OPTIONS = [
    # binning, select, pool_coeffs
    ("equi-width", "variance", 0),
    ("equi-depth", "first", 0),
    ("equi-depth", "variance", 16),
    ("equi-width", "first", 16),
]


@pytest.mark.parametrize("binning,select,pool", OPTIONS)
def test_build_options_match_oracle(sofa, binning, select, pool):
    N, n, l, alpha, ratio = 20000, 128, 16, 256, 0.1
    x = datagen.mixed_walks(N, n, seed=301, device=DEV)
    xc = x.cpu().numpy()
    ix = sofa.Index(x, l, alpha, sample_ratio=ratio, binning=binning, select=select, pool_coeffs=pool,
                    precision=1)
    inf = ix.info()
    delta = inf["delta_data"]
    # the learned summary: the same selection, variances and breakpoints
    osum = orc.learn_summary(xc, l, alpha, ratio=ratio, binning=binning, select=select, pool=pool)
    sel, var, beta = ix.summary()
    assert np.array_equal(sel.numpy(), osum["ids"])
    assert np.allclose(var.numpy(), osum["var"], rtol=1e-5)
    gb = beta.numpy().astype(np.float64)[:, 1:alpha]
    ob = osum["beta"].astype(np.float64)[:, 1:alpha]
    # each breakpoint is a sample value (equi-depth) or min + a (max - min) / alpha
    # (equi-width) of values computed in FP32 on the GPU, FP64 in the oracle:
    # within the projection margin, plus the rounding of the stored fp32
    tol = delta + 4 * np.finfo(np.float32).eps * np.abs(ob)
    assert np.all(np.abs(gb - ob) <= tol), np.max(np.abs(gb - ob) - tol)
    if binning == "equi-width":
        step = np.diff(ob, axis=1)
        assert np.allclose(step, step[:, :1], rtol=1e-4)
    if select == "first":
        assert np.array_equal(sel.numpy(), np.arange(len(sel)))
    # words and bounds under the GPU's own summary
    z, _, _ = orc.znorm(xc)
    gsum = summary_from_gpu(ix, n, l, alpha, pool)
    gw, ow = check_words(ix, z, gsum, delta)
    q = datagen.half_perturbed_queries(x, 24, seed=302)
    zq, _, _ = orc.znorm(q.cpu().numpy())
    check_bounds(ix, z, zq, q, gsum, np.all(gw == ow, axis=1))
    # exact k-NN in the plain and the filtered forms
    oi, od = oracle_knn(x, q, 5)
    for t in (dict(dense=1), dict(dense=1, refine_filter=2, bound_precision=1)):
        ix.set_tuning(**t)
        gi, gd = ix.query(q, 5)
        torch.cuda.synchronize()
        assert ix.status() == 0
        assert_knn_equal(gi, gd, oi, od)
    ix.close()


@pytest.mark.parametrize("N,n,l,k,amp", [(20000, 128, 16, 1, 5.0), (15000, 128, 16, 10, 5.0),
                                         (12000, 256, 32, 3, 8.0)])
def test_planted_nyquist_value(sofa, N, n, l, k, amp):
    alpha = 256
    x = datagen.alternating_walks(N, n, amp, seed=310 + n + l, device=DEV)
    xc = x.cpu().numpy()
    osum = orc.learn_summary(xc, l, alpha, ratio=0.1)
    assert osum["ks"][0] == n // 2 and osum["parts"][0] == 0 and osum["w"][0] == 1.0
    ix = sofa.Index(x, l, alpha, sample_ratio=0.1, precision=1)
    inf = ix.info()
    assert inf["nyquist_first"] == 1
    sel, _, _ = ix.summary()
    assert np.array_equal(sel.numpy()[:l], osum["ids"][:l])
    z, _, _ = orc.znorm(xc)
    gsum = summary_from_gpu(ix, n, l, alpha, 0)
    gw, ow = check_words(ix, z, gsum, inf["delta_data"])
    q = datagen.half_perturbed_queries(x, 24, seed=311)
    zq, _, _ = orc.znorm(q.cpu().numpy())
    check_bounds(ix, z, zq, q, gsum, np.all(gw == ow, axis=1))
    oi, od = oracle_knn(x, q, k)
    for t in (dict(dense=1), dict(dense=1, bound_precision=1), dict(dense=1, refine_filter=2),
              dict(dense=1, cand_cap=3, pool_cap=7, group=5)):
        ix.set_tuning(**t)
        gi, gd = ix.query(q, k)
        torch.cuda.synchronize()
        assert ix.status() == 0, t
        assert_knn_equal(gi, gd, oi, od)
    ix.close()
