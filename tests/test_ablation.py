"""The summarisation ablation's CPU iSAX baseline, pinned by its definition
(PAA means, equiprobable N(0,1) breakpoints, LB <= ED), and the GPU harness
on a small case."""
import statistics

import numpy as np
import pytest
import torch

from oracle import sofa_oracle as orc
from paper_2411_17483_gb300 import ablation


def rw(N, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal((N, n)), axis=1).astype(np.float32)


def test_paa_is_segment_mean():
    z, _, _ = orc.znorm(rw(50, 64, 1))
    p = ablation.paa(z, 8)
    for i in (0, 17, 49):
        for s in range(8):
            assert p[i, s] == pytest.approx(float(np.mean(z[i, 8 * s:8 * s + 8].astype(np.float64))), abs=1e-12)


def test_breakpoints_are_equiprobable():
    b = ablation.gaussian_breakpoints(16)
    assert b[0] == -np.inf and b[-1] == np.inf and len(b) == 17
    nd = statistics.NormalDist()
    for a in range(1, 16):
        assert nd.cdf(b[a]) == pytest.approx(a / 16, abs=1e-12)
    assert np.allclose(b[1:8], -b[15:8:-1])   # symmetric


@pytest.mark.parametrize("w,alpha", [(16, 256), (8, 4), (64, 2)])
def test_isax_bound_never_exceeds_distance(w, alpha):
    z, _, _ = orc.znorm(rw(3000, 64, 2))
    zq, _, _ = orc.znorm(rw(20, 64, 3))
    beta = ablation.gaussian_breakpoints(alpha)
    words = ablation.isax_words(ablation.paa(z, w), beta)
    qp = ablation.paa(zq, w)
    for i in range(20):
        lb2 = ablation.isax_lb(qp[i], words, beta, 64)
        d2 = orc.sqdist(z, zq[i])
        assert np.all(lb2 <= d2 * (1 + 1e-12) + 1e-12)


def test_isax_bound_approaches_distance_with_full_resolution():
    # one segment per value and a very fine alphabet: the bound tends to ED^2
    z, _, _ = orc.znorm(rw(200, 16, 4))
    beta = ablation.gaussian_breakpoints(1 << 16)
    words = ablation.isax_words(ablation.paa(z, 16), beta)
    lb2 = ablation.isax_lb(z[0].astype(np.float64) + 0.5, words, beta, 16)
    d2 = ((z.astype(np.float64) - (z[0].astype(np.float64) + 0.5)) ** 2).sum(1)
    assert np.all(lb2 <= d2) and np.all(lb2 >= 0.95 * d2 - 1e-3)


def test_measures_definition():
    lb2 = torch.tensor([[1.0, 4.0, 0.0], [9.0, 0.25, 1.0]], dtype=torch.float64)
    d2 = torch.tensor([[4.0, 4.0, 1.0], [9.0, 1.0, 4.0]], dtype=torch.float64)
    tlb, prune = ablation.measures(lb2, d2)
    assert tlb == pytest.approx((0.5 + 1.0 + 0.0 + 1.0 + 0.5 + 0.5) / 6)
    # 1-NN distances 1 and 1: bounds above them are 2 (row 0) and 3 (row 1)
    assert prune == pytest.approx(2 / 6)


@pytest.mark.gpu
def test_ablation_harness_small():
    rows = ablation.run(N=20000, n=64, Q=10, l=8, ratios=(0.1,), isax_segments=8)
    assert len(rows) == 5
    for r in rows:
        assert 0.0 < r["tlb"] <= 1.0 + 1e-9 and 0.0 <= r["pruning"] <= 1.0
    text = ablation.table(rows, "t")
    assert text.count("\n| ") == 6


@pytest.mark.gpu
@pytest.mark.parametrize("binning,select", [("equi-depth", "variance"), ("equi-width", "first")])
def test_ablation_sfa_measures_match_oracle(binning, select):
    """The harness's SFA measures (the library's bounds, the GPU's FP64
    distances) against the oracle's: its Eq. (1) SFA bound (orc.lb2) on the
    oracle's words under the same summary, and its brute-force distances."""
    from paper_2411_17483_gb300 import datagen, sofa
    N, n, Q, l = 20000, 64, 10, 8
    dev = "cuda:0"
    x = datagen.random_walks(N, n, seed=71, device=dev)
    q = datagen.random_walks(Q, n, seed=72, device=dev)
    ix = sofa.Index(x, l, 256, sample_ratio=0.1, binning=binning, select=select)
    z_gpu = sofa.znorm(x)
    zq_gpu = sofa.znorm(q)
    d2 = ablation.exact_sqdist(zq_gpu, z_gpu)
    tlb_g, prune_g = ablation.measures(ix.lower_bounds(q).double(), d2)
    # the oracle under the GPU's summary
    sel, var, beta = ix.summary()
    tab = orc.value_table(n, 0)
    ids = sel.numpy().astype(np.int32)
    ks = np.array([tab[c][0] for c in ids], np.int32)
    parts = np.array([tab[c][1] for c in ids], np.int32)
    summ = dict(ids=ids, ks=ks, parts=parts, w=np.array([orc.weight(n, int(k)) for k in ks]),
                var=var.numpy(), beta=beta.numpy(), n=n, l=l, alpha=256)
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    W = orc.words(z, summ)
    qv = orc.selected_values(zq, summ)[:, :l]
    olb2 = np.stack([orc.lb2(qv[i], W, summ) for i in range(Q)])
    od2 = np.stack([orc.sqdist(z, zq[i]) for i in range(Q)])
    # the harness's distances are the oracle's
    assert np.allclose(d2.cpu().numpy(), od2, rtol=1e-9, atol=1e-9)
    tlb_o, prune_o = ablation.measures(torch.from_numpy(olb2), torch.from_numpy(od2))
    # the library's bounds carry the projection margins: never above the
    # oracle's, and within a hair of them
    assert tlb_g <= tlb_o + 1e-6 and tlb_g >= tlb_o - 2e-3, (tlb_g, tlb_o)
    assert prune_g <= prune_o + 1e-3 and prune_g >= prune_o - 5e-3, (prune_g, prune_o)
    ix.close()
