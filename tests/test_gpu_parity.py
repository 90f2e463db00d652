"""CUDA path vs the CPU oracle, element by element, on seeded synthetic inputs."""
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
    # the final re-score is the oracle's FP64 sum: equal after rounding to fp32
    assert np.array_equal(gd.astype(np.float32), od.astype(np.float32))


# ------------------------------------------------------------------ z-norm
def test_znorm_bit_exact(sofa):
    x = datagen.random_walks(3000, 200, seed=3, device=DEV)
    x[7] = 5.0                                      # constant row
    z = sofa.znorm(x)
    zo, _, _ = orc.znorm(x.cpu().numpy())
    assert np.array_equal(z.cpu().numpy(), zo)


# ------------------------------------------------------------------ summary
def test_learned_summary_matches_oracle(sofa):
    N, n, l, alpha = 20000, 128, 16, 256
    x = datagen.random_walks(N, n, seed=5, device=DEV)
    ix = sofa.Index(x, l, alpha, sample_ratio=0.1)
    sel, var, beta = ix.summary()
    summ = orc.learn_summary(x.cpu().numpy(), l, alpha, ratio=0.1)
    assert np.array_equal(sel.numpy()[:l], summ["ids"][:l])
    assert np.allclose(var.numpy(), summ["var"], rtol=1e-5)
    # equi-depth breakpoints: GPU values are sample values of the FP32 transform;
    # each must lie within a few ulps of the oracle's FP64 sample quantile
    ob = summ["beta"].astype(np.float64)
    gb = beta.numpy().astype(np.float64)
    inner = slice(1, alpha)
    assert np.allclose(gb[:, inner], ob[:, inner], rtol=0, atol=1e-4)
    ix.close()


# ------------------------------------------------------------------ words
@pytest.mark.parametrize("n,l,alpha", [(64, 8, 4), (128, 16, 256), (256, 16, 256), (1024, 32, 256)])
def test_words_match_oracle_with_oracle_bins(sofa, n, l, alpha):
    N = 6000
    x = datagen.random_walks(N, n, seed=n + l, device=DEV)
    xc = x.cpu().numpy()
    summ = orc.learn_summary(xc, l, alpha, ratio=0.1)
    ix = sofa.Index(x, l, alpha, user_sel=summ["ids"], user_beta=summ["beta"])
    inf = ix.info()
    gw = ix.words().numpy()
    z, _, _ = orc.znorm(xc)
    ow = orc.words(z, summ)
    v = orc.selected_values(z, summ)[:, :l]
    diff = gw != ow
    # allowed only where the FP64 value lies within the projection margin of a breakpoint
    for r, j in zip(*np.nonzero(diff)):
        b = summ["beta"][j].astype(np.float64)
        near = np.min(np.abs(b[1:-1] - v[r, j]))
        assert near <= inf["delta_data"], (r, j, near)
        assert abs(int(gw[r, j]) - int(ow[r, j])) == 1
    # equi-depth breakpoints are values of sampled series (every 10th row), so
    # those rows sit exactly on breakpoints; elsewhere differences are rare
    unsampled = np.arange(N) % orc.sample_stride(0.1) != 0
    assert diff[unsampled].mean() < 2e-3
    ix.close()


# ------------------------------------------------------------------ lower bounds
@pytest.mark.parametrize("gen", ["rw", "sin"])
def test_lower_bounds_never_exceed_distance(sofa, gen):
    N, n, l = 8000, 128, 16
    if gen == "rw":
        x = datagen.random_walks(N, n, seed=11, device=DEV)
    else:
        x = datagen.sinusoid_mix(N, n, seed=11, device=DEV)
    q = x[:24].clone() + 0.05 * torch.randn(24, n, device=DEV, generator=torch.Generator(DEV).manual_seed(1))
    xc = x.cpu().numpy()
    summ = orc.learn_summary(xc, l, 256, ratio=0.1)
    ix = sofa.Index(x, l, 256, user_sel=summ["ids"], user_beta=summ["beta"])
    lb = ix.lower_bounds(q).cpu().numpy().astype(np.float64)
    z, _, _ = orc.znorm(xc)
    zq, _, _ = orc.znorm(q.cpu().numpy())
    W = orc.words(z, summ)
    same = np.all(ix.words().numpy() == W, axis=1)     # rows whose GPU word is the oracle's
    assert same.mean() > 0.9
    qv = orc.selected_values(zq, summ)[:, :l]
    for i in range(q.shape[0]):
        ed2 = orc.sqdist(z, zq[i])
        assert np.all(lb[i] <= ed2 * (1 + 1e-5)), "GPU bound above the true distance"
        olb = orc.lb2(qv[i], W, summ)
        # same word: the GPU bound is the oracle's bound with widened intervals
        assert np.all(lb[i][same] <= olb[same] * (1 + 1e-5) + 1e-6)
        assert np.mean(lb[i][same] >= 0.98 * olb[same] - 0.05) > 0.99
    ix.close()


# ------------------------------------------------------------------ exact k-NN
CASES = [
    # N, n, l, alpha, k, Q, generator
    (20000, 128, 16, 256, 1, 64, "rw"),
    (20000, 256, 16, 256, 5, 48, "mixed"),
    (12345, 64, 8, 4, 10, 32, "rw"),
    (9000, 96, 16, 16, 50, 16, "sin"),
    (30000, 1024, 32, 256, 1, 16, "sin"),
    (257, 32, 4, 256, 3, 8, "rw"),
    (100, 16, 6, 2, 64, 4, "rw"),
    (1, 8, 4, 256, 1, 3, "rw"),
]


def make(gen, N, n, seed):
    if gen == "rw":
        return datagen.random_walks(N, n, seed=seed, device=DEV)
    if gen == "mixed":
        return datagen.mixed_walks(N, n, seed=seed, device=DEV)
    return datagen.sinusoid_mix(N, n, seed=seed, device=DEV)


@pytest.mark.parametrize("N,n,l,alpha,k,Q,gen", CASES)
def test_knn_matches_oracle(sofa, N, n, l, alpha, k, Q, gen):
    k = min(k, N)
    x = make(gen, N, n, seed=N + n)
    if N > 10:
        q = datagen.half_perturbed_queries(x, Q, seed=1)
    else:
        q = datagen.random_walks(Q, n, seed=9, device=DEV)
    ix = sofa.Index(x, l, alpha)
    gi, gd = ix.query(q, k)
    torch.cuda.synchronize()
    assert ix.status() == 0
    oi, od = oracle_knn(x, q, k)
    assert_knn_equal(gi, gd, oi, od)
    ix.close()


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("N,n,l,alpha,k,Q,gen", [CASES[1], CASES[3], CASES[4], CASES[5]])
def test_knn_reduced_precision_match_oracle(sofa, N, n, l, alpha, k, Q, gen, level):
    """FP16x2 series bounds and the refinement filters (int8 rows; value
    codes then int8 rows), each with its derived margin: the same exact
    answers."""
    x = make(gen, N, n, seed=N + n + 1)
    q = datagen.half_perturbed_queries(x, Q, seed=4)
    ix = sofa.Index(x, l, alpha, precision=1)
    ix.set_tuning(bound_precision=1, refine_filter=level)
    gi, gd = ix.query(q, k)
    oi, od = oracle_knn(x, q, k)
    assert_knn_equal(gi, gd, oi, od)
    assert ix.status() == 0
    ix.close()


def test_duplicates_and_member_queries(sofa):
    N, n = 5000, 64
    x = datagen.random_walks(N, n, seed=21, device=DEV)
    x[4000] = x[17]
    x[4001] = x[17] * 3.0 + 1.0                    # same after z-normalisation
    x[2] = x[17] + 1e-7
    q = torch.stack([x[17], x[100], x[4001] + 0.001])
    ix = sofa.Index(x, 8, 256)
    gi, gd = ix.query(q, 5)
    oi, od = oracle_knn(x, q, 5)
    assert_knn_equal(gi, gd, oi, od)
    assert gi[0, 0].item() == 17 and gd[0, 0].item() == 0.0
    ix.close()


@pytest.mark.parametrize("tuning", [dict(group=1), dict(group=64), dict(cand_cap=1), dict(cand_cap=7, group=3),
                                    dict(cand_cap=3, pool_cap=5), dict(cand_cap=64, pool_cap=1),
                                    dict(seed_count=1), dict(seed_count=256), dict(seed_window=4096, seed_count=128),
                                    dict(seed_window=256), dict(bound_precision=1),
                                    dict(bound_precision=1, cand_cap=5, group=7), dict(refine_filter=1),
                                    dict(refine_filter=1, bound_precision=1, cand_cap=9, pool_cap=40),
                                    dict(refine_filter=2), dict(refine_filter=2, cand_cap=3, pool_cap=5),
                                    dict(cand_cap=2, pool_cap=3, cand_budget=4),
                                    dict(refine_filter=2, cand_cap=1, pool_cap=1, cand_budget=1),
                                    dict(dense=2), dict(dense=2, cand_cap=2, pool_cap=3),
                                    dict(dense=2, refine_filter=2, cand_cap=3, pool_cap=7, cand_budget=6)])
def test_tuning_invariance(sofa, tuning):
    N, n = 15000, 128
    x = datagen.mixed_walks(N, n, seed=31, device=DEV)
    q = datagen.half_perturbed_queries(x, 40, seed=2)
    ix = sofa.Index(x, 16, 256, leaf_tiles=4, precision=1)
    gi0, gd0 = ix.query(q, 10)
    t = dict(tuning)
    if "pool_cap" in t and "dense" not in t:
        t["dense"] = 1             # the series scan, whose candidates overflow the tiny pool
    ix.set_tuning(**t)
    ix.stats(reset=True)
    gi1, gd1 = ix.query(q, 10)
    assert torch.equal(gi0, gi1) and torch.equal(gd0, gd1)
    if "pool_cap" in t and t["dense"] == 1:   # a full pool: the queries concerned are scanned again
        assert ix.stats()["overflow_passes"] > 0
    ix.close()


def test_value_code_filter_prunes(sofa):
    """The value-code bound drops most candidates before any int8 row is read,
    and the answers stay those of the oracle."""
    N, n = 60000, 256
    x = datagen.random_walks(N, n, seed=41, device=DEV)
    q = datagen.random_walks(64, n, seed=42, device=DEV)
    ix = sofa.Index(x, 16, 256, precision=1)
    ix.set_tuning(refine_filter=2, dense=1)   # the series scan's candidates (the dense form's are near-exact)
    ix.stats(reset=True)
    gi, gd = ix.query(q, 3)
    st = ix.stats()
    assert ix.status() == 0
    assert st["value_filtered"] > 0
    oi, od = oracle_knn(x, q, 3)
    assert_knn_equal(gi, gd, oi, od)
    ix.close()


def test_host_buffers_and_batches(sofa):
    N, n = 10000, 64
    x = datagen.random_walks(N, n, seed=41, device=DEV)
    q = datagen.random_walks(9000, n, seed=42, device=DEV)      # > one internal batch
    ix = sofa.Index(x.cpu(), 8, 256)                             # host data
    gi, gd = ix.query(q, 2)
    hi, hd = ix.query(q.cpu(), 2)                                # host queries and outputs
    assert hi.device.type == "cpu"
    assert torch.equal(gi.cpu(), hi) and torch.equal(gd.cpu(), hd)
    sub = torch.arange(0, 9000, 450)
    oi, od = oracle_knn(x, q[sub], 2)
    assert_knn_equal(gi[sub], gd[sub], oi, od)
    ix.close()


def test_query_multi(sofa):
    xs = [datagen.random_walks(4000, n, seed=n, device=DEV) for n in (32, 64, 128)]
    ixs = [sofa.Index(x, 8, 256) for x in xs]
    g = torch.Generator().manual_seed(0)
    lens = [32, 64, 128][0:3]
    qs, offs, ql, qk, oo = [], [], [], [], []
    pos = out = 0
    for i in range(30):
        n = lens[int(torch.randint(0, 3, (1,), generator=g))]
        k = [1, 5, 10][i % 3]
        qs.append(datagen.random_walks(1, n, seed=100 + i, device=DEV)[0])
        offs.append(pos)
        ql.append(n)
        qk.append(k)
        oo.append(out)
        pos += n
        out += k
    packed = torch.cat(qs)
    idx, dist = sofa.query_multi(ixs, packed, offs, ql, qk, oo, out)
    for i in range(30):
        x = xs[lens.index(ql[i])]
        oi, od = oracle_knn(x, qs[i][None, :], qk[i])
        assert_knn_equal(idx[oo[i]:oo[i] + qk[i]][None, :], dist[oo[i]:oo[i] + qk[i]][None, :], oi, od)
    for ix in ixs:
        ix.close()


def test_autotune_keeps_answers_and_caches(sofa, tmp_path):
    N, n = 40000, 128
    x = datagen.random_walks(N, n, seed=61, device=DEV)
    q = datagen.half_perturbed_queries(x, 64, seed=62)
    ix = sofa.Index(x, 16, 256, precision=1)
    gi0, gd0 = ix.query(q, 3)
    cache = str(tmp_path / "tune.txt")
    t1 = ix.autotune(q, 3, cache)
    gi1, gd1 = ix.query(q, 3)
    assert torch.equal(gi0, gi1) and torch.equal(gd0, gd1)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    ix.set_tuning()                          # back to defaults, then a cache hit
    t2 = ix.autotune(q, 3, cache)
    assert t1 == t2 and len(open(cache).read().splitlines()) == 1
    ix.close()


@pytest.mark.parametrize("extra", [dict(), dict(pool_cap=3, cand_cap=2), dict(refine_filter=1)])
def test_graph_replay_matches_eager(sofa, extra):
    N, n = 50000, 128
    x = datagen.mixed_walks(N, n, seed=71, device=DEV)
    ix = sofa.Index(x, 16, 256, precision=1)
    batches = [datagen.half_perturbed_queries(x, 96, seed=72 + i) for i in range(4)]
    ix.set_tuning(**extra)
    eager = [ix.query(q, 4) for q in batches]
    ix.set_tuning(use_graph=1, **extra)
    for _ in range(2):                      # first call records, later calls replay
        for q, (ei, ed) in zip(batches, eager):
            gi, gd = ix.query(q, 4)
            torch.cuda.synchronize()
            assert torch.equal(gi, ei) and torch.equal(gd, ed)
    assert ix.status() == 0
    st = ix.stats()
    assert st["graphs_recorded"] >= 1 and st["graph_replays"] >= 4
    ix.close()


def test_approximate_mode(sofa):
    """The approximate search alone (no pruning scan): every answer is a real
    distance of the returned series, never better than the exact k-th, and
    most perturbed-member queries find their source row."""
    N, n, k = 50000, 128, 5
    x = datagen.random_walks(N, n, seed=81, device=DEV)
    q = datagen.half_perturbed_queries(x, 64, seed=82)
    ix = sofa.Index(x, 16, 256)
    ge, gde = ix.query(q, k)
    ix.set_tuning(approximate=1)
    ga, gda = ix.query(q, k)
    torch.cuda.synchronize()
    assert ix.status() == 0
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    ga_n, gda_n = ga.cpu().numpy(), gda.cpu().numpy()
    for i in range(q.shape[0]):
        d = np.sqrt(orc.sqdist(z[ga_n[i]], zq[i]))
        assert np.array_equal(d.astype(np.float32), gda_n[i])
    assert bool(torch.all(gda[:, -1] >= gde[:, -1] * (1 - 1e-6)))
    # half the queries are perturbed members: their 1-NN is usually the key window's
    hit = np.mean([ge[i, 0].item() in set(ga_n[i]) for i in range(32)])
    assert hit >= 0.5
    ix.set_tuning()
    gi, gd = ix.query(q, k)                  # back to exact
    assert torch.equal(gi, ge) and torch.equal(gd, gde)
    ix.close()


def test_save_load_roundtrip(sofa, tmp_path):
    """An index written by sofa_save and read by sofa_load answers exactly as
    the original, in every precision and seed mode."""
    N, n = 30000, 128
    x = datagen.random_walks(N, n, seed=91, device=DEV)
    q = datagen.half_perturbed_queries(x, 40, seed=92)
    ix = sofa.Index(x, 16, 256, precision=2)      # every optional copy, FP16 included
    ix.train_proposal(n_train=8192, n_classes=64, epochs=1, batch=2048, seed=2, top_m=4)
    path = str(tmp_path / "index.sofa")
    ix.save(path)
    iy = sofa.Index.load(path)
    assert iy.info()["N"] == N and iy.info()["proposal_classes"] == 64
    assert torch.equal(iy.perm(), ix.perm()) and torch.equal(iy.words(), ix.words())
    oi, od = oracle_knn(x, q, 4)
    for tuning, seed_mode in ((dict(), 0), (dict(refine_filter=2), 1), (dict(approximate=1), 1), (dict(dense=2), 0)):
        for h in (ix, iy):
            h.set_seed_mode(seed_mode)
            h.set_tuning(**tuning)
        a = ix.query(q, 4)
        b = iy.query(q, 4)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), tuning
        if not tuning.get("approximate"):
            assert_knn_equal(b[0], b[1], oi, od)   # the loaded index answers the oracle's k-NN
    ix.close()
    iy.close()


def test_unprunable_data_on_the_scan_path(sofa):
    """High-frequency data where the bound prunes nothing, forced through the
    series scan with a tiny pool and region budget: the pool counter stops at
    its capacity, overflow passes regrow the regions (a few queries at a time),
    and the answers are the oracle's."""
    N, n, Q, k = 20000, 256, 24, 3
    x = datagen.sinusoid_mix(N, n, seed=95, device=DEV)
    q = datagen.sinusoid_mix(Q, n, seed=96, device=DEV)
    ix = sofa.Index(x, 16, 256)
    ix.set_tuning(dense=1, cand_cap=16, pool_cap=500, cand_budget=4096)
    ix.stats(reset=True)
    gi, gd = ix.query(q, k)
    torch.cuda.synchronize()
    assert ix.status() == 0
    assert ix.stats()["overflow_passes"] >= 3
    oi, od = oracle_knn(x, q, k)
    assert_knn_equal(gi, gd, oi, od)
    ix.close()
