"""The tensor-core series bound (series_bound = 1), CUDA path vs the CPU oracle.

Eq. (1) restricted to the selected Fourier values, from int8 value codes, as
one tcgen05 contraction per (work unit, tile) with a derived FP16 margin:
* every pair's bound (sofa_value_bounds) is at most the oracle's FP64 value
  of Eq. (1) on the selected values, and close to it (a wrong operand layout
  or descriptor would break either side);
* exact k-NN answers equal the oracle's brute force over many shapes,
  tunings and the Nyquist word value;
* the bound prunes more than the SFA word bound on random walks.
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


def assert_knn_equal(gi, gd, oi, od):
    gi = gi.cpu().numpy()
    gd = gd.cpu().numpy().astype(np.float64)
    bad = np.nonzero(np.any(gi != oi, axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} queries differ, first {bad[:5]}: gpu {gi[bad[0]]} oracle {oi[bad[0]]}"
    rel = np.abs(gd - od) / np.maximum(od, 1e-30)
    assert rel.max() <= 1e-4
    assert np.array_equal(gd.astype(np.float32), od.astype(np.float32))


def gpu_summary(ix, n, l, alpha):
    sel, var, beta = ix.summary()
    tab = orc.value_table(n, 0)
    ids = sel.numpy().astype(np.int32)
    ks = np.array([tab[c][0] for c in ids], np.int32)
    parts = np.array([tab[c][1] for c in ids], np.int32)
    w = np.array([orc.weight(n, int(kk)) for kk in ks], np.float64)
    return dict(ids=ids, ks=ks, parts=parts, w=w, var=var.numpy(), beta=beta.numpy(), n=n, l=l, alpha=alpha)


def make(gen, N, n, seed):
    if gen == "rw":
        return datagen.random_walks(N, n, seed=seed, device=DEV)
    if gen == "mixed":
        return datagen.mixed_walks(N, n, seed=seed, device=DEV)
    if gen == "nyq":
        return datagen.alternating_walks(N, n, 5.0, seed=seed, device=DEV)
    return datagen.sinusoid_mix(N, n, seed=seed, device=DEV)


@pytest.mark.parametrize("gen,N,n,l", [("rw", 20000, 128, 16), ("mixed", 9000, 256, 16), ("nyq", 7000, 128, 16),
                                       ("rw", 6000, 256, 32), ("sin", 5000, 128, 12), ("rw", 777, 64, 8)])
def test_value_bounds_are_tight_lower_bounds(sofa, gen, N, n, l):
    x = make(gen, N, n, seed=601 + N)
    q = datagen.half_perturbed_queries(x, 70, seed=602)           # 70 queries: two column groups
    ix = sofa.Index(x, l, 256, precision=1)
    lb, M = sofa.value_bounds(ix, q)
    torch.cuda.synchronize()
    lb = lb.cpu().numpy().astype(np.float64)
    assert 0.0 < M < 2e-3 * n
    summ = gpu_summary(ix, n, l, 256)
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    v = orc.selected_values(z, summ)
    qv = orc.selected_values(zq, summ)
    assert np.all(np.isfinite(lb)) and np.all(lb >= 0)
    for i in range(q.shape[0]):
        exact = orc.dft_lb2(qv[i], v, summ["w"])              # Eq. (1) on the selected values, FP64
        ed2 = orc.sqdist(z, zq[i])
        assert np.all(exact <= ed2 * (1 + 1e-9) + 1e-9)        # the oracle's own invariant
        assert np.all(lb[i] <= exact * (1 + 1e-6) + 1e-6), "tensor-core bound above Eq. (1)"
        # tight: the codes' margin r and M' cost a fraction of a distance unit
        far = exact > 4.0
        assert np.mean(lb[i][far] >= (np.sqrt(exact[far]) - 1.0) ** 2) > 0.99
    ix.close()


CASES = [
    # N, n, l, k, Q, generator
    (20000, 128, 16, 1, 64, "rw"),
    (20000, 256, 16, 5, 48, "mixed"),
    (12345, 64, 8, 10, 32, "rw"),
    (9000, 96, 16, 50, 16, "sin"),
    (8000, 256, 32, 3, 40, "rw"),
    (6000, 128, 16, 4, 40, "nyq"),
    (257, 32, 4, 3, 8, "rw"),
    (100, 16, 6, 64, 4, "rw"),
    (1, 8, 4, 1, 3, "rw"),
]


@pytest.mark.parametrize("N,n,l,k,Q,gen", CASES)
def test_knn_with_tensor_core_bound_matches_oracle(sofa, N, n, l, k, Q, gen):
    k = min(k, N)
    x = make(gen, N, n, seed=N + n + 3)
    q = datagen.half_perturbed_queries(x, Q, seed=5) if N > 10 else datagen.random_walks(Q, n, seed=9, device=DEV)
    ix = sofa.Index(x, l, 256, precision=1)
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, k)
    for t in (dict(series_bound=1, dense=1), dict(series_bound=1, dense=1, refine_filter=2),
              dict(series_bound=1, dense=1, refine_filter=1, cand_cap=3, pool_cap=7, group=5),
              dict(series_bound=1, dense=1, group=64, cand_cap=1),
              dict(series_bound=1, dense=1, tile_checks=1), dict(series_bound=1, dense=1, tile_checks=1, group=7)):
        ix.set_tuning(**t)
        gi, gd = ix.query(q, k)
        torch.cuda.synchronize()
        assert ix.status() == 0, t
        assert_knn_equal(gi, gd, oi, od)
    ix.close()


def test_tensor_core_bound_prunes_more_than_the_word_bound(sofa):
    N, n = 200_000, 256
    x = datagen.random_walks(N, n, seed=611, device=DEV)
    q = datagen.random_walks(200, n, seed=612, device=DEV)
    ix = sofa.Index(x, 16, 256, precision=1)
    res = {}
    for sb in (0, 1):
        ix.set_tuning(series_bound=sb, dense=1, tile_checks=1)
        ix.stats(reset=True)
        gi, gd = ix.query(q, 1)
        torch.cuda.synchronize()
        assert ix.status() == 0
        res[sb] = (gi, gd, ix.stats())
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    # the same (query, tile) pairs are bounded; far fewer series survive
    assert res[1][2]["tile_pairs"] == res[0][2]["tile_pairs"]
    assert res[1][2]["candidates"] * 3 < res[0][2]["candidates"], (res[0][2]["candidates"], res[1][2]["candidates"])
    sub = list(range(0, 200, 20))
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q[sub].cpu().numpy())
    oi, od = orc.knn(z, zq, 1)
    assert_knn_equal(res[1][0][sub], res[1][1][sub], oi, od)
    ix.close()


def test_tensor_core_bound_with_graphs_insert_and_learned_seed(sofa):
    n = 128
    x0 = datagen.random_walks(30000, n, seed=621, device=DEV)
    x1 = datagen.mixed_walks(5000, n, seed=622, device=DEV)
    ix = sofa.Index(x0, 16, 256, precision=1)
    ix.train_proposal(n_train=16384, n_classes=64, epochs=2, batch=2048, seed=2, top_m=4)
    ix.insert(x1)
    X = torch.cat([x0, x1])
    q = torch.cat([datagen.perturbed_members(x1, 12, seed=623)[0], datagen.half_perturbed_queries(x0, 20, seed=624)])
    z, _, _ = orc.znorm(X.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, 3)
    for mode in (0, 1):
        ix.set_seed_mode(mode)
        ix.set_tuning(series_bound=1, refine_filter=2, use_graph=1)
        for _ in range(2):                          # recorded, then replayed
            gi, gd = ix.query(q, 3)
            torch.cuda.synchronize()
            assert ix.status() == 0
            assert_knn_equal(gi, gd, oi, od)
    assert ix.stats()["graph_replays"] >= 1
    ix.close()


def test_series_bound_needs_the_value_codes(sofa):
    x = datagen.random_walks(3000, 64, seed=631, device=DEV)
    ix = sofa.Index(x, 8, 256)                      # precision 0: no value codes
    with pytest.raises(sofa.SofaError) as e:
        ix.set_tuning(series_bound=1)
    assert e.value.code == -1
    with pytest.raises(sofa.SofaError):
        sofa.value_bounds(ix, x[:2])
    ix.close()


def test_tile_checks_keep_answers_and_only_skip_tiles(sofa):
    """With the tensor-core bound the per-tile envelope checks are optional:
    on or off, the answers equal the oracle's; with them on, no more tiles
    are loaded than with them off, and every tile of a routed leaf block is
    loaded when they are off."""
    N, n = 60000, 128
    x = datagen.random_walks(N, n, seed=641, device=DEV)
    q = datagen.half_perturbed_queries(x, 96, seed=642)
    ix = sofa.Index(x, 16, 256, precision=1)
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, 2)
    loads = {}
    for tc in (0, 1):
        ix.set_tuning(series_bound=1, dense=1, refine_filter=2, tile_checks=tc)
        ix.stats(reset=True)
        ix.profile(reset=True)
        ix.set_profiling(True)
        gi, gd = ix.query(q, 2)
        torch.cuda.synchronize()
        assert ix.status() == 0
        assert_knn_equal(gi, gd, oi, od)
        loads[tc] = ix.profile(reset=True)["scan_tile_loads"]
        ix.set_profiling(False)
    assert 0 < loads[1] <= loads[0]
    with pytest.raises(sofa.SofaError):
        ix.set_tuning(series_bound=1, tile_checks=2)
    ix.close()
