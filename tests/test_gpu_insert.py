"""Incremental insert (sofa_insert), CUDA path vs the CPU oracle.

An index is built on one batch of series and grown by two more batches, one
from device and one from host memory, of other generators and ragged sizes.
The exact k-NN over the union (new rows numbered after the old ones) must be
the oracle's brute force over the concatenated collection: in the series
scan, the filtered scan, the dense contraction and the learned seed, and
after the grown index is saved and loaded again.  The words of the new rows
are the oracle's under the index's summary, and the bounds stay below the
distances."""
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


def summary_record(ix, n, l, alpha):
    sel, var, beta = ix.summary()
    tab = orc.value_table(n, 0)
    ids = sel.numpy().astype(np.int32)
    ks = np.array([tab[c][0] for c in ids], np.int32)
    parts = np.array([tab[c][1] for c in ids], np.int32)
    w = np.array([orc.weight(n, int(kk)) for kk in ks], np.float64)
    return dict(ids=ids, ks=ks, parts=parts, w=w, var=var.numpy(), beta=beta.numpy(), n=n, l=l, alpha=alpha)


def grown_workload():
    n = 128
    x0 = datagen.random_walks(30000, n, seed=501, device=DEV)
    x1 = datagen.mixed_walks(7000, n, seed=502, device=DEV)
    x2 = datagen.random_walks(1234, n, seed=503, device=DEV)
    X = torch.cat([x0, x1, x2])
    q = torch.cat([datagen.perturbed_members(x1, 16, seed=504)[0], datagen.perturbed_members(x2, 8, seed=505)[0],
                   datagen.half_perturbed_queries(x0, 16, seed=506)])
    return n, x0, x1, x2, X, q


def test_insert_two_batches_matches_oracle(sofa, tmp_path):
    n, x0, x1, x2, X, q = grown_workload()
    l, alpha, k = 16, 256, 5
    ix = sofa.Index(x0, l, alpha, precision=2)          # every optional copy, the FP16 one included
    ix.insert(x1)                                       # device rows
    ix.insert(x2.cpu())                                 # host rows
    inf = ix.info()
    N = X.shape[0]
    assert inf["N"] == N and inf["appended"] == x1.shape[0] + x2.shape[0]
    assert inf["n_tiles"] == (N + 255) // 256
    z, _, _ = orc.znorm(X.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, k)
    assert np.mean(oi[:24, 0] >= x0.shape[0]) > 0.9     # most nearest neighbours are inserted rows
    for t in (dict(dense=1), dict(dense=1, refine_filter=2), dict(dense=2),
              dict(dense=1, bound_precision=1, cand_cap=3, pool_cap=7, group=5), dict(dense=1, use_graph=1)):
        ix.set_tuning(**t)
        for _ in range(2 if t.get("use_graph") else 1):  # a graph is recorded, then replayed
            gi, gd = ix.query(q, k)
            torch.cuda.synchronize()
            assert ix.status() == 0, t
            assert_knn_equal(gi, gd, oi, od)
    # words of every row (original order) under the index's summary
    summ = summary_record(ix, n, l, alpha)
    gw = ix.words().numpy()
    ow = orc.words(z, summ)
    v = orc.selected_values(z, summ)[:, :l]
    for r, j in zip(*np.nonzero(gw != ow)):
        near = np.min(np.abs(summ["beta"][j].astype(np.float64)[1:-1] - v[r, j]))
        assert near <= inf["delta_data"] and abs(int(gw[r, j]) - int(ow[r, j])) == 1
    perm = ix.perm().numpy()
    assert np.array_equal(np.sort(perm), np.arange(N))
    # bounds over the grown index never exceed the distances
    lb = ix.lower_bounds(q[:6]).cpu().numpy().astype(np.float64)
    for i in range(6):
        assert np.all(lb[i] <= orc.sqdist(z, zq[i]) * (1 + 1e-5))
    # the grown index persists, answers the same, and grows further after loading
    path = str(tmp_path / "grown.sofa")
    ix.set_tuning(refine_filter=2)
    a = ix.query(q, k)
    ix.save(path)
    iy = sofa.Index.load(path)
    assert iy.info()["appended"] == inf["appended"]
    iy.set_tuning(refine_filter=2)
    b = iy.query(q, k)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    x3 = datagen.random_walks(500, n, seed=507, device=DEV)
    iy.insert(x3)
    X3 = torch.cat([X, x3])
    q3 = torch.cat([q, datagen.perturbed_members(x3, 8, seed=508)[0]])
    z3, _, _ = orc.znorm(X3.cpu().numpy())
    zq3, _, _ = orc.znorm(q3.cpu().numpy())
    oi3, od3 = orc.knn(z3, zq3, k)
    gi3, gd3 = iy.query(q3, k)
    torch.cuda.synchronize()
    assert iy.status() == 0
    assert_knn_equal(gi3, gd3, oi3, od3)
    ix.close()
    iy.close()


def test_insert_keeps_learned_seed_exact(sofa):
    """A proposal network trained before the insert keeps seeding (its blocks
    cover the positions it was trained on); the answers stay exact."""
    n, x0, x1, x2, X, q = grown_workload()
    ix = sofa.Index(x0, 16, 256, precision=1)
    ix.train_proposal(n_train=16384, n_classes=64, epochs=2, batch=2048, seed=2, top_m=4)
    ix.insert(x1)
    ix.insert(x2)
    z, _, _ = orc.znorm(X.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, 3)
    for mode in (0, 1):
        ix.set_seed_mode(mode)
        ix.set_tuning(refine_filter=2)
        gi, gd = ix.query(q, 3)
        torch.cuda.synchronize()
        assert ix.status() == 0
        assert_knn_equal(gi, gd, oi, od)
    ix.close()


def test_insert_argument_checks(sofa):
    x = datagen.random_walks(2000, 64, seed=509, device=DEV)
    ix = sofa.Index(x, 8, 256)
    with pytest.raises(ValueError):
        ix.insert(datagen.random_walks(10, 32, seed=510, device=DEV))   # wrong length
    lib = sofa.load()
    assert lib.sofa_insert(ix.h, None, 5, None) == -1
    assert lib.sofa_insert(ix.h, sofa._ptr(x), -1, None) == -1
    assert lib.sofa_insert(ix.h, sofa._ptr(x), 0, None) == 0
    assert ix.info()["N"] == 2000 and ix.info()["appended"] == 0
    ix.close()
