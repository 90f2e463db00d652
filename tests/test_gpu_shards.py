"""Series sharding on one GPU: two indexes over disjoint row ranges of one
collection, each answering sofa_query_window; the host merge of their
windows (shards.merge_windows) must equal the oracle's brute-force k-NN over
the whole collection.

A planted cross-shard near tie makes per-shard top-k lists insufficient.
Row A (shard 1) is the nearest; row B (shard 0) lies within the 1e-6 tie
window of A and has the lower id, so the global 1-NN is B.  Row C (shard 0,
lowest id of the three) lies within the tie window of B but not of A, so
shard 0's own 1-NN is C.  A merge of the two shards' top-1 answers would
therefore return A."""
import numpy as np
import pytest
import torch

from oracle import sofa_oracle as orc
from paper_2411_17483_gb300 import datagen, shards

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

N, n, SPLIT = 20000, 64, 10000
ROW_A, ROW_B, ROW_C = 12000, 700, 600


@pytest.fixture(scope="module")
def sofa():
    from paper_2411_17483_gb300 import sofa as s
    s.load()
    return s


def planted_collection():
    """Random walks with three rows planted around query 0: candidates
    q + (1 + i 4e-8) 0.3 w on a fine grid, of which the oracle's FP64
    distances pick a triple with the gaps described above."""
    x = datagen.random_walks(N, n, seed=403, device="cpu")
    q = datagen.random_walks(1, n, seed=401, device="cpu")[0].to(torch.float64)
    w = datagen.random_walks(1, n, seed=402, device="cpu")[0].to(torch.float64)
    w = w - w.mean()
    cands = torch.stack([(q + (1.0 + i * 4e-8) * 0.3 * w) for i in range(400)]).to(torch.float32).numpy()
    z, _, _ = orc.znorm(cands)
    zq, _, _ = orc.znorm(q[None].to(torch.float32).numpy())
    d = np.sqrt(orc.sqdist(z, zq[0]))
    o = np.argsort(d)
    ds = d[o]
    pick = None
    for i in range(len(ds)):
        for j in range(i + 1, len(ds)):
            if ds[j] > ds[i] * (1 + 0.9e-6):
                break
            if ds[j] < ds[i] * (1 + 0.2e-6):
                continue
            for k in range(j + 1, len(ds)):
                if ds[k] > ds[j] * (1 + 0.8e-6):
                    break
                if ds[k] > ds[i] * (1 + 1.2e-6):
                    pick = (o[i], o[j], o[k])
                    break
            if pick:
                break
        if pick:
            break
    assert pick is not None, "no planted triple found on the grid"
    a, b, c = pick
    x[ROW_A] = torch.from_numpy(cands[a])
    x[ROW_B] = torch.from_numpy(cands[b])
    x[ROW_C] = torch.from_numpy(cands[c])
    queries = torch.cat([q[None].to(torch.float32), datagen.half_perturbed_queries(x, 31, seed=404)])
    return x, queries


def oracle_window(z_shard, zq, k, row0):
    """One shard's window by the oracle: (ids, FP64 squared distances),
    ascending by (distance, id)."""
    d2 = orc.sqdist(z_shard, zq)
    ids, wd2 = shards.window_of(np.arange(z_shard.shape[0], dtype=np.int64) + row0, d2, k)
    o = np.lexsort((ids, np.sqrt(wd2)))
    return ids[o], wd2[o]


@pytest.mark.parametrize("k", [1, 5])
def test_sharded_windows_merge_to_the_exact_knn(sofa, k):
    x, q = planted_collection()
    z, _, _ = orc.znorm(x.numpy())
    zq, _, _ = orc.znorm(q.numpy())
    # the plant: globally B is the 1-NN, in shard 0 alone C is, and the
    # per-shard top-1 lists would merge to A
    gi, _ = orc.knn(z, zq[:1], 1)
    s0, _ = orc.knn(z[:SPLIT], zq[:1], 1)
    assert gi[0, 0] == ROW_B and s0[0, 0] == ROW_C
    naive, _ = shards.merge_windows([[(np.array([ROW_C]), orc.sqdist(z[ROW_C:ROW_C + 1], zq[0]))],
                                     [(np.array([ROW_A]), orc.sqdist(z[ROW_A:ROW_A + 1], zq[0]))]], 1)
    assert naive[0, 0] == ROW_A

    xd, qd = x.to(DEV), q.to(DEV)
    parts = []
    for lo, hi in ((0, SPLIT), (SPLIT, N)):
        ix = sofa.Index(xd[lo:hi].contiguous(), 8, 256, precision=1)
        ix.set_tuning(refine_filter=2)
        ids, d2, cnt = ix.query_window(qd, k)
        torch.cuda.synchronize()
        assert ix.status() == 0
        ids, d2, cnt = ids.cpu().numpy(), d2.cpu().numpy(), cnt.cpu().numpy()
        win = []
        for i in range(q.shape[0]):
            c = int(cnt[i])
            assert c >= min(k, hi - lo)
            assert np.all(ids[i, c:] == -1) and np.all(np.isinf(d2[i, c:]))
            oi, od2 = oracle_window(z[lo:hi], zq[i], k, lo)
            # the same rows, in the same order, with the oracle's FP64 distances bit for bit
            assert np.array_equal(ids[i, :c] + lo, oi), (i, ids[i, :c] + lo, oi)
            assert np.array_equal(d2[i, :c], od2)
            win.append((ids[i, :c] + lo, d2[i, :c]))
        parts.append(win)
        ix.close()
    mi, md = shards.merge_windows(parts, k)
    oi, od = orc.knn(z, zq, k)
    assert np.array_equal(mi, oi)
    assert np.array_equal(md, od)
    assert mi[0, 0] == ROW_B


def test_window_host_buffers_and_argument_checks(sofa):
    x = datagen.random_walks(3000, 32, seed=405, device=DEV)
    q = datagen.random_walks(5, 32, seed=406, device=DEV)
    ix = sofa.Index(x, 8, 256)
    ids, d2, cnt = ix.query_window(q, 3, cap=8)
    hq = q.cpu()
    hi = torch.empty((5, 8), dtype=torch.int64)
    hd = torch.empty((5, 8), dtype=torch.float64)
    hc = torch.empty((5,), dtype=torch.int32)
    lib = sofa.load()
    sofa._check(lib.sofa_query_window(ix.h, sofa._ptr(hq), 5, 3, 8, sofa._ptr(hi), sofa._ptr(hd), sofa._ptr(hc),
                                      sofa._stream(None)))
    assert torch.equal(hi, ids.cpu()) and torch.equal(hd, d2.cpu()) and torch.equal(hc, cnt.cpu())
    for k, cap in ((3, 2), (3, 97), (0, 8)):
        with pytest.raises(sofa.SofaError) as e:
            ix.query_window(q, k, cap=cap)
        assert e.value.code == -1
    ix.close()
