"""Host-side logic of bench.py, on CPU: the mixed-length workload's packing."""
import types

import torch

import bench
from paper_2411_17483_gb300 import datagen


def test_multi_queries_packing():
    a = types.SimpleNamespace(Q=64)
    packed, qo, ql, qk, oo, total, which = bench.multi_queries(a, 0, "cpu")
    lens = [n for _, n in bench.MULTI_SETS]
    assert ql.tolist() == [lens[w] for w in which.tolist()]
    assert set(qk.tolist()) <= set(bench.MULTI_KS)
    assert int(qo[0]) == 0 and torch.equal(qo[1:], torch.cumsum(ql.long(), 0)[:-1])
    assert int(oo[0]) == 0 and torch.equal(oo[1:], torch.cumsum(qk.long(), 0)[:-1])
    assert total == int(qk.sum()) and packed.numel() == int(ql.sum())
    # query i is the next fresh walk of its dataset's query stream (seed 1000 + dataset at rank 0)
    seen = [0] * len(lens)
    for i, si in enumerate(which.tolist()):
        n = lens[si]
        ref = datagen.random_walks(seen[si] + 1, n, seed=1000 + si, device="cpu")[seen[si]]
        assert torch.equal(packed[int(qo[i]):int(qo[i]) + n], ref)
        seen[si] += 1
    # every dataset's share is drawn uniformly: all four appear in 64 draws
    assert sorted(set(which.tolist())) == [0, 1, 2, 3]


def test_workload_names():
    a = types.SimpleNamespace(gen="multi", Q=10_000, l=16, alphabet=256)
    assert "25Mx128" in bench.workload_name(a) and "6Mx1024" in bench.workload_name(a)
    b = types.SimpleNamespace(gen="rw", N=100_000_000, n=256, Q=10_000, k=1, l=16, alphabet=256)
    assert bench.workload_name(b).startswith("random walks 100000000x256")
