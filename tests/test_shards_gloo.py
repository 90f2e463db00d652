"""Series sharding, host side: per-shard k-NN windows merged into the exact
answer of the whole collection, alone and over two gloo ranks on CPU; a rank
that never joins the exchange makes it fail instead of returning a partial
answer.  Each shard's window comes from the oracle's FP64 distances."""
import os
import socket
import sys
from datetime import timedelta

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rw(N, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal((N, n)), axis=1).astype(np.float32)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def collection():
    """Random walks (canonical, norm sqrt(32) from the origin) plus a planted
    cross-shard tie around query 0 = the origin: row 2000 (shard 1) at
    distance 1, rows 700 and 600 (shard 0) at 1 + 4.8e-7 and 1 + 1.4e-6 (fp32
    steps of the first coordinate).  Globally row 2000 anchors a run that row
    700 joins (and row 600 does not), so the 1-NN is row 700.  Alone, shard 0
    anchors its run at row 700, row 600 joins it, and its own 1-NN is row 600:
    a merge of per-shard top-1 lists would answer row 2000."""
    from oracle import sofa_oracle as orc
    z, _, _ = orc.znorm(rw(3000, 32, 40))
    q, _, _ = orc.znorm(rw(5, 32, 41))
    q[0] = 0.0
    z[2000] = 0.0
    z[2000, 0] = 1.0
    z[700] = 0.0
    z[700, 0] = np.float32(1 + 4.8e-7)
    z[600] = 0.0
    z[600, 0] = np.float32(1 + 1.4e-6)
    return z, q


SHARDS = [(0, 1500), (1500, 3000)]


def shard_windows(z, q, lo, hi, k):
    """One shard's answer: per query, the window of its rows (global ids)."""
    from oracle import sofa_oracle as orc
    from paper_2411_17483_gb300 import shards
    out = []
    for i in range(q.shape[0]):
        d2 = orc.sqdist(z[lo:hi], q[i])
        out.append(shards.window_of(np.arange(lo, hi, dtype=np.int64), d2, k))
    return out


def test_merge_of_windows_equals_the_whole_search():
    from oracle import sofa_oracle as orc
    from paper_2411_17483_gb300 import shards
    z, q = collection()
    for k in (1, 2, 10):
        parts = [shard_windows(z, q, lo, hi, k) for lo, hi in SHARDS]
        idx, dist = shards.merge_windows(parts, k)
        bi, bd = orc.knn_full(z, q, k)
        assert np.array_equal(idx, bi)
        assert np.array_equal(dist, bd)
    # query 0, k = 1: row 700; shard 0's own top 1 is row 600, and merging
    # the per-shard top-1 lists instead of the windows answers row 2000
    idx1, _ = shards.merge_windows([shard_windows(z, q, lo, hi, 1) for lo, hi in SHARDS], 1)
    assert idx1[0, 0] == 700
    tops = []
    for lo, hi in SHARDS:
        ti, td = shards.tie_ordered(*shard_windows(z, q, lo, hi, 1)[0])
        tops.append([(np.array([ti[0]]), np.array([td[0] ** 2]))])
    assert tops[0][0][0][0] == 600
    naive, _ = shards.merge_windows(tops, 1)
    assert naive[0, 0] == 2000


def test_merge_rejects_inconsistent_parts():
    from paper_2411_17483_gb300 import shards
    a = [(np.array([1, 2]), np.array([1.0, 2.0]))]
    with pytest.raises(ValueError):
        shards.merge_windows([a, a], 1)          # the same row in two shards
    with pytest.raises(ValueError):
        shards.merge_windows([a, a + a], 1)      # different numbers of queries


def _rank(rank, port, k, out, leave_early):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2411_17483_gb300 import shards
    dist.init_process_group("gloo", timeout=timedelta(seconds=10))
    if leave_early and rank == 1:
        out.put((rank, "left"))
        os._exit(0)                              # never joins the exchange
    z, q = collection()
    lo, hi = SHARDS[rank]
    try:
        idx, dist_ = shards.gather_and_merge(shard_windows(z, q, lo, hi, k), k)
        out.put((rank, (idx, dist_)))
    except Exception as e:                       # the exchange failed: no answer
        out.put((rank, f"error: {type(e).__name__}"))
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def _run(k, leave_early):
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, k, out, leave_early)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        if p.is_alive():
            p.kill()
    got = {}
    while not out.empty():
        r, v = out.get()
        got[r] = v
    return got


def test_gather_and_merge_over_two_gloo_ranks():
    from oracle import sofa_oracle as orc
    z, q = collection()
    bi, bd = orc.knn_full(z, q, 3)
    got = _run(3, False)
    assert set(got) == {0, 1}
    for r in (0, 1):
        idx, dist_ = got[r]
        assert np.array_equal(idx, bi) and np.array_equal(dist_, bd)


def test_a_rank_that_leaves_fails_the_exchange():
    got = _run(3, True)
    assert got.get(1) == "left"
    assert isinstance(got.get(0), str) and got[0].startswith("error")
