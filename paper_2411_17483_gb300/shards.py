"""Series sharding over ranks: merging per-shard k-NN windows (host logic).

The collection can be split into contiguous row ranges, one per rank, each
searched exactly on its own.  The answer of the whole is then a merge of the
ranks' answers, which must respect the tie rule of the exact k-NN: results
are ordered by distance, and a run of consecutive results whose distances
lie within 1e-6 relative of the run's first is ordered by ascending row id.

Because that rule groups results into runs anchored at their first member, a
shard's own top k is not enough: a row can fall out of its shard's top k
(another row of the shard anchors a run that pulls a lower id in front of
it) and still belong to the global top k (in the global order a different
row anchors its run).  What is enough is each shard's *window*: every row
whose distance d satisfies d <= D_k (1 + 1e-6), D_k the shard's k-th
smallest distance.  The global k-th distance is at most any shard's, so
every row of the global window lies in its shard's window; the merge cuts
the union by the same rule with the global D_k and orders it by the tie
rule.

Distances here are FP64 squared distances, the precision in which the tie
rule is decided.  `window_of` cuts a shard's candidate list to its window;
`merge_windows` merges the ranks' windows; `gather_and_merge` exchanges the
windows over torch.distributed (one all-gather of objects) and merges them
on every rank.  A rank that never joins the exchange makes it fail with the
process group's timeout: no partial answer is ever returned.
"""
from __future__ import annotations

import numpy as np

TIE_REL = 1e-6


def window_of(ids: np.ndarray, d2: np.ndarray, k: int):
    """The entries of one query's candidate list (ids, FP64 squared
    distances) whose distance is within the tie window of the k-th smallest:
    sqrt(d2) <= D_k (1 + 1e-6).  With fewer than k entries, all of them."""
    ids = np.asarray(ids, np.int64)
    d = np.sqrt(np.asarray(d2, np.float64))
    if d.size <= k:
        return ids.copy(), np.asarray(d2, np.float64).copy()
    dk = np.partition(d, k - 1)[k - 1]
    keep = d <= dk + TIE_REL * dk
    return ids[keep], np.asarray(d2, np.float64)[keep]


def tie_ordered(ids: np.ndarray, d2: np.ndarray):
    """Entries in the final order: by distance (then id), each run of
    distances within 1e-6 relative of the run's first reordered by id.
    Returns (ids, distances), distances not squared."""
    d = np.sqrt(np.asarray(d2, np.float64))
    ids = np.asarray(ids, np.int64)
    o = np.lexsort((ids, d))
    d, ids = d[o], ids[o]
    out_i = np.empty_like(ids)
    out_d = np.empty_like(d)
    i = 0
    while i < d.size:
        j = i
        while j + 1 < d.size and d[j + 1] <= d[i] + TIE_REL * d[i]:
            j += 1
        seg = np.argsort(ids[i:j + 1], kind="stable")
        out_i[i:j + 1] = ids[i:j + 1][seg]
        out_d[i:j + 1] = d[i:j + 1][seg]
        i = j + 1
    return out_i, out_d


def merge_windows(parts, k: int):
    """Merge per-shard windows into the global k-NN.

    parts: one entry per shard, each a list over queries of (ids, d2) -- the
    query's window in that shard (global row ids, FP64 squared distances).
    Every shard must cover the same queries.  Returns (idx, dist): Q x k
    int64 row ids and FP64 distances in the tie-rule order; -1 / inf pad a
    query with fewer than k rows in all shards together."""
    if not parts:
        raise ValueError("no shard answers to merge")
    Q = len(parts[0])
    if any(len(p) != Q for p in parts):
        raise ValueError("shards answered different numbers of queries")
    idx = np.full((Q, k), -1, np.int64)
    dist = np.full((Q, k), np.inf, np.float64)
    for q in range(Q):
        ids = np.concatenate([np.asarray(p[q][0], np.int64) for p in parts])
        d2 = np.concatenate([np.asarray(p[q][1], np.float64) for p in parts])
        if np.unique(ids).size != ids.size:
            raise ValueError(f"query {q}: a row id appears in more than one shard")
        wi, wd2 = window_of(ids, d2, k)
        oi, od = tie_ordered(wi, wd2)
        m = min(k, oi.size)
        idx[q, :m] = oi[:m]
        dist[q, :m] = od[:m]
    return idx, dist


def gather_and_merge(local_windows, k: int, group=None):
    """Exchange this rank's windows (a list over queries of (ids, d2)) with
    every rank of the process group and merge them; every rank returns the
    same (idx, dist).  Raises when the exchange fails (a rank missing from
    it fails the collective after the group's timeout)."""
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    gathered = [None] * ws
    dist.all_gather_object(gathered, [(np.asarray(i, np.int64), np.asarray(d, np.float64))
                                      for i, d in local_windows], group=group)
    if any(g is None for g in gathered):
        raise RuntimeError("a shard's answer is missing")
    return merge_windows(gathered, k)
