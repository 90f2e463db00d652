"""Summarisation ablation on synthetic data.

This reproduces the *structure* of the paper's summarisation experiments
(Sec. V, Tables IV-VI): how tight each summary's lower bound is, and how much
it prunes, for
* SFA variants: equi-depth or equi-width bins (Sec. IV "Learned Quantization"),
  variance-ranked or first-l value selection (Sec. IV "Novel Feature
  Selection"), at several sampling ratios (Alg. 1);
* iSAX: PAA means quantised with N(0,1) breakpoints, the summary the tree
  indexes of Sec. II-B use, computed here on the CPU.

All of them are measured on the same series and queries.  The datasets of the
paper are not available, so the absolute values are not the paper's.

Measures, over Q queries and all N series:
* TLB: the mean over (query, series) pairs of LB / ED.
* pruning: the fraction of series whose LB exceeds the query's exact 1-NN
  distance (such series never reach the refinement).

The SFA bounds are the library's own (sofa_lower_bounds, margins included).
The series are z-normalised by the library (sofa_znorm).  The exact distances
come from an FP64 contraction on the GPU.  This is a measurement aid, not part
of the query path.

    python -m paper_2411_17483_gb300.ablation --N 1000000 --n 256 --Q 100
"""
from __future__ import annotations

import argparse
import statistics
import time

import numpy as np
import torch


# ---------------------------------------------------------------- iSAX (CPU)
def paa(z: np.ndarray, w: int) -> np.ndarray:
    """Piecewise aggregate approximation: the means of w equal segments."""
    N, n = z.shape
    if n % w:
        raise ValueError("n must be a multiple of the number of segments")
    return z.reshape(N, w, n // w).mean(axis=2, dtype=np.float64)


def gaussian_breakpoints(alpha: int) -> np.ndarray:
    """The alpha - 1 equiprobable N(0, 1) breakpoints, with -inf / +inf ends."""
    nd = statistics.NormalDist()
    inner = [nd.inv_cdf(a / alpha) for a in range(1, alpha)]
    return np.array([-np.inf] + inner + [np.inf])


def isax_words(p: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Symbol of each PAA value: the a with beta[a] <= v < beta[a + 1]."""
    return (np.searchsorted(beta, p, side="right") - 1).astype(np.int32)


def isax_lb(q_paa: np.ndarray, words: np.ndarray, beta: np.ndarray, n: int) -> np.ndarray:
    """Squared PAA-iSAX lower bound of one query (its PAA values) against every
    word: (n / w) * sum_i dist(q_i, [beta(s_i), beta(s_i + 1)])^2."""
    w = words.shape[1]
    lo = beta[words]
    hi = beta[words + 1]
    d = np.maximum(np.maximum(lo - q_paa[None, :], q_paa[None, :] - hi), 0.0)
    return (n / w) * (d * d).sum(axis=1)


# ---------------------------------------------------------------- measures
def exact_sqdist(zq: torch.Tensor, z: torch.Tensor) -> torch.Tensor:
    """Q x N squared distances in FP64 (||q||^2 + ||x||^2 - 2 q.x, clamped at 0)."""
    zq64, z64 = zq.double(), z.double()
    d = (zq64 * zq64).sum(1)[:, None] + (z64 * z64).sum(1)[None, :] - 2.0 * zq64 @ z64.T
    return d.clamp_min_(0.0)


def measures(lb2: torch.Tensor, d2: torch.Tensor) -> tuple[float, float]:
    """(TLB, pruning rate) from squared lower bounds and squared distances."""
    ed = d2.sqrt()
    lb = lb2.clamp_min(0).sqrt()
    ok = ed > 1e-9
    tlb = float((lb[ok] / ed[ok]).mean())
    dnn = d2.min(dim=1).values.sqrt()
    prune = float((lb > dnn[:, None]).double().mean())
    return tlb, prune


# sampling ratios of Table IV (Sec. V): 0.1 % to 20 %
TABLE_IV_RATIOS = (0.001, 0.005, 0.01, 0.05, 0.1, 0.15, 0.2)


def run(N=1_000_000, n=256, Q=100, l=16, alphabet=256, ratios=TABLE_IV_RATIOS, isax_segments=16,
        seed=0, device="cuda:0", chunk=200_000):
    from . import datagen, sofa
    x = datagen.random_walks(N, n, seed=seed, device=device)
    q = datagen.random_walks(Q, n, seed=seed + 1, device=device)
    z = sofa.znorm(x)
    zq = sofa.znorm(q)
    d2 = torch.cat([exact_sqdist(zq, z[i:i + chunk]) for i in range(0, N, chunk)], dim=1)
    rows = []
    for binning in ("equi-depth", "equi-width"):
        for select in ("variance", "first"):
            for r in ratios:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ix = sofa.Index(x, l, alphabet, sample_ratio=r, binning=binning, select=select)
                torch.cuda.synchronize()
                build = time.perf_counter() - t0
                lb2 = ix.lower_bounds(q).double()
                tlb, prune = measures(lb2, d2)
                rows.append({"summary": f"SFA {binning}, {select}, r={r:g}", "tlb": tlb, "pruning": prune,
                             "build_s": build})
                ix.close()
    # iSAX on the CPU, same canonical series
    zc = z.cpu().numpy()
    beta = gaussian_breakpoints(alphabet)
    t0 = time.perf_counter()
    words = isax_words(paa(zc, isax_segments), beta)
    build = time.perf_counter() - t0
    qp = paa(zq.cpu().numpy(), isax_segments)
    lb2 = torch.from_numpy(np.stack([isax_lb(qp[i], words, beta, n) for i in range(Q)])).to(d2.device)
    tlb, prune = measures(lb2, d2)
    rows.append({"summary": f"iSAX, {isax_segments} PAA segments, N(0,1) breakpoints", "tlb": tlb,
                 "pruning": prune, "build_s": build})
    return rows


def table(rows, title: str) -> str:
    out = [title, "", "| summary | TLB | pruning rate | build (s) |", "|---|---|---|---|"]
    for r in rows:
        out.append(f"| {r['summary']} | {r['tlb']:.4f} | {r['pruning']:.4f} | {r['build_s']:.3f} |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--Q", type=int, default=100)
    ap.add_argument("--l", type=int, default=16)
    ap.add_argument("--alphabet", type=int, default=256)
    ap.add_argument("--segments", type=int, default=16)
    a = ap.parse_args()
    rows = run(a.N, a.n, a.Q, a.l, a.alphabet, isax_segments=a.segments)
    print(table(rows, f"Random walks {a.N} x {a.n}, {a.Q} fresh random-walk queries, l = {a.l}, "
                      f"alphabet {a.alphabet}"))


if __name__ == "__main__":
    main()
