"""Seeded synthetic workloads shaped like the paper's benchmark (Sec. V, Table I).

This module holds only input generators: no part of the search method.  Both
the CUDA path and the CPU oracle receive the very same arrays from it.  The
paper's 17 datasets are not available, so these stand in for them:

* random walks ............ cumsum of N(0, 1) steps, FP64 cumsum cast to fp32
* noisy random walks ...... a random walk plus N(0, 0.5^2) white noise per point
* sinusoid mixtures ....... sum of 8 sinusoids, frequency U(0, n/2) cycles per
                            series, phase U(0, 2pi), amplitude LogNormal(0, 1),
                            plus N(0, 0.3^2) noise (high-frequency stress)
* perturbed members ....... a uniformly chosen dataset row plus N(0, 0.1^2)
* alternating walks ....... a random walk plus A (-1)^t with A ~ N(0, amp^2)
                            per series (energy at the Nyquist frequency)

Every generator is deterministic for (seed, device): rows are produced in
fixed chunks, each chunk drawing from its own torch.Generator seeded with
(seed, chunk index).
"""
from __future__ import annotations

import math

import torch

CHUNK = 1 << 14


def _gen(seed: int, chunk: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_003 + int(chunk) * 7919 + 17) & ((1 << 63) - 1))
    return g


def random_walks(N: int, n: int, seed: int = 0, device="cpu", out: torch.Tensor | None = None,
                 noise_sigma: float = 0.0, row0: int = 0) -> torch.Tensor:
    """N x n fp32 random walks; rows row0..row0+N-1 of the seeded stream."""
    device = torch.device(device)
    if out is None:
        out = torch.empty((N, n), dtype=torch.float32, device=device)
    done = 0
    while done < N:
        r = row0 + done
        c = r // CHUNK
        start_in_chunk = r - c * CHUNK
        rows = min(CHUNK - start_in_chunk, N - done)
        g = _gen(seed, c, device)
        steps = torch.randn((CHUNK, n), generator=g, dtype=torch.float64, device=device)
        steps = steps[start_in_chunk:start_in_chunk + rows]
        walk = torch.cumsum(steps, dim=1)
        if noise_sigma > 0.0:
            g2 = _gen(seed + 101, c, device)
            noise = torch.randn((CHUNK, n), generator=g2, dtype=torch.float64, device=device)
            walk = walk + noise_sigma * noise[start_in_chunk:start_in_chunk + rows]
        out[done:done + rows] = walk.to(torch.float32)
        done += rows
    return out


def mixed_walks(N: int, n: int, seed: int = 0, device="cpu", total: int | None = None,
                row0: int = 0) -> torch.Tensor:
    """Rows row0..row0+N-1 of a set of `total` rows (default N): the first
    half random walks, the second half random walks plus N(0, 0.5^2) noise."""
    total = N if total is None else total
    out = torch.empty((N, n), dtype=torch.float32, device=torch.device(device))
    h = total // 2
    a = max(0, min(N, h - row0))        # rows of this range in the first half
    if a > 0:
        random_walks(a, n, seed, device, out=out[:a], row0=row0)
    if N - a > 0:
        random_walks(N - a, n, seed + 1, device, out=out[a:], noise_sigma=0.5, row0=row0 + a - h)
    return out


def sinusoid_mix(N: int, n: int, seed: int = 0, device="cpu", n_waves: int = 8,
                 noise_sigma: float = 0.3, row0: int = 0) -> torch.Tensor:
    """Sum of n_waves sinusoids with non-integer frequencies in (0, n/2) cycles
    per series, uniform phases, LogNormal(0, 1) amplitudes, plus white noise;
    rows row0..row0+N-1 of the seeded stream."""
    device = torch.device(device)
    out = torch.empty((N, n), dtype=torch.float32, device=device)
    t = torch.arange(n, dtype=torch.float64, device=device)
    done = 0
    while done < N:
        r = row0 + done
        c = r // CHUNK
        s0 = r - c * CHUNK
        rows = min(CHUNK - s0, N - done)
        g = _gen(seed, c, device)
        f = torch.rand((CHUNK, n_waves), generator=g, dtype=torch.float64, device=device)[s0:s0 + rows] * (n / 2)
        ph = torch.rand((CHUNK, n_waves), generator=g, dtype=torch.float64, device=device)[s0:s0 + rows]
        ph = ph * (2 * math.pi)
        amp = torch.exp(torch.randn((CHUNK, n_waves), generator=g, dtype=torch.float64, device=device)[s0:s0 + rows])
        x = torch.zeros((rows, n), dtype=torch.float64, device=device)
        for i in range(n_waves):
            x += amp[:, i:i + 1] * torch.sin(2 * math.pi * f[:, i:i + 1] * t[None, :] / n + ph[:, i:i + 1])
        noise = torch.empty((rows, n), dtype=torch.float64, device=device)
        for b in range(0, CHUNK, 2048):   # the chunk's noise in slabs, keeping only this range
            lo, hi = max(b, s0), min(b + 2048, s0 + rows)
            slab = torch.randn((2048, n), generator=g, dtype=torch.float64, device=device)
            if lo < hi:
                noise[lo - s0:hi - s0] = slab[lo - b:hi - b]
        x += noise_sigma * noise
        out[done:done + rows] = x.to(torch.float32)
        done += rows
    return out


def alternating_walks(N: int, n: int, amp: float, seed: int = 0, device="cpu", row0: int = 0) -> torch.Tensor:
    """Random walks plus A (-1)^t, one amplitude A ~ N(0, amp^2) per series
    (stream seed + 211); rows row0..row0+N-1 of the seeded stream."""
    device = torch.device(device)
    out = random_walks(N, n, seed=seed, device=device, row0=row0)
    sign = torch.ones(n, dtype=torch.float64, device=device)
    sign[1::2] = -1.0
    done = 0
    while done < N:
        r = row0 + done
        c = r // CHUNK
        s0 = r - c * CHUNK
        rows = min(CHUNK - s0, N - done)
        g = _gen(seed + 211, c, device)
        a = torch.randn((CHUNK, 1), generator=g, dtype=torch.float64, device=device)[s0:s0 + rows] * amp
        out[done:done + rows] = (out[done:done + rows].to(torch.float64) + a * sign[None, :]).to(torch.float32)
        done += rows
    return out


def perturbed_members(data: torch.Tensor, count: int, seed: int = 1, sigma: float = 0.1):
    """count queries: a uniformly drawn row of data plus N(0, sigma^2) per point
    (before z-normalisation).  Returns (queries, source row ids)."""
    g = _gen(seed, 0, data.device)
    rows = torch.randint(0, data.shape[0], (count,), generator=g, device=data.device)
    noise = torch.randn((count, data.shape[1]), generator=g, dtype=torch.float64, device=data.device)
    q = (data[rows].to(torch.float64) + sigma * noise).to(torch.float32)
    return q, rows


def half_perturbed_queries(data: torch.Tensor, count: int, seed: int = 1):
    """Half perturbed dataset members, half fresh random walks."""
    h = count // 2
    q1, _ = perturbed_members(data, h, seed)
    q2 = random_walks(count - h, data.shape[1], seed=seed + 7, device=data.device)
    return torch.cat([q1, q2], dim=0)
