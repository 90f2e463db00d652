#!/usr/bin/env python
"""Benchmark: exact k-NN queries/s of SOFA on GB300 (sm_103a).

Default workload: 100,000,000 random-walk series of length 256 (fp32, ~102 GB,
generated on the device, seed 0), SFA l=16, alphabet 256, equi-depth bins on a
10% sample; 10,000 fresh random-walk queries (seed 1), exact 1-NN.  One step is
one sofa_query call over the whole query batch: query z-normalisation and
projection, seed, leaf / tile / series lower-bound scan, refinement, top-k.

--impl reference times the CPU oracle (FP64 brute force) on the host cores on a
bounded sample of the same workload, scaled to the full N (brute force is
linear in N).  Under torchrun every rank holds a replica and answers its own
query batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact k-NN queries/s, 100M×256 fp32 series (chosen vs plain); % of HBM roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sofa", choices=["sofa", "reference"])
    ap.add_argument("--N", type=int, default=100_000_000)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--Q", type=int, default=10_000)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--l", type=int, default=16)
    ap.add_argument("--alphabet", type=int, default=256)
    ap.add_argument("--seed-mode", default="chosen", choices=["chosen", "plain", "learned"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n-train", type=int, default=1 << 20)
    ap.add_argument("--classes", type=int, default=4096)
    ap.add_argument("--top-m", type=int, default=1, help="proposal-network blocks probed by the learned seed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", type=int, default=1, choices=[1, 2],
                    help="index copies: 1 int8 copies for the refinement filters; 2 also an FP16 copy for "
                         "the dense tensor-core form")
    ap.add_argument("--no-autotune", action="store_true",
                    help="chosen mode with the default tuning instead of the autotuner's choice")
    ap.add_argument("--tune", default="",
                    help="comma-separated knob=value overrides applied to the tuned modes after the autotuner, "
                         "e.g. series_bound=1")
    ap.add_argument("--modes", default="",
                    help="comma-separated subset of the modes to time (plain, plain_seed, learned); default all")
    ap.add_argument("--gen", default="rw", choices=["rw", "mixed", "sin", "multi"],
                    help="rw: random walks (default); mixed: half walks + noisy walks with half perturbed-member "
                         "queries; sin: 8-sinusoid mixtures (high-frequency stress, bounds prune little); multi: "
                         "four random-walk datasets (25M x 128, 25M x 256, 12M x 512, 6M x 1024) in one index set, "
                         "--Q mixed-length queries with k uniform in {1, 5, 10, 50}, one sofa_query_multi call "
                         "per step (--N, --n and --k are ignored)")
    return ap.parse_args()


# DRAM traffic of the series-bound scan from one ncu capture of a small case
# of the same kernel (random walks 4M x 256, 2000 queries, k = 1, learned
# seed + filters; one launch, --metrics dram__bytes_read.sum,
# dram__bytes_write.sum), with the units that launch processed.  A full-size
# launch's traffic is scaled from it: reads by the tile loads (each loads a
# tile's words), writes by the candidates emitted.  Reported only while the
# kernel's source is the one that was captured (sha256 of its template text).
SCAN_CAPTURE = {}


def kernel_source_sha(name="k_scan", path=None):
    """sha256 (16 hex digits) of a kernel template's text."""
    import hashlib
    path = path or os.path.join(ROOT, "paper_2411_17483_gb300", "csrc", "query_kernels.cu")
    s = open(path).read()
    i = s.index(f" {name}(")
    a = s.rindex("template <", 0, i)
    b = s.index("\n}\n", i) + 3
    return hashlib.sha256(s[a:b].encode()).hexdigest()[:16]


KERNEL_FILES = {"k_scan": "query_kernels.cu", "k_vscan": "vscan.cu"}


def scaled_scan_traffic(tile_loads, candidates, kernel="k_scan"):
    """Per-launch DRAM bytes of a scan kernel scaled from its stored
    small-case capture, or None when there is none for its current source."""
    c = SCAN_CAPTURE.get(kernel)
    path = os.path.join(ROOT, "paper_2411_17483_gb300", "csrc", KERNEL_FILES[kernel])
    if not c or kernel_source_sha(kernel, path) != c["source_sha"]:
        return None
    return (c["dram_read"] * tile_loads / c["tile_loads"]
            + c["dram_write"] * candidates / max(1, c["candidates"]))


def precision_text(a, stats) -> str:
    """Arithmetic of the chosen mode, stage by stage."""
    if stats.get("dense_pairs", 0) > 0:
        bound = "tcgen05 " + ("fp16" if a.precision == 2 else "tf32") + " contraction (derived margin)"
    else:
        bound = "fp32 SFA bounds"
    return (f"{bound}, int8 value-code and int8 row filters (derived margins), fp32 refine, "
            "fp64 final re-score")


MULTI_SETS = [(25_000_000, 128), (25_000_000, 256), (12_000_000, 512), (6_000_000, 1024)]
MULTI_KS = (1, 5, 10, 50)


def workload_name(a):
    if a.gen == "multi":
        sets = ", ".join(f"{N // 1_000_000}Mx{n}" for N, n in MULTI_SETS)
        return (f"random walks in four datasets ({sets}) fp32, {a.Q} fresh random-walk queries, length uniform "
                f"over the four, exact k-NN with k uniform in {{1, 5, 10, 50}}, l={a.l}, alphabet {a.alphabet}")
    data = {"rw": "random walks", "mixed": "random walks + noisy random walks",
            "sin": "8-sinusoid mixtures + N(0,0.3^2) noise"}[a.gen]
    queries = {"rw": "fresh random-walk queries", "mixed": "queries (half perturbed members, half fresh walks)",
               "sin": "queries of the same generator"}[a.gen]
    return f"{data} {a.N}x{a.n} fp32, {a.Q} {queries}, exact {a.k}-NN, l={a.l}, alphabet {a.alphabet}"


def make_rows(a, rows, seed, device, out=None, row0=0):
    """Rows row0.. of the workload's data (seed 0) or query (seed 1 + rank) stream."""
    from paper_2411_17483_gb300 import datagen
    if a.gen == "sin":
        x = datagen.sinusoid_mix(rows, a.n, seed=seed, device=device, row0=row0)
    elif a.gen == "mixed" and seed == 0:
        x = datagen.mixed_walks(rows, a.n, seed=seed, device=device, total=a.N, row0=row0)
    else:
        return datagen.random_walks(rows, a.n, seed=seed, device=device, out=out, row0=row0)
    if out is not None:
        out.copy_(x)
        return out
    return x


def make_queries(a, x, seed, device):
    from paper_2411_17483_gb300 import datagen
    if a.gen == "mixed":
        return datagen.half_perturbed_queries(x, a.Q, seed=seed)
    return make_rows(a, a.Q, seed, device)


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def nvtx_push(name):
    """Host-thread NVTX range around one mode's warm-up and timed steps, so a
    profiler can select that mode's launches (ncu --nvtx --nvtx-include)."""
    try:
        torch.cuda.nvtx.range_push(name)
        return True
    except (AttributeError, RuntimeError):
        return False


def nvtx_pop(pushed):
    if pushed:
        torch.cuda.nvtx.range_pop()


def tensor_peaks(rname):
    """(sustained, burst, description) bf16 tensor peaks in TFLOP/s: the
    measured ones from MEASURED_PEAKS.json, else the fallbacks (1700 / 1900).
    Kernels timed inside a long step are held against the sustained peak."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return (float(pk["bf16_tflops_sustained"]), float(pk["bf16_tflops"]),
                f"measured bf16 sustained under the power cap ({rname})")
    except (OSError, KeyError, ValueError):
        return 1700.0, 1900.0, f"fallback bf16 sustained ({rname})"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(z, zq, k, N_full, seconds):
    """Time the oracle's brute-force k-NN of canonical queries zq over the
    canonical row sample z; scale the rate to N_full series."""
    from oracle import sofa_oracle as orc
    done = 0
    t0 = time.perf_counter()
    while True:
        orc.knn(z, zq[done:done + 1], k)
        done += 1
        el = time.perf_counter() - t0
        if (el >= seconds and done >= 2) or done >= zq.shape[0]:
            break
    rate_sample = done / el
    rate_full = rate_sample * z.shape[0] / N_full
    return rate_full, done, el, orc.num_threads()


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws, dev):
    if ws == 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- reference arm
def run_reference(a, ws, rank):
    if rank != 0:
        return
    from paper_2411_17483_gb300 import datagen
    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    if a.gen == "multi":
        rows_per_set = [datagen.random_walks(min(N, 500_000), n, seed=10 + si, device=dev).cpu().numpy()
                        for si, (N, n) in enumerate(MULTI_SETS)]
        packed, qo, _, _, _, _, which = multi_queries(a, 0, dev)
        per_step = max(4.0, 60.0 / max(1, a.steps + a.warmup))
        multi_oracle_rate(a, rows_per_set, packed, qo, which, min(per_step, 8.0))   # warm-up
        rates, secs = [], 0.0
        for _ in range(a.steps):
            rate, cores, sample, el = multi_oracle_rate(a, rows_per_set, packed, qo, which, per_step)
            rates.append(rate)
            secs += el
        value = statistics.mean(rates)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / max(1, a.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "oracle": "CPU FP64 brute force (oracle/)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return
    rows = min(a.N, 2_000_000)
    xs = make_rows(a, rows, 0, dev).cpu().numpy()
    q = make_queries(a, make_rows(a, rows, 0, dev), 1, dev).cpu().numpy()
    from oracle import sofa_oracle as orc
    zq, _, _ = orc.znorm(q)
    xs, _, _ = orc.znorm(xs)
    per_step = max(1.0, 60.0 / max(1, a.steps + a.warmup))
    for _ in range(a.warmup):
        cpu_oracle_rate(xs, zq, a.k, a.N, min(per_step, 5.0))
    rates, secs = [], 0.0
    nq = 0
    for _ in range(a.steps):
        r, done, el, cores = cpu_oracle_rate(xs, zq, a.k, a.N, per_step)
        rates.append(r)
        secs += el
        nq += done
    value = statistics.mean(rates)
    sample = f"{nq} queries over the first {rows} of {a.N} series, brute force FP64, scaled by {rows}/{a.N}"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / max(1, a.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "oracle": "CPU FP64 brute force (oracle/)"},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- mixed workload
def multi_queries(a, rank, dev):
    """The mixed workload's queries: dataset (hence length) uniform over the
    four, k uniform over MULTI_KS, each row a fresh random walk of its
    dataset's length (stream seed 1000 (1 + rank) + dataset).  Returns the
    packed rows and per-query offsets, lengths, k's and output offsets, and
    the total output length."""
    from paper_2411_17483_gb300 import datagen
    g = torch.Generator().manual_seed(1 + rank)
    which = torch.randint(0, len(MULTI_SETS), (a.Q,), generator=g)
    ks = torch.tensor(MULTI_KS, dtype=torch.int32)[torch.randint(0, len(MULTI_KS), (a.Q,), generator=g)]
    lens = torch.tensor([n for _, n in MULTI_SETS], dtype=torch.int64)[which]
    rows = [datagen.random_walks(int((which == si).sum()), n, seed=1000 * (1 + rank) + si, device=dev)
            for si, (_, n) in enumerate(MULTI_SETS)]
    cursor = [0] * len(MULTI_SETS)
    parts = []
    for si in which.tolist():
        parts.append(rows[si][cursor[si]])
        cursor[si] += 1
    packed = torch.cat(parts).contiguous()
    q_off = torch.cumsum(lens, 0) - lens
    o_off = torch.cumsum(ks.to(torch.int64), 0) - ks.to(torch.int64)
    return packed, q_off, lens.to(torch.int32), ks, o_off, int(ks.sum()), which


def multi_oracle_rate(a, rows_per_set, packed, qo, which, seconds):
    """The oracle's brute force on the mixed workload: per dataset, up to
    50 of its queries over the sample rows_per_set[si] (the dataset's first
    rows), the rate scaled to the dataset's size; the rates are combined by
    the query mix (seconds per query = sum of share / rate)."""
    from oracle import sofa_oracle as orc
    per_query_s, done_all, el_all, cores = 0.0, 0, 0.0, 1
    for si, (N, n) in enumerate(MULTI_SETS):
        zs, _, _ = orc.znorm(rows_per_set[si])
        sel = (which == si).nonzero().flatten()[:50].tolist()
        zq, _, _ = orc.znorm(torch.stack([packed[int(qo[i]):int(qo[i]) + n] for i in sel]).cpu().numpy())
        rate, done, el, cores = cpu_oracle_rate(zs, zq, 10, N, seconds / len(MULTI_SETS))
        per_query_s += float((which == si).sum()) / which.numel() / rate
        done_all += done
        el_all += el
    rows = rows_per_set[0].shape[0]
    sample = (f"{done_all} queries brute-forced (FP64, k=10) over the first {rows} series of each dataset in "
              f"{el_all:.1f} s, each dataset's rate scaled by {rows}/N and combined by the query mix")
    return 1.0 / per_query_s, cores, sample, el_all


def precision_multi(tunings) -> str:
    tc = any(t.get("series_bound") for t in tunings)
    return ("fp32 SFA bounds" + (", tensor-core FP16 value-code series bound (derived margin)" if tc else "") +
            ", int8 value-code and int8 row filters (derived margins), fp32 refine, fp64 final re-score")


def run_sofa_multi(a, ws, rank, local):
    """Four random-walk indexes answered together by sofa_query_multi: plain
    FP32 refinement vs the refinement filters (both exact, same answers)."""
    from paper_2411_17483_gb300 import datagen, sofa
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    hbm_peak, peak_kind = peaks()
    ixs, cpu_rows, gen_s, build_s = [], [], 0.0, 0.0
    for si, (N, n) in enumerate(MULTI_SETS):
        ta = time.perf_counter()
        x = torch.empty((N, n), dtype=torch.float32, device=dev)
        datagen.random_walks(N, n, seed=10 + si, device=dev, out=x)
        if rank == 0 and ws == 1 and not a.no_cpu_baseline:
            cpu_rows.append(x[: min(N, 500_000)].cpu().numpy())
        torch.cuda.synchronize()
        tb = time.perf_counter()
        ixs.append(sofa.Index(x, a.l, a.alphabet, sample_ratio=0.1, precision=1))
        torch.cuda.synchronize()
        gen_s += tb - ta
        build_s += time.perf_counter() - tb
        del x
        torch.cuda.empty_cache()
    packed, qo, ql, qk, oo, total, which = multi_queries(a, rank, dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    # plain FP32 refinement; the refinement filters; and each index with the
    # autotuner's pick, made on fresh queries of its own length (as many as
    # the workload sends it, stream seed 200 + 1000 rank + dataset), never on
    # the timed ones, at the mix's largest k: its queries have the loosest
    # thresholds and dominate the cost (tuned at k = 10, the indexes dropped
    # the tile envelope checks and the mixed run was 7 % slower)
    modes = {"plain": [{}] * len(ixs), "filters": [dict(refine_filter=2)] * len(ixs)}
    chosen = "filters"
    if not a.no_autotune:
        tuned = []
        for si, ((N, n), ix) in enumerate(zip(MULTI_SETS, ixs)):
            qt = datagen.random_walks(max(64, int((which == si).sum())), n, seed=200 + 1000 * rank + si, device=dev)
            ix.set_seed_mode(0)
            ix.set_tuning(refine_filter=2)
            t = ix.autotune(qt, max(MULTI_KS))
            tuned.append({k: v for k, v in t.items() if v})
            del qt
        modes["tuned"] = tuned
        chosen = "tuned"
    results, answers = {}, {}
    for name, tun in modes.items():
        for ix, t in zip(ixs, tun):
            ix.set_seed_mode(0)
            ix.set_tuning(**t)
        for _ in range(a.warmup):
            sofa.query_multi(ixs, packed, qo, ql, qk, oo, total)
        torch.cuda.synchronize()
        for ix in ixs:
            ix.stats(reset=True)
            ix.profile(reset=True)
            ix.set_profiling(True)
        clk = Clocks(local)
        barrier(ws)
        torch.cuda.synchronize()
        clk.start()
        tot_ms = 0.0
        st = torch.cuda.current_stream()
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            idx, dist = sofa.query_multi(ixs, packed, qo, ql, qk, oo, total)
            e1.record(st)
            e1.synchronize()
            tot_ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        clocks = clk.stop()
        for ix in ixs:
            if ix.status() != 0:
                raise RuntimeError(f"query status {ix.status()} in mode {name}: answers not valid")
            ix.set_profiling(False)
        barrier(ws)
        profs = [ix.profile(reset=True) for ix in ixs]
        stats = [ix.stats(reset=True) for ix in ixs]
        prof = {"ms": {k: sum(p["ms"][k] for p in profs) for k in profs[0]["ms"]},
                "launches": {k: sum(p["launches"][k] for p in profs) for k in profs[0]["launches"]},
                "scan_tile_loads": sum(p["scan_tile_loads"] for p in profs),
                "scan_tile_checks": sum(p["scan_tile_checks"] for p in profs)}
        results[name] = dict(ms=max_over_ranks(tot_ms / a.steps, ws, dev), prof=prof, profs=profs, stats=stats,
                             clocks=clocks)
        answers[name] = idx.clone()
    for name in modes:
        if not torch.equal(answers["plain"], answers[name]):
            raise RuntimeError(f"modes plain and {name} gave different answers")
    r = results[chosen]
    value = ws * a.Q / (r["ms"] / 1e3)
    prof = r["prof"]
    phase = max(prof["ms"], key=lambda k: prof["ms"][k])
    launches = max(1, prof["launches"][phase])
    per_launch_s = prof["ms"][phase] / 1e3 / launches
    LW = ixs[0].info()["word_bytes"]
    roof = {"kernel": phase, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None}
    alu = None
    if phase == "scan":
        # each index's scan is the word bound (k_scan: LW bytes per (query,
        # series) pair bounded) or the tensor-core bound (k_vscan: 256 x
        # (2 NB + 16) bytes per (work unit, tile) load), by its own tuning;
        # both add 2 LW bytes per tile envelope checked
        tc = [bool(t.get("series_bound")) for t in modes[chosen]]
        tile_pairs = sum(s_["tile_pairs"] for s_ in r["stats"])
        alg = 0.0
        for use_tc, p_, s_ in zip(tc, r["profs"], r["stats"]):
            alg += p_["scan_tile_checks"] * 2 * LW
            alg += p_["scan_tile_loads"] * 256 * (4 * LW + 16) if use_tc else s_["tile_pairs"] * 256 * LW
        alg /= launches
        ach = alg / per_launch_s / 1e9
        kname = "k_vscan" if all(tc) else ("k_scan" if not any(tc) else "k_vscan+k_scan")
        roof = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": None, "algorithmic_bytes_per_launch": alg,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "note": "per index: k_vscan moves 256 x (2 NB bytes of FP16 codes + 16 bytes of constants) per "
                        "(work unit, tile) load; k_scan counts LW logical bytes per (query, series) pair "
                        "bounded (the queries of a work unit share each tile's read, so its frac can exceed 1); "
                        "plus 2 LW per tile envelope checked"}
        if not any(tc):
            clk = (r["clocks"].get("sm_mhz") or 1920.0) * 1e6
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak_b = sms * 128 * clk / (3 * LW) / 1e9
            ach_b = tile_pairs * 256 / launches / per_launch_s / 1e9
            alu = {"kernel": "k_scan", "achieved": ach_b, "peak": peak_b, "unit": "G (query, series) bounds/s",
                   "frac": ach_b / peak_b,
                   "peak_kind": f"derived from the kernel's own 3 FP32 lane operations per value: {sms} SMs x "
                                f"128 lanes x {clk / 1e6:.0f} MHz / (3 x {LW})"}
    step_bytes = 0.0
    for (N, n), s_, p_, t_ in zip(MULTI_SETS, r["stats"], r["profs"], modes[chosen]):
        vf, f8, rf = s_.get("value_filtered", 0), s_.get("filtered", 0), s_["refined"]
        value_checked = vf + f8 + rf if vf else 0
        int8_rows = f8 + rf if (vf or f8) else 0
        bound = p_["scan_tile_loads"] * 256 * (4 * LW + 16) if t_.get("series_bound") else s_["tile_pairs"] * 256 * LW
        step_bytes += (bound + value_checked * (2 * LW + 8) + int8_rows * n + rf * n * 4)
    step_bytes /= a.steps
    step_roof = step_bytes / (r["ms"] / 1e3) / 1e9

    e2e = None
    if not a.no_e2e:
        ph = packed.cpu().pin_memory()
        qo_h, ql_h, qk_h, oo_h = qo.cpu(), ql.cpu(), qk.cpu(), oo.cpu()
        ih, _ = sofa.query_multi(ixs, ph, qo_h, ql_h, qk_h, oo_h, total)
        barrier(ws)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(a.steps):
            ih, dh = sofa.query_multi(ixs, ph, qo_h, ql_h, qk_h, oo_h, total)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - w0, ws, dev)
        e2e = {"value": ws * a.Q * a.steps / el, "unit": "queries/s",
               "h2d_bytes_per_step": packed.numel() * 4 + a.Q * (8 + 4 + 4 + 8), "d2h_bytes_per_step": total * 12}
        assert torch.equal(ih, answers[chosen].cpu())

    cpu = None
    if cpu_rows:
        rate, cores, sample, _ = multi_oracle_rate(a, cpu_rows, packed, qo, which, a.cpu_seconds)
        cpu = {"value": rate, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "datasets": [f"{N}x{n}" for N, n in MULTI_SETS],
                       "Q_per_gpu": a.Q, "k": "uniform in {1, 5, 10, 50}", "l": a.l, "alphabet": a.alphabet,
                       "seed_mode": "plain", "tuning": modes[chosen],
                       "precision": precision_multi(modes[chosen]),
                       "l2": "flushed between timed steps (256 MB write)", "build_s": round(build_s, 3),
                       "gen_s": round(gen_s, 3), "parallelism": f"replicas x{ws}"},
            "roofline": roof,
            "alu_view": alu,
            "step_roofline": {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_roof,
                              "frac": step_roof / hbm_peak, "peak": hbm_peak},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": r["clocks"],
            "gpu_launches": int(sum(prof["launches"].values())),
            "modes": {m: {"queries_per_s": ws * a.Q / (results[m]["ms"] / 1e3), "ms_per_step": results[m]["ms"],
                          "phases_ms_per_step": {k: v / a.steps for k, v in results[m]["prof"]["ms"].items()},
                          "pruning": {k: sum(s_[k] for s_ in results[m]["stats"]) / a.steps
                                      for k in ("tile_pairs", "candidates", "refined", "filtered",
                                                "value_filtered", "overflow_passes", "dense_passes")}}
                      for m in results},
        }
        print(json.dumps(out), flush=True)
    for ix in ixs:
        ix.close()


# ---------------------------------------------------------------- GPU arm
def run_sofa(a, ws, rank, local):
    from paper_2411_17483_gb300 import datagen, sofa
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    hbm_peak, peak_kind = peaks()

    t0 = time.perf_counter()
    x = torch.empty((a.N, a.n), dtype=torch.float32, device=dev)
    if a.gen == "sin":   # chunk by chunk: the generator works in FP64
        for r0 in range(0, a.N, 1 << 22):
            r = min(1 << 22, a.N - r0)
            make_rows(a, r, 0, dev, out=x[r0:r0 + r], row0=r0)
    else:
        make_rows(a, a.N, 0, dev, out=x)
    cpu_rows = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu_rows = x[: min(a.N, 2_000_000)].cpu().numpy()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ix = sofa.Index(x, a.l, a.alphabet, sample_ratio=0.1, precision=a.precision)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # each rank answers its own batch: rank r uses query stream seed 1 + r
    q = make_queries(a, x, 1 + rank, dev)
    del x
    torch.cuda.empty_cache()
    info = ix.info()
    idx = torch.empty((a.Q, a.k), dtype=torch.int64, device=dev)
    dist = torch.empty((a.Q, a.k), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    # plain: key-window seed, FP32 bounds and refinement, default tuning;
    # plain_seed: the same seed with the chosen mode's refinement filters and
    # autotuned knobs; learned: the proposal network's seed with those same
    # filters and knobs.  plain_seed and learned differ only in the seed.
    # All three are exact and must give identical answers.
    modes = {"plain": (0, False), "plain_seed": (0, True)}
    chosen = "plain_seed"
    train = None
    if a.seed_mode in ("chosen", "learned"):
        torch.cuda.synchronize()
        tt0 = time.perf_counter()
        ix.train_proposal(n_train=a.n_train, n_classes=min(a.classes, a.N), epochs=4, batch=4096, seed=2,
                          top_m=a.top_m)
        torch.cuda.synchronize()
        inf2 = ix.info()
        train = {"seconds": round(time.perf_counter() - tt0, 2), "pairs": inf2["proposal_train"],
                 "classes": inf2["proposal_classes"], "loss": inf2["proposal_loss"],
                 "heldout_top1": inf2["proposal_top1"], "heldout_top4": inf2["proposal_topm"]}
        modes["learned"] = (1, True)
        chosen = "learned"
    if a.modes:
        keep = [m.strip() for m in a.modes.split(",") if m.strip()]
        if chosen not in keep:
            raise SystemExit(f"--modes must include the chosen mode ({chosen})")
        modes = {m: modes[m] for m in modes if m in keep}
    # run-time tuning of the tuned modes: the autotuner's pick for each seed
    # mode, on one full batch (8192 queries, at most the workload's) of a
    # separate stream (seed 100 + rank), never on the timed queries; both
    # start from the same refinement filters
    tunings = {m: dict(refine_filter=2) for m in modes}
    if not a.no_autotune:
        qt = make_rows(a, min(8192, a.Q), 100 + rank, dev)
        for m, (mode, tuned) in modes.items():
            if not tuned:
                continue
            ix.set_seed_mode(mode)
            ix.set_tuning(refine_filter=2)
            t = ix.autotune(qt, a.k)
            tunings[m] = {k: v for k, v in t.items() if v}
        del qt
    if a.tune:
        over = {kv.split("=")[0].strip(): int(kv.split("=")[1]) for kv in a.tune.split(",") if "=" in kv}
        for m, (mode, tuned) in modes.items():
            if tuned:
                tunings[m] = {**tunings[m], **over}
    chosen_tuning = tunings[chosen]
    results, answers = {}, {}
    for mode_name, (mode, tuned) in modes.items():
        ix.set_seed_mode(mode)
        if tuned:
            ix.set_tuning(**tunings[mode_name])
        else:
            ix.set_tuning()
        pushed = nvtx_push(f"mode_{mode_name}")
        for _ in range(a.warmup):
            ix.query(q, a.k, idx, dist)
        torch.cuda.synchronize()
        ix.stats(reset=True)
        ix.profile(reset=True)
        ix.set_profiling(True)
        clk = Clocks(local)
        barrier(ws)
        torch.cuda.synchronize()
        clk.start()
        tot_ms = 0.0
        st = torch.cuda.current_stream()
        wall0 = time.perf_counter()
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ix.query(q, a.k, idx, dist)
            e1.record(st)
            e1.synchronize()
            tot_ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        nvtx_pop(pushed)
        clocks = clk.stop()
        code = ix.status()
        if code != 0:
            raise RuntimeError(f"query status {code} in mode {mode_name}: answers not valid")
        barrier(ws)
        ix.set_profiling(False)
        prof = ix.profile(reset=True)
        stats = ix.stats(reset=True)
        ms_step = max_over_ranks(tot_ms / a.steps, ws, dev)
        results[mode_name] = dict(ms=ms_step, prof=prof, stats=stats, clocks=clocks, wall=wall)
        answers[mode_name] = (idx.clone(), dist.clone())
    for m in answers:
        if not (torch.equal(answers[m][0], answers[chosen][0]) and torch.equal(answers[m][1], answers[chosen][1])):
            raise RuntimeError(f"modes {m} and {chosen} gave different answers")
    r = results[chosen]
    value = ws * a.Q / (r["ms"] / 1e3)

    # roofline of the dominant kernel (live CUDA-event times from the library,
    # recorded on the stream the kernels run on)
    prof, stats = r["prof"], r["stats"]
    phase = max(prof["ms"], key=lambda k: prof["ms"][k])
    launches = max(1, prof["launches"][phase])
    per_launch_s = prof["ms"][phase] / 1e3 / launches
    LW = info["word_bytes"]
    dense_pairs = stats.get("dense_pairs", 0)
    scan_units = None
    tc_scan = phase == "scan" and dense_pairs == 0 and chosen_tuning.get("series_bound", 0) == 1
    NB = 2 * LW
    if tc_scan:
        # the tensor-core bound: the unit of work is a (work unit, tile) load,
        # which reads the tile's 256 FP16 code rows (2 NB bytes each) and
        # per-series constants (16 bytes each) once for up to 64 queries;
        # plus the tile envelopes checked (2 LW bytes each)
        alg_bytes = (prof["scan_tile_loads"] * 256 * (2 * NB + 16) + prof["scan_tile_checks"] * 2 * LW) / launches
        scan_units = dict(tile_loads=prof["scan_tile_loads"] / launches, candidates=stats["candidates"] / launches)
    elif phase == "scan" and dense_pairs == 0:
        # algorithmic bytes: the word of every (query, series) pair bounded
        # (LW bytes each) and the tile envelopes checked (2 LW bytes each);
        # above 1 means the queries of a work unit share each tile's read
        alg_bytes = (stats["tile_pairs"] * 256 * LW + prof["scan_tile_checks"] * 2 * LW) / launches
        scan_units = dict(tile_loads=prof["scan_tile_loads"] / launches, candidates=stats["candidates"] / launches)
    elif phase == "refine":
        alg_bytes = stats["refined"] * a.n * 4 / launches
    elif phase == "seed":
        alg_bytes = (a.Q * a.steps * (info["n_leaves"] * 2 * LW + 256 * LW + 32 * a.n * 4)) / launches
    else:
        alg_bytes = None
    hbm = {"kernel": phase, "bound": "hbm", "achieved": None, "peak": hbm_peak, "unit": "GB/s", "frac": None,
           "traffic": None, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    if alg_bytes is not None and per_launch_s > 0:
        ach = alg_bytes / per_launch_s / 1e9
        hbm.update(achieved=ach, frac=ach / hbm_peak, algorithmic_bytes_per_launch=alg_bytes)
    if scan_units is not None:
        kname = "k_vscan" if tc_scan else "k_scan"
        hbm["kernel"] = kname
        if tc_scan:
            hbm["note"] = ("bytes a (work unit, tile) load must move: 256 x (2 NB bytes of FP16 codes + 16 bytes "
                           "of constants), plus 2 LW per tile envelope checked")
        else:
            hbm["note"] = ("logical bytes: LW bytes per (query, series) pair bounded plus 2 LW per tile envelope "
                           "checked; the queries of a work unit share each tile's read, so frac can exceed 1")
        hbm["traffic"] = scaled_scan_traffic(scan_units["tile_loads"], scan_units["candidates"], kname)
        if hbm["traffic"] is not None:
            hbm["traffic_kind"] = ("scaled from the stored ncu capture of " + SCAN_CAPTURE[kname]["case"] +
                                   ": reads by tile loads, writes by candidates")
    roof = hbm
    alu = None
    if phase == "scan" and dense_pairs > 0:
        # dense batches: the bound phase is the tcgen05 contraction, TF32
        # operands, or FP16 when the index holds an FP16 copy.  Tensor
        # roofline: the measured bf16 peak sustained under the power cap (the
        # launch runs for milliseconds inside the step), times the nominal
        # TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s) for TF32; FP16 runs at the
        # BF16 rate
        f16 = a.precision == 2 and a.n % 8 == 0
        ratio, rname = (1.0, "fp16 = bf16 rate") if f16 else (1.1 / 2.25, "x 1.1/2.25 (nominal tf32/bf16)")
        bf16, burst, pk_kind = tensor_peaks(rname)
        peak_t = bf16 * ratio
        npad = (a.n + 31) // 32 * 32
        # one k_dense launch per dense pass; the phase also holds the query
        # norms (and the FP16 query copy), a few microseconds, so the time per
        # launch is an upper bound of the contraction's
        dense_launches = max(1, stats.get("dense_passes", 0))
        per_dense_s = prof["ms"][phase] / 1e3 / dense_launches
        flops = 2.0 * dense_pairs * npad / dense_launches
        ach_t = flops / per_dense_s / 1e12
        roof = {"kernel": "k_dense", "bound": "tensor", "achieved": ach_t, "peak": peak_t, "unit": "TFLOP/s",
                "frac": ach_t / peak_t, "traffic": None, "peak_kind": pk_kind,
                "frac_of_burst_peak": ach_t / (burst * ratio),
                "flops_per_launch": flops, "launch_ms": per_dense_s * 1e3,
                "note": "launch_ms is the dense phase's time per k_dense launch, including the query-side "
                        "helper kernels of the phase"}
    elif tc_scan:
        # the tensor pipe's share: per tile load 2 halves x (NB/16 + 1) MMAs
        # of 128 x 64 x 16 (the codes' K steps and the folded test's), i.e.
        # 2 x 256 x 64 x (NB + 16) FLOP, against the FP16 rate (the measured
        # bf16 peak sustained under the power cap; FP16 runs at the BF16 rate)
        bf16, burst, pk_kind = tensor_peaks("fp16 = bf16 rate")
        flops = prof["scan_tile_loads"] * 2.0 * 256 * 64 * (NB + 16) / launches
        alu = {"kernel": "k_vscan", "view": "tensor", "achieved": flops / per_launch_s / 1e12, "peak": bf16,
               "unit": "TFLOP/s", "frac": flops / per_launch_s / 1e12 / bf16, "peak_kind": pk_kind}
    elif phase == "scan":
        # a second view of the same kernel: its own instruction mix is 3 FP32
        # lane operations per value (q - c, the scaled clamp, the
        # square-accumulate), so the FP32 pipe's 128 lanes per SM per clock
        # cap it at SMs x 128 x SM clock / (3 LW) bounds/s.  The denominator
        # is this kernel's formulation, not an algorithmic bound.
        clk = (r["clocks"].get("sm_mhz") or 1920.0) * 1e6
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_b = sms * 128 * clk / (3 * LW) / 1e9
        bounds = stats["tile_pairs"] * 256 / launches
        ach_b = bounds / per_launch_s / 1e9
        alu = {"kernel": "k_scan", "achieved": ach_b, "peak": peak_b, "unit": "G (query, series) bounds/s",
               "frac": ach_b / peak_b,
               "peak_kind": f"derived from the kernel's own 3 FP32 lane operations per value: {sms} SMs x 128 "
                            f"lanes x {clk / 1e6:.0f} MHz / (3 x {LW})"}
    # whole-step algorithmic bytes: the series bound's reads (the word
    # scan: the SFA word of every bounded (query, series) pair, logical; the
    # tensor-core scan: 256 x (2 NB + 16) bytes per (unit, tile) load); for
    # each candidate reaching a filter, its value codes (2 LW bytes + scale
    # and margin) and / or its int8 row; the fp32 rows refined
    vf, f8, rf = stats.get("value_filtered", 0), stats.get("filtered", 0), stats["refined"]
    value_checked = vf + f8 + rf if vf else 0
    int8_rows = f8 + rf if (vf or f8) else 0
    bound_bytes = (prof["scan_tile_loads"] * 256 * (2 * NB + 16) if tc_scan
                   else stats["tile_pairs"] * 256 * LW)
    step_bytes = (bound_bytes + value_checked * (2 * LW + 8) + int8_rows * a.n + rf * a.n * 4) / a.steps
    step_roof = step_bytes / (r["ms"] / 1e3) / 1e9

    # end to end through the public API with host buffers, in the chosen mode
    ix.set_seed_mode(modes[chosen][0])
    ix.set_tuning(**chosen_tuning)
    e2e = None
    if not a.no_e2e:
        qh = q.cpu().pin_memory()
        ih = torch.empty((a.Q, a.k), dtype=torch.int64).pin_memory()
        dh = torch.empty((a.Q, a.k), dtype=torch.float32).pin_memory()
        ix.query(qh, a.k, ih, dh)
        barrier(ws)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(a.steps):
            ix.query(qh, a.k, ih, dh)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - w0, ws, dev)
        e2e = {"value": ws * a.Q * a.steps / el, "unit": "queries/s", "h2d_bytes_per_step": a.Q * a.n * 4,
               "d2h_bytes_per_step": a.Q * a.k * 12}
        assert torch.equal(ih, idx.cpu())

    # small-batch latency of the chosen mode, eager vs recorded CUDA graph
    latency = None
    if not a.no_e2e:
        qs = q[:64].contiguous()
        li = torch.empty((64, a.k), dtype=torch.int64, device=dev)
        ld = torch.empty((64, a.k), dtype=torch.float32, device=dev)
        lat = {}
        for use_graph in (0, 1):
            ix.set_tuning(**{**chosen_tuning, "use_graph": use_graph})
            for _ in range(3):
                ix.query(qs, a.k, li, ld)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for _ in range(20):
                ix.query(qs, a.k, li, ld)
            torch.cuda.synchronize()
            lat["graph_ms" if use_graph else "eager_ms"] = (time.perf_counter() - w0) / 20 * 1e3
        ix.set_tuning(**chosen_tuning)
        latency = {"queries": 64, **lat, "graph_replays": ix.stats()["graph_replays"]}

    # the approximate search alone (same seed mode): throughput and recall@k
    # against this run's exact answers
    approx = None
    if not a.no_e2e:
        ix.query(q, a.k, idx, dist)                     # exact answers of the chosen mode
        exact = idx.clone()
        ix.set_tuning(**{**chosen_tuning, "approximate": 1})
        ai = torch.empty_like(idx)
        ad = torch.empty_like(dist)
        for _ in range(2):
            ix.query(q, a.k, ai, ad)
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(3):
            ix.query(q, a.k, ai, ad)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 3
        A, E = ai.cpu().numpy(), exact.cpu().numpy()
        hits = sum(len(set(A[i]) & set(E[i])) for i in range(a.Q))
        approx = {"queries_per_s": a.Q / (ms / 1e3), "ms_per_step": ms, "recall_at_k": hits / (a.Q * a.k)}
        ix.set_tuning(**chosen_tuning)

    cpu = None
    if cpu_rows is not None:
        from oracle import sofa_oracle as orc
        zq, _, _ = orc.znorm(q[:200].cpu().numpy())
        zs, _, _ = orc.znorm(cpu_rows)
        rate, done, el, cores = cpu_oracle_rate(zs, zq, a.k, a.N, a.cpu_seconds)
        cpu = {"value": rate, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} queries brute-forced (FP64) over the first {cpu_rows.shape[0]} of {a.N} series "
                         f"in {el:.1f} s, scaled by {cpu_rows.shape[0]}/{a.N}"}

    # the learned seed against the plain seed, both with the chosen filters
    # and tuning: the proposal network's own effect
    seed_gain = None
    if "learned" in results and "plain_seed" in results:
        L_, P_ = results["learned"], results["plain_seed"]
        seed_gain = {"queries_per_s_ratio": P_["ms"] / L_["ms"],
                     "tile_pairs_ratio": L_["stats"]["tile_pairs"] / max(1, P_["stats"]["tile_pairs"]),
                     "candidates_ratio": L_["stats"]["candidates"] / max(1, P_["stats"]["candidates"]),
                     "seed_ms_per_step": {m: (results[m]["prof"]["ms"]["seed"] + results[m]["prof"]["ms"]["proposal"])
                                          / a.steps for m in ("plain_seed", "learned")},
                     "seed_over_final_dist": {m: results[m]["stats"]["seed_dist_sum"] /
                                              max(1e-9, results[m]["stats"]["final_dist_sum"])
                                              for m in ("plain_seed", "learned")}}
    build_bytes = a.N * a.n * 4
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "N": a.N, "n": a.n, "Q_per_gpu": a.Q, "k": a.k, "l": a.l,
                       "alphabet": a.alphabet, "seed_mode": chosen, "tuning": chosen_tuning, "precision": precision_text(a, stats),
                       "l2": "flushed between timed steps (256 MB write)", "build_s": round(t2 - t1, 3),
                       "gen_s": round(t1 - t0, 3), "parallelism": f"replicas x{ws}"},
            "build": {"seconds": round(t2 - t1, 3), "input_bytes": build_bytes,
                      "input_gbs": build_bytes / max(1e-9, t2 - t1) / 1e9,
                      "frac_of_hbm_read": build_bytes / max(1e-9, t2 - t1) / 1e9 / hbm_peak},
            "roofline": roof,
            "alu_view": alu,
            "learned_vs_plain_seed": seed_gain,
            "tunings": {m: (tunings[m] if modes[m][1] else "defaults") for m in modes},
            "step_roofline": {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_roof,
                              "frac": step_roof / hbm_peak, "peak": hbm_peak,
                              "series_bound_bytes": "tensor-core scan: 256 x (2 NB + 16) per (unit, tile) load"
                              if tc_scan else "word scan: LW per (query, series) pair bounded (logical)"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": r["clocks"],
            "gpu_launches": int(sum(prof["launches"].values())),
            "modes": {m: {"queries_per_s": ws * a.Q / (results[m]["ms"] / 1e3), "ms_per_step": results[m]["ms"],
                          "seed_over_final_dist": results[m]["stats"]["seed_dist_sum"] /
                          max(1e-9, results[m]["stats"]["final_dist_sum"]),
                          "pruning": {k: v / a.steps for k, v in results[m]["stats"].items()
                                      if k not in ("n_leaves", "n_tiles", "seed_dist_sum", "final_dist_sum")},
                          "scan_tile_loads_per_step": results[m]["prof"]["scan_tile_loads"] / a.steps,
                          "phases_ms_per_step": {k: v / a.steps for k, v in results[m]["prof"]["ms"].items()},
                          "launches_per_step": {k: v / a.steps for k, v in results[m]["prof"]["launches"].items()}}
                      for m in results},
            "proposal_training": train,
            "latency_64_queries": latency,
            "approximate_search": approx,
            "index": {"n_leaves": info["n_leaves"], "n_tiles": info["n_tiles"], "device_GB": info["device_bytes"] / 1e9},
        }
        print(json.dumps(out), flush=True)
    ix.close()


def main():
    a = parse()
    ws, rank, local = dist_init()
    if a.impl == "reference":
        run_reference(a, ws, rank)
    elif a.gen == "multi":
        run_sofa_multi(a, ws, rank, local)
    else:
        run_sofa(a, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
