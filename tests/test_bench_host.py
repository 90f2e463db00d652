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


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints the
    contract's line; a tiny workload keeps it to a few seconds."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--N", "20000",
                          "--Q", "2", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "queries/s"
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("random walks 20000x256")


def test_scan_traffic_scales_from_the_stored_capture(monkeypatch):
    """The scan's per-launch DRAM traffic is scaled from a stored small-case
    capture (reads by tile loads, writes by candidates), and only while the
    kernel's source matches the captured one."""
    sha = bench.kernel_source_sha("k_scan")
    assert len(sha) == 16 and sha == bench.kernel_source_sha("k_scan")
    cap = {"case": "test", "source_sha": sha, "dram_read": 1000.0, "dram_write": 300.0, "tile_loads": 10,
           "candidates": 30}
    monkeypatch.setattr(bench, "SCAN_CAPTURE", {"k_scan": cap})
    assert bench.scaled_scan_traffic(40, 60) == 1000.0 * 4 + 300.0 * 2
    assert bench.scaled_scan_traffic(40, 60, "k_vscan") is None          # no capture of that kernel
    monkeypatch.setattr(bench, "SCAN_CAPTURE", {"k_scan": {**cap, "source_sha": "0" * 16}})
    assert bench.scaled_scan_traffic(40, 60) is None
    monkeypatch.setattr(bench, "SCAN_CAPTURE", {})
    assert bench.scaled_scan_traffic(40, 60) is None
    import os
    vs = os.path.join(bench.ROOT, "paper_2411_17483_gb300", "csrc", "vscan.cu")
    assert len(bench.kernel_source_sha("k_vscan", vs)) == 16
