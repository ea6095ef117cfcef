"""bench.py's host-side pieces, on the CPU: the reference arm's JSON line
(the CPU oracle timed on a small workload), the served trace generator and
the batch-trace summary of the server's batch log."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "delaunay_2k", "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"] == "delaunay_2k"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert set(line["host"]["stage_ms_per_step"]) == set(oracle.TIME_NAMES)


def test_served_trace_is_poisson_with_the_recipes_mix():
    t, pick = bench.serve_trace(20.0, 512, 32, seed=3)
    r = bench.SERVE_RECIPE
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 20.0
    assert abs(len(t) / 20.0 - r["rate"]) < 4 * np.sqrt(r["rate"] / 20.0)   # Poisson count within 4 sigma
    gaps = np.diff(t)
    assert abs(gaps.mean() * r["rate"] - 1) < 0.05 and abs(gaps.std() / gaps.mean() - 1) < 0.05  # exponential
    large = pick >= 512
    assert abs(large.mean() - r["p_large"]) < 0.02
    assert pick.min() >= 0 and pick.max() < 544
    t2, pick2 = bench.serve_trace(20.0, 512, 32, seed=3)
    assert np.array_equal(t, t2) and np.array_equal(pick, pick2)


def _record(t_form, in_ms, run_ms, out_ms, lane=0, n=1, tri=1000):
    t_enq = t_form + 1e-5
    t_meta = t_enq + 1e-3 * (in_ms + run_ms) + 2e-5
    t_oe = t_meta + 1e-5
    return {"t_form": t_form, "t_enqueued": t_enq, "t_meta_seen": t_meta, "t_out_enqueued": t_oe,
            "t_done": t_oe + 1e-3 * out_ms + 2e-5, "in_ms": in_ms, "run_ms": run_ms, "idle_ms": 0.0,
            "out_ms": out_ms, "n_triangles": tri, "n_requests": n, "slot": 0 if lane else 1, "lane": lane,
            "t_stream_start": t_form + 1e-5, "t_meta_landed": t_meta - 1e-5}


def test_batch_trace_summarises_the_log():
    assert bench.batch_trace([]) is None
    log = [_record(0.01 * i, 0.1, 0.2, 0.1, lane=1) for i in range(98)]
    log += [_record(1.0, 30.0, 4.0, 40.0, n=20, tri=50_000_000), _record(1.1, 10.0, 2.0, 12.0, n=5, tri=9_000_000)]
    tr = bench.batch_trace(log)
    assert tr["batches"] == 100 and tr["lane_batches"] == 98
    assert tr["in_ms"]["max"] == 30.0 and tr["in_ms"]["p50"] == pytest.approx(0.1)
    assert tr["out_ms"]["max"] == 40.0
    slow = tr["slowest"]
    assert len(slow) == 5 and slow[-1]["triangles"] == 50_000_000 and slow[-2]["triangles"] == 9_000_000
    assert [s["total_ms"] for s in slow] == sorted(s["total_ms"] for s in slow)
    assert slow[-1]["total_ms"] == pytest.approx(74.0 + 0.07, abs=0.01)
    # lane batches have no copy-engine metadata step: their notice delay is left out
    assert len(log) - tr["lane_batches"] == 2
    assert tr["meta_notice_delay_ms"]["max"] == pytest.approx(0.01, abs=1e-3)
    assert tr["stream_start_delay_ms"]["max"] == pytest.approx(0.01, abs=1e-3)


def test_roofline_traffic_only_for_the_profiled_workload_and_kernels():
    """The bench line's per-kernel DRAM traffic comes from the committed ncu
    summary only for the workload that summary is scaled to, and only while
    the method kernels hash to the digest it records; the shares it is
    compared with sum to B_alg."""
    from paper_2403_14723_gb300 import build

    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    wl = d["workload"]
    for k, rec in d["kernels"].items():
        want = rec["dram_bytes_per_launch_full_workload"] if d["core_kernel_digest"] == build.core_digest() else None
        assert bench.ncu_traffic(k, wl) == want
        assert bench.ncu_traffic(k, "pgrid_2048") is None
        assert bench.ncu_traffic(k, "batch_4096") is None
    assert bench.ncu_traffic("no_such_kernel", wl) is None
    T, V, NF, P = 33_538_050, 16_777_216, 59_815_876, 13_138_913
    total, per = bench.algorithmic_bytes(T, V, NF, P)
    assert total == 24 * T + 16 * V + 16 * NF + 8 * P and sum(per.values()) == total
