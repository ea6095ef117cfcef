#!/usr/bin/env python3
"""Benchmark: triangles/s from a device-resident half-edge triangulation to
the Polylla polygon mesh, on one or more GPUs (independent replicas).

One step = polylla_generate (all five stages) + the device part of
polylla_get_polygons on the whole mesh, inputs already in HBM.  The default
workload is the largest single mesh: the 4096 x 4096 perturbed grid
(33,538,050 triangles).  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle, timed on the host
    python bench.py --workload batch_4096  # 4,096 meshes in one batched run
    python bench.py --workload served      # Poisson request stream, continuous batching

The batched workload (4,096 independent triangulations, sizes log-uniform in
[100, 200,000] triangles, alternately Delaunay and perturbed grids) runs
every stage once over all meshes from a CUDA graph with autotuned launch
settings, and reports beside it the plain one-mesh-at-a-time path on the
same meshes.

Under torchrun (N > 1) every rank runs its own replica of the mesh on its own
GPU (a single mesh does not shard); value = triangles of all ranks / max
time over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "triangles/sec to polygon mesh (device-resident), % HBM roofline; served p50/p99"
UNIT = "triangles/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="pgrid_4096")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="single mesh only: no batched and served sub-records in the default line")
    ap.add_argument("--extras-serve-seconds", type=float, default=10.0,
                    help="served sub-record: length of the request trace")
    ap.add_argument("--extras-serve-baseline-seconds", type=float, default=5.0,
                    help="served sub-record: trace length through the one-mesh-at-a-time server")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch settings (profiling runs: no tuning launches before the steps)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served request trace (served workload)")
    ap.add_argument("--serve-baseline-seconds", type=float, default=10.0,
                    help="trace length replayed through the one-mesh-at-a-time server")
    ap.add_argument("--serve-slots", type=int, default=3, help="batches in flight (served workload)")
    ap.add_argument("--serve-lane", type=int, default=0,
                    help="largest request of the server's low-latency lane (0: default, negative: no lane)")
    ap.add_argument("--serve-batch-triangles", type=int, default=0,
                    help="triangles at which a served batch stops growing (0: slot capacity)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: the one collective is the timing max)
# ---------------------------------------------------------------------------

def dist_setup(n_gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, ws, local


def dist_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------------------
# measurement helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.lines:
            return None
        sm, mx, reasons, load_sm = [], [], set(), []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                s, m_ = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            sm.append(s)
            mx.append(m_)
            pw = parts[3]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
            try:
                if float(pw) > 250.0:
                    load_sm.append(s)
            except ValueError:
                pass
        if not sm:
            return None
        use = load_sm if load_sm else sm
        return {"sm_mhz": statistics.median(use), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "samples_under_load": len(load_sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_digest() -> str:
    from paper_2403_14723_gb300 import build

    return build._digest()


def core_kernel_digest() -> str:
    from paper_2403_14723_gb300 import build

    return build.core_digest()


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of ``kernel`` on ``workload`` from the committed
    ncu summary, if the summary is scaled to that workload and was taken on
    the current kernel sources (else None)."""
    from paper_2403_14723_gb300 import build

    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("core_kernel_digest") != build.core_digest() or d.get("workload") != workload:
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k.get("dram_bytes_per_launch_full_workload")


def algorithmic_bytes(T, V, NF, P):
    """Bytes the method must move once, B_alg = 24T + 16V + 16 N_F + 8P
    (next/prev of interior half-edges are implicit in the layout; label
    bytes are L2-resident and not counted), and each kernel's share of it:
    the longest edge reads origin and coords (12T + 16V), the relink reads
    twin and writes next/prev of the frontier (12T + 8 N_F), the listing
    kernel writes the CSR (8 N_F + 8P); the repair kernels, the polygon
    count (a second read of next), the tile scan and the batch metadata
    move no bytes of B_alg.  The shares sum to B_alg, so a
    kernel's traffic over its share is the bytes it re-reads."""
    total = 24 * T + 16 * V + 16 * NF + 8 * P
    per_stage = {
        "longest_edge": 12 * T + 16 * V,
        "label_relink": 12 * T + 8 * NF,
        "chords": 0,
        "chord_links": 0,
        "poly_count": 0,
        "tile_scan": 0,
        "poly_list": 8 * NF + 8 * P,
        "batch_meta": 0,
    }
    assert sum(per_stage.values()) == total
    return total, per_stage


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------

def ref_sample_mesh(workload: str, runs: int = 3):
    """A bounded sample of the workload for the oracle: about 10-30 s of
    single-threaded CPU work over ``runs`` runs on the host cores beside the GPU."""
    from paper_2403_14723_gb300 import meshgen

    if workload == "served":
        # the first 64 small and 2 large meshes of the request pool's recipe
        r = SERVE_RECIPE
        small = meshgen.batch_sizes(r["pool_small"], *r["small"], seed=r["seed"])[:64]
        large = meshgen.batch_sizes(r["pool_large"], *r["large"], seed=r["seed"] + 1)[:2]
        ms = [meshgen.batch_member(i, int(t), 10_000 + r["seed"]) for i, t in enumerate(small)]
        ms += [meshgen.batch_member(i, int(t), 20_000 + r["seed"]) for i, t in enumerate(large)]
        return ms, f"64 small + 2 large meshes of the request pool ({sum(m.n_triangles for m in ms):,} triangles)"
    if workload.startswith("batch_"):
        # the first 64 meshes of the batch recipe; the oracle runs them one by one
        r = BATCH_RECIPE
        sizes = meshgen.batch_sizes(int(workload.split("_")[1]), r["t_min"], r["t_max"], r["seed"])[:64]
        ms = [meshgen.batch_member(i, int(t), r["seed"]) for i, t in enumerate(sizes)]
        return ms, f"the first {len(ms)} meshes of the batch ({sum(m.n_triangles for m in ms):,} triangles)"

    if workload.startswith("pgrid_"):
        # about 60 ns per triangle on one Grace core: 2048^2 for a few runs,
        # smaller grids of the same recipe for many
        side = 2048 if runs <= 40 else (1024 if runs <= 160 else 512)
        m = meshgen.perturbed_grid(side, 0.3, seed=3)
        return m, f"perturbed grid {side}x{side} ({m.n_triangles:,} triangles), same recipe"
    if workload == "delaunay_1m":
        return meshgen.random_delaunay(1_000_000, seed=2), "the full 1M-point Delaunay mesh"
    return meshgen.workload(workload), f"the full {workload} mesh"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    mesh, sample = ref_sample_mesh(args.workload, runs=args.steps + args.warmup)
    meshes = mesh if isinstance(mesh, list) else [mesh]
    n_tri = sum(m.n_triangles for m in meshes)
    oracle.build()
    times = []
    n_poly = 0
    stage_s = {}
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rs = [oracle.run_mesh(m) for m in meshes]
        dt = time.perf_counter() - t0
        n_poly = sum(r.n_polygons for r in rs)
        if i >= args.warmup:
            times.append(dt)
            for r in rs:
                for k, v in r.times.items():
                    stage_s[k] = stage_s.get(k, 0.0) + v
    tot = sum(times)
    value = n_tri * len(times) / tot
    host = dict(host_info(), threads_used=1,
                stage_ms_per_step={k: 1e3 * v / len(times) for k, v in stage_s.items()})
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample, "triangles": n_tri,
                   "polygons": n_poly},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample}; single-threaded sequential oracle (1 of {os.cpu_count()} "
                                   f"host cores), {len(times)} timed runs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------

def run_gb300(args):
    # the batched and served workloads' host meshes are built meanwhile, in
    # spawned processes (single-GPU runs of the default workload only)
    bg = None
    if args.workload == "pgrid_4096" and not args.no_extras and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        bg = BackgroundPools(BATCH_RECIPE["meshes"])
    import numpy as np
    import torch

    from paper_2403_14723_gb300 import build, meshgen, polylla

    rank, ws, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build_library()
    mesh = meshgen.workload(args.workload)
    T, V, H = mesh.n_triangles, mesh.n_vertices, mesh.n_halfedges
    dm = polylla.DeviceMesh.from_host(mesh, device=dev)
    # a stream of its own (CUDA graphs cannot capture the legacy stream);
    # torch's work (the L2 flush, events) goes to it too
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = polylla.polylla_create(dm, stream=stream)
    lib = polylla.load_library()
    # launch settings picked by the library's autotuner on this mesh
    if args.no_autotune:
        tuning = polylla.polylla_get_tuning(ctx)
    else:
        tuning = polylla.polylla_autotune(ctx, reps=5, stream=stream)
    # the whole generate as one CUDA graph launch per step
    polylla.polylla_capture_graph(ctx, stream)

    def step():
        polylla.polylla_generate(ctx, stream)
        return polylla.polylla_get_polygons(ctx, stream)

    for _ in range(max(args.warmup, 3)):
        out = step()
    P, NF = out["n_polygons"], out["n_frontier"]

    # ---- timed region: K steps, each bracketed by events, L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    torch.cuda.synchronize()
    dist_barrier(ws)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i)
            starts[i].record(stream)
            polylla.polylla_generate(ctx, stream)
            ends[i].record(stream)
            launches += polylla.polylla_launch_count(ctx)
        torch.cuda.synchronize()
    dist_barrier(ws)
    o = polylla.polylla_get_polygons(ctx, stream)
    assert o["n_polygons"] == P and o["n_frontier"] == NF
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = dist_max(statistics.mean(step_ms), ws)
    value = ws * T / (ms * 1e-3)

    # ---- per-kernel times (CUDA events on the launching stream) ----------
    polylla.polylla_release_graph(ctx)
    polylla.polylla_set_timing(ctx, True)
    stage_acc = {}
    for i in range(min(args.steps, 50)):
        flush.fill_(i)
        polylla.polylla_generate(ctx, stream)
        for k, v in polylla.polylla_get_stage_times(ctx).items():
            stage_acc.setdefault(k, []).append(v)
    polylla.polylla_set_timing(ctx, False)
    stage_ms = {k: statistics.mean(v) for k, v in stage_acc.items()}
    total_alg, per_stage = algorithmic_bytes(T, V, NF, P)
    dominant = max(stage_ms, key=stage_ms.get)
    peak, peak_kind = measured_peaks()
    ach = per_stage[dominant] / (stage_ms[dominant] * 1e-3) / 1e9
    traffic = ncu_traffic(dominant, args.workload)
    kernels = {}
    for k, t_ms in stage_ms.items():
        if t_ms <= 0.0:
            continue
        share = per_stage.get(k, 0)
        tr = ncu_traffic(k, args.workload)
        kernels[k] = {"ms": t_ms, "share_bytes": share,
                      "frac": (share / (t_ms * 1e-3) / 1e9 / peak) if share else None,
                      "traffic": tr, "traffic_over_share": (tr / share) if (tr and share) else None}
    roofline = {
        "whole_step": {"algorithmic_bytes": total_alg, "achieved": total_alg / (ms * 1e-3) / 1e9,
                       "frac": total_alg / (ms * 1e-3) / 1e9 / peak, "ms": ms},
        "bound": "hbm", "kernel": dominant, "achieved": ach, "peak": peak, "unit": "GB/s",
        "frac": ach / peak, "peak_source": f"{peak_kind} hbm_gbs",
        "traffic": traffic,
        "algorithmic_bytes": per_stage[dominant],
        "stage_ms": stage_ms,
        "kernels": kernels,
    }

    # ---- the Lepp primitive over the same mesh (after a generate) ---------
    term_buf = torch.empty(T, dtype=torch.int32, device=dev)
    len_buf = torch.empty(T, dtype=torch.int32, device=dev)
    polylla.polylla_generate(ctx, stream)
    lib.polylla_lepp_terminal(ctypes.c_void_p(ctx), ctypes.c_void_p(term_buf.data_ptr()),
                              ctypes.c_void_p(len_buf.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    l_steps = max(3, min(args.steps, 50))
    ls = [torch.cuda.Event(enable_timing=True) for _ in range(l_steps)]
    le_ = [torch.cuda.Event(enable_timing=True) for _ in range(l_steps)]
    for i in range(l_steps):
        flush.fill_(i)
        ls[i].record(stream)
        lib.polylla_lepp_terminal(ctypes.c_void_p(ctx), ctypes.c_void_p(term_buf.data_ptr()),
                                  ctypes.c_void_p(len_buf.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        le_[i].record(stream)
    torch.cuda.synchronize()
    lepp_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(ls, le_))
    lepp_mean = float(len_buf.double().mean())
    lepp = {"ms": lepp_ms, "triangles_per_s": T / (lepp_ms * 1e-3), "mean_path_triangles": lepp_mean,
            "api": "polylla_lepp_terminal: terminal seed and path length of every triangle"}
    del term_buf, len_buf

    # ---- convexification of the same mesh (post-processing) --------------
    cv_steps = max(3, min(args.steps, 20))
    cs = [torch.cuda.Event(enable_timing=True) for _ in range(cv_steps)]
    ce = [torch.cuda.Event(enable_timing=True) for _ in range(cv_steps)]
    for i in range(cv_steps + 1):
        polylla.polylla_generate(ctx, stream)
        flush.fill_(i)
        if i > 0:
            cs[i - 1].record(stream)
        polylla.polylla_convexify(ctx, stream)
        if i > 0:
            ce[i - 1].record(stream)
    torch.cuda.synchronize()
    cv_out = polylla.polylla_get_polygons(ctx, stream)
    cv_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(cs, ce))
    convex = {"ms": cv_ms, "triangles_per_s": T / (cv_ms * 1e-3), "polygons_before": P,
              "polygons_after": cv_out["n_polygons"], "chords": cv_out["n_polygons"] - P,
              "frontier_halfedges_after": cv_out["n_frontier"],
              "api": "polylla_convexify after a generate: chords at reflex corners, relink, CSR again"}
    polylla.polylla_generate(ctx, stream)

    # the host-buffer copies below share the host's memory bandwidth with the
    # processes building the batched and served meshes: let those finish
    # first, so that the end-to-end figure sees a quiet host
    if bg is not None:
        meshes, gen_b = bg.batch()
        small, large, gen_s = bg.serve()
        bg.close()

    # ---- end to end through the host-buffer entry point ------------------
    e2e = None
    if not args.no_e2e:
        hctx = polylla.polylla_create_host(V, T, H)
        hin = {k: torch.from_numpy(getattr(mesh, k)).pin_memory() for k in ("coords", "origin", "twin", "next", "prev")}
        hout = {"seeds": torch.empty(T, dtype=torch.int32).pin_memory(),
                "offsets": torch.empty(T + 1, dtype=torch.int32).pin_memory(),
                "he_list": torch.empty(3 * T, dtype=torch.int32).pin_memory(),
                "v_list": torch.empty(3 * T, dtype=torch.int32).pin_memory(),
                "next": torch.empty(H, dtype=torch.int32).pin_memory(),
                "prev": torch.empty(H, dtype=torch.int32).pin_memory()}
        for _ in range(2):
            polylla.polylla_generate_host(hctx, hin, hout, stream=stream)
        e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        dist_barrier(ws)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            p2, nf2 = polylla.polylla_generate_host(hctx, hin, hout, stream=stream)
        torch.cuda.synchronize()
        dist_barrier(ws)
        e_ms = dist_max(1e3 * (time.perf_counter() - t0) / e_steps, ws)
        assert p2 == P and nf2 == NF
        polylla.polylla_destroy(hctx)
        h2d = 16 * V + 2 * 4 * H                     # coords, origin, twin (next/prev are not read)
        d2h = 4 * (P + (P + 1) + 2 * NF + 2 * 3 * T) + 32   # CSR, interior next/prev, control block
        e2e = {"value": ws * T / (e_ms * 1e-3), "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "polylla_generate_host (pinned host buffers, copies inside the timed region)"}
        # the same steps as a stream of requests through the serving loop:
        # one step's copies in overlap another's copies out (no small
        # requests here, so no low-latency lane)
        hr = polylla.HostRequest(mesh)
        with polylla.Server(memory_budget=SERVE_RECIPE["budget"], n_slots=3, lane_triangles=-1) as srv:
            srv.replay([hr] * 2, [0.0, 0.0])
            dist_barrier(ws)
            rc, lat, infos = srv.replay([hr] * e_steps, [0.0] * e_steps)
            assert rc == 0 and infos[-1]["n_polygons"] == P
            span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
        p_ms = dist_max(1e3 * span / e_steps, ws)
        e2e["pipelined"] = {"value": ws * T / (p_ms * 1e-3), "unit": UNIT, "ms_per_step": p_ms,
                            "api": f"polylla_server_replay of {e_steps} requests of the mesh, all arriving at once"}
        del hr

    polylla.polylla_destroy(ctx)
    clocks = clk.summary()
    del dm

    # ---- batched and served sub-records (same process, same GPU) --------
    batched = served = None
    if bg is not None:
        bctx, bdb, b = measure_batched(meshes, max(10, min(args.steps, 50)), args.warmup, dev, ws, local,
                                       clock=False)
        polylla.polylla_destroy(bctx)
        del bdb
        r = BATCH_RECIPE
        batched = {
            "workload": f"batch_{len(meshes)}", "meshes": len(meshes), "triangles": b["T"],
            "polygons": b["P"], "frontier_halfedges": b["NF"],
            "sizes": f"log-uniform [{r['t_min']}, {r['t_max']}] triangles, seed {r['seed']}; "
                     "even meshes Delaunay of uniform points, odd perturbed grids (jitter 0.3)",
            "value": b["T"] / (b["ms"] * 1e-3), "unit": UNIT, "ms_per_step": b["ms"],
            "steps": max(10, min(args.steps, 50)), "cuda_graph": True, "whole_step": b["whole_step"],
            "stage_ms": b["stage_ms"], "tuning": b["tuning"], "gpu_launches": b["launches"],
            "without_graph": {"value": b["T"] / (b["ms_nograph"] * 1e-3), "ms_per_step": b["ms_nograph"]},
            "one_mesh_at_a_time": {"value": b["T"] / (b["ms_loop"] * 1e-3), "unit": UNIT,
                                   "ms_per_step": b["ms_loop"], "launches_per_step": b["launches_loop"],
                                   "how": "polylla_generate per mesh, back to back on one stream"},
            "l2": f"256 MiB buffer written between timed steps; inputs {(16 * b['V'] + 16 * b['H']) / 1e9:.2f} GB",
            "host_generation_s": gen_b,
        }
        del meshes
        sv = measure_served(small, large, args.extras_serve_seconds, args.extras_serve_baseline_seconds,
                            args.serve_slots, args.serve_batch_triangles, args.serve_lane, rank, ws, local)
        m_, b_, st = sv["main"], sv["base"], sv["stats"]
        rs = SERVE_RECIPE
        served = {
            "workload": "served", "rate_req_per_s": rs["rate"], "seconds": args.extras_serve_seconds,
            "requests": m_["requests"], "triangles": m_["triangles"],
            "value": sv["value"], "unit": UNIT, "latency_ms": {"p50": m_["p50_ms"], "p99": m_["p99_ms"]},
            "queue_ms": m_["queue_ms"], "service_ms": m_["service_ms"], "mean_batch": m_["mean_batch"],
            "batches": sv["batches"], "gpu_launches": sv["launches"], "batch_trace": m_["batch_trace"],
            "mix": f"{int(100 * (1 - rs['p_large']))}% log-uniform {rs['small']} triangles, "
                   f"{int(100 * rs['p_large'])}% log-uniform {rs['large']}; Delaunay and perturbed grids",
            "pool": f"{len(small)} small + {len(large)} large seeded meshes in pinned host memory",
            "memory_budget_bytes": rs["budget"], "slots": st["n_slots"], "lane_triangles": st["lane_triangles"],
            "one_mesh_at_a_time": {"value": b_["tri_per_s"], "unit": UNIT, "seconds": args.extras_serve_baseline_seconds,
                                   "requests": b_["requests"],
                                   "latency_ms": {"p50": b_["p50_ms"], "p99": b_["p99_ms"]},
                                   "how": "same server loop with one slot and one mesh per batch, same recipe"},
            "copy_check": sv["copy_check"], "clocks": sv["clocks"], "host_generation_s": gen_s,
        }
        del small, large

    # ---- CPU baseline: the oracle, bounded sample, rank 0, N = 1 only -----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        smesh, sample = ref_sample_mesh(args.workload)
        oracle.build()
        runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            res = oracle.run_mesh(smesh)
            runs.append((time.perf_counter() - t0, res.times))
        runs.sort(key=lambda r: r[0])
        med, med_stages = runs[1]
        cpu = {"value": smesh.n_triangles / med, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample}; median of 3 single-threaded runs (1 of {os.cpu_count()} host cores)",
               "stage_ms": {k: 1e3 * v for k, v in med_stages.items()}, "host": host_info()}


    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/int32", "data": "synthetic",
            "config": {"workload": args.workload, "triangles": T, "vertices": V, "halfedges": H,
                       "polygons": P, "frontier_halfedges": NF, "parallelism": f"replicas x{ws}",
                       "tuning": tuning, "cuda_graph": True,
                       "l2": f"256 MiB buffer written between timed steps (L2 flush); inputs "
                             f"{(16 * V + 16 * H) / 1e9:.2f} GB"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "lepp": lepp,
            "batched": batched, "served": served, "convexify": convex,
            "gpu_launches": launches, "clocks": clocks,
            "kernel_digest": kernel_digest(), "core_kernel_digest": core_kernel_digest(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# batched workload: many meshes, one launch per stage
# ---------------------------------------------------------------------------

BATCH_RECIPE = {"meshes": 4096, "t_min": 100, "t_max": 200_000, "seed": 4}


def batch_meshes(n_meshes: int):
    from paper_2403_14723_gb300 import meshgen

    workers = max(1, min(16, os.cpu_count() or 1))
    r = BATCH_RECIPE
    return meshgen.random_batch(n_meshes, r["t_min"], r["t_max"], r["seed"], workers=workers)


def measure_batched(meshes, steps: int, warmup: int, dev, ws: int, local: int, clock: bool = True):
    """The batched mode on ``meshes``: autotuned, one CUDA graph launch per
    step, timed with CUDA events (L2 flushed between steps), beside the
    plain one-mesh-at-a-time path on the same meshes.  Returns the batch
    context (still alive, for the end-to-end leg), its device batch, and a
    dict of the measurements."""
    import numpy as np
    import torch

    from paper_2403_14723_gb300 import polylla

    n_meshes = len(meshes)
    db = polylla.DeviceBatch.from_host(meshes, device=dev)
    T = int(db.triangle_offset[-1])
    V = int(db.vertex_offset[-1])
    H = int(db.halfedge_offset[-1])
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    res = {}
    with torch.cuda.stream(stream):
        ctx = polylla.polylla_batch_create(db, stream=stream)
        tuning = polylla.polylla_autotune(ctx, reps=3, stream=stream)

        # per-stage times (CUDA events on the launching stream), untimed region
        polylla.polylla_set_timing(ctx, True)
        stage_acc = {}
        for i in range(10):
            flush.fill_(i)
            polylla.polylla_generate(ctx, stream)
            for k, v in polylla.polylla_get_stage_times(ctx).items():
                stage_acc.setdefault(k, []).append(v)
        polylla.polylla_set_timing(ctx, False)
        stage_ms = {k: statistics.mean(v) for k, v in stage_acc.items()}

        # without a graph (stream launches), a few steps
        def timed(k, fn):
            st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            for i in range(k):
                flush.fill_(i)
                st[i].record(stream)
                fn()
                en[i].record(stream)
            stream.synchronize()
            return statistics.mean(s.elapsed_time(e) for s, e in zip(st, en))

        def step():
            polylla.polylla_generate(ctx, stream)

        for _ in range(3):
            step()
        ms_nograph = timed(max(3, min(steps, 20)), step)
        polylla.polylla_capture_graph(ctx, stream)
        for _ in range(max(warmup, 3)):
            step()
        stream.synchronize()
        dist_barrier(ws)
        if clock:
            with ClockSampler(local) as clk:
                ms = timed(steps, step)
            res["clocks"] = clk.summary()
        else:
            ms = timed(steps, step)
        dist_barrier(ws)
        ms = dist_max(ms, ws)
        launches = steps * polylla.polylla_launch_count(ctx)
        out = polylla.polylla_get_polygons(ctx, stream)
        P, NF = out["n_polygons"], out["n_frontier"]
        po = polylla.polylla_batch_polygon_offsets(ctx, n_meshes).cpu().numpy()

        # ---- the plain one-mesh-at-a-time path on the same meshes --------
        dms = [polylla.DeviceMesh.from_host(m, device=dev) for m in meshes]
        ctxs = [polylla.polylla_create(d, stream=stream) for d in dms]

        def loop():
            for c in ctxs:
                polylla.polylla_generate(c, stream)

        loop()
        ms_loop = dist_max(timed(3, loop), ws)
        p_loop = [polylla.polylla_get_polygons(c, stream)["n_polygons"] for c in ctxs]
        assert np.array_equal(np.diff(po), np.array(p_loop)), "batched and per-mesh polygon counts differ"
        launches_loop = sum(polylla.polylla_launch_count(c) for c in ctxs)
        for c in ctxs:
            polylla.polylla_destroy(c)
        del dms
    total_alg, per_stage = algorithmic_bytes(T, V, NF, P)
    peak, peak_kind = measured_peaks()
    res.update({"T": T, "V": V, "H": H, "P": P, "NF": NF, "ms": ms, "ms_nograph": ms_nograph, "ms_loop": ms_loop,
                "launches_loop": launches_loop, "stage_ms": stage_ms, "tuning": tuning, "launches": launches,
                "stream": stream, "flush": flush,
                "whole_step": {"algorithmic_bytes": total_alg, "achieved": total_alg / (ms * 1e-3) / 1e9,
                               "frac": total_alg / (ms * 1e-3) / 1e9 / peak, "peak_source": f"{peak_kind} hbm_gbs"}})
    return ctx, db, res


def run_batched(args):
    n_meshes = int(args.workload.split("_")[1])
    meshes = batch_meshes(n_meshes)        # process pool, before any CUDA call
    import numpy as np
    import torch

    from paper_2403_14723_gb300 import build, polylla

    rank, ws, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build_library()
    ctx, db, res = measure_batched(meshes, args.steps, args.warmup, dev, ws, local)
    T, V, H, P, NF = res["T"], res["V"], res["H"], res["P"], res["NF"]
    ms, ms_nograph, ms_loop = res["ms"], res["ms_nograph"], res["ms_loop"]
    stage_ms, tuning, launches = res["stage_ms"], res["tuning"], res["launches"]
    stream = res["stream"]
    with torch.cuda.stream(stream):
        # ---- end to end: host arrays in, CSR and links out, copies timed ---
        e2e = None
        if not args.no_e2e:
            host = {k: torch.from_numpy(np.concatenate([getattr(m, k) for m in meshes])).pin_memory()
                    for k in ("coords", "origin", "twin", "next", "prev")}
            o_he = torch.empty(NF, dtype=torch.int32).pin_memory()
            o_v = torch.empty(NF, dtype=torch.int32).pin_memory()
            o_seed = torch.empty(P, dtype=torch.int32).pin_memory()
            o_off = torch.empty(P + 1, dtype=torch.int32).pin_memory()
            o_po = torch.empty(n_meshes + 1, dtype=torch.int32).pin_memory()
            o_nx = torch.empty(H, dtype=torch.int32).pin_memory()
            o_pv = torch.empty(H, dtype=torch.int32).pin_memory()

            def e2e_step():
                for k in ("coords", "origin", "twin", "next", "prev"):
                    getattr(db, k).copy_(host[k], non_blocking=True)
                polylla.polylla_generate(ctx, stream)
                o = polylla.polylla_get_polygons(ctx, stream)
                o_he.copy_(o["he_list"], non_blocking=True)
                o_v.copy_(o["v_list"], non_blocking=True)
                o_seed.copy_(o["seeds"], non_blocking=True)
                o_off.copy_(o["offsets"], non_blocking=True)
                o_po.copy_(polylla.polylla_batch_polygon_offsets(ctx, n_meshes), non_blocking=True)
                o_nx.copy_(db.next, non_blocking=True)
                o_pv.copy_(db.prev, non_blocking=True)
                stream.synchronize()

            e2e_step()
            e_steps = max(3, min(args.steps, 10))
            dist_barrier(ws)
            t0 = time.perf_counter()
            for _ in range(e_steps):
                e2e_step()
            e_ms = dist_max(1e3 * (time.perf_counter() - t0) / e_steps, ws)
            h2d = 16 * V + 4 * 4 * H
            d2h = 4 * (2 * NF + P + (P + 1) + (n_meshes + 1) + 2 * H) + 32
            e2e = {"value": ws * T / (e_ms * 1e-3), "unit": UNIT, "ms_per_step": e_ms,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "api": "pinned host arrays -> polylla_generate (batch, CUDA graph) -> CSR and links back"}
        polylla.polylla_destroy(ctx)

    total_alg, per_stage = algorithmic_bytes(T, V, NF, P)
    per_stage["batch_meta"] = 0                      # serving only
    dominant = max(stage_ms, key=stage_ms.get)
    peak, peak_kind = measured_peaks()
    ach = per_stage[dominant] / (stage_ms[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": f"{peak_kind} hbm_gbs", "traffic": ncu_traffic(dominant, args.workload),
                "algorithmic_bytes": per_stage[dominant], "stage_ms": stage_ms,
                "whole_step": {"algorithmic_bytes": total_alg, "achieved": total_alg / (ms * 1e-3) / 1e9,
                               "frac": total_alg / (ms * 1e-3) / 1e9 / peak}}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        sample = meshes[: min(len(meshes), 256)]
        t0 = time.perf_counter()
        for m in sample:
            oracle.run_mesh(m)
        dt = time.perf_counter() - t0
        cpu = {"value": sum(m.n_triangles for m in sample) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {len(sample)} meshes of the batch "
                         f"({sum(m.n_triangles for m in sample):,} triangles), one pass, single-threaded"}
    clocks = res.get("clocks")
    if rank == 0:
        r = BATCH_RECIPE
        line = {
            "metric": METRIC, "value": ws * T / (ms * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/int32", "data": "synthetic",
            "config": {"workload": args.workload, "meshes": n_meshes, "triangles": T, "vertices": V,
                       "halfedges": H, "polygons": P, "frontier_halfedges": NF,
                       "sizes": f"log-uniform [{r['t_min']}, {r['t_max']}] triangles, seed {r['seed']}; "
                                "even meshes Delaunay of uniform points, odd perturbed grids (jitter 0.3)",
                       "parallelism": f"replicas x{ws}", "cuda_graph": True, "tuning": tuning,
                       "l2": f"256 MiB buffer written between timed steps (L2 flush); inputs "
                             f"{(16 * V + 16 * H) / 1e9:.2f} GB"},
            "one_mesh_at_a_time": {"value": ws * T / (ms_loop * 1e-3), "unit": UNIT, "ms_per_step": ms_loop,
                                   "launches_per_step": res["launches_loop"],
                                   "how": "polylla_generate per mesh, back to back on one stream"},
            "without_graph": {"value": ws * T / (ms_nograph * 1e-3), "unit": UNIT, "ms_per_step": ms_nograph},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "kernel_digest": kernel_digest(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# served workload: Poisson request stream through the serving loop
# ---------------------------------------------------------------------------

SERVE_RECIPE = {"rate": 2000.0, "small": (1_000, 50_000), "large": (500_000, 8_000_000), "p_large": 0.2,
                "pool_small": 512, "pool_large": 32, "budget": 40 << 30, "seed": 5}


def serve_pool_args():
    """Arguments of meshgen's batch-member builder for the request pool:
    sizes log-uniform per band, Delaunay and perturbed grids alternately."""
    from paper_2403_14723_gb300 import meshgen

    r = SERVE_RECIPE
    small = meshgen.batch_sizes(r["pool_small"], *r["small"], seed=r["seed"])
    large = meshgen.batch_sizes(r["pool_large"], *r["large"], seed=r["seed"] + 1)
    return ([(i, int(t), 10_000 + r["seed"]) for i, t in enumerate(small)],
            [(i, int(t), 20_000 + r["seed"]) for i, t in enumerate(large)])


def serve_pool():
    """Seeded pool of request meshes (built in a spawned process pool)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from paper_2403_14723_gb300 import meshgen

    small_args, large_args = serve_pool_args()
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        ms = list(ex.map(meshgen._batch_member_args, small_args + large_args, chunksize=4))
    return ms[: len(small_args)], ms[len(small_args):]


def serve_trace(seconds: float, n_small: int, n_large: int, seed: int):
    """Poisson arrivals at the recipe's rate; each request picks a small
    pool mesh (80 %) or a large one (20 %)."""
    import numpy as np

    r = SERVE_RECIPE
    rng = np.random.default_rng(seed)
    n = int(r["rate"] * seconds * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / r["rate"], size=n))
    t = t[t < seconds]
    large = rng.random(len(t)) < r["p_large"]
    pick = np.where(large, n_small + rng.integers(0, n_large, len(t)), rng.integers(0, n_small, len(t)))
    return t, pick


def batch_trace(log):
    """Where the served batches' time went: percentiles of each segment of
    the server's batch log, and the slowest batches in full."""
    import numpy as np

    if not log:
        return None
    seg = {
        "host_enqueue_ms": [1e3 * (b["t_enqueued"] - b["t_form"]) for b in log],
        "in_ms": [b["in_ms"] for b in log], "run_ms": [b["run_ms"] for b in log],
        "idle_ms": [b["idle_ms"] for b in log], "out_ms": [b["out_ms"] for b in log],
        "host_meta_wait_ms": [1e3 * (b["t_meta_seen"] - b["t_enqueued"]) for b in log],
        "host_out_wait_ms": [1e3 * (b["t_done"] - b["t_out_enqueued"]) for b in log],
        "total_ms": [1e3 * (b["t_done"] - b["t_form"]) for b in log],
        # scheduler time spent enqueueing the result copies of a copy-engine batch
        "host_out_enqueue_ms": [1e3 * (b["t_out_enqueued"] - b["t_meta_seen"]) for b in log],
        # the slot's stream began the batch this long after the scheduler enqueued it
        "stream_start_delay_ms": [1e3 * (b["t_stream_start"] - b["t_form"]) for b in log if b["t_stream_start"] > 0],
        # the scheduler saw the metadata this long after the stream finished it
        "meta_notice_delay_ms": [1e3 * (b["t_meta_seen"] - b["t_meta_landed"]) for b in log
                                 if b["t_meta_landed"] > 0 and not b["lane"]],
        # host-observed time not covered by the batch's stream segments
        "host_gap_ms": [1e3 * (b["t_done"] - b["t_form"]) - (b["in_ms"] + b["run_ms"] + b["idle_ms"] + b["out_ms"])
                        for b in log],
    }
    out = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "max": float(np.max(v))}
           for k, v in seg.items() if v}
    slow = sorted(log, key=lambda b: b["t_done"] - b["t_form"])[-5:]
    out["batches"] = len(log)
    out["lane_batches"] = sum(1 for b in log if b["lane"])
    out["slowest"] = [{"total_ms": round(1e3 * (b["t_done"] - b["t_form"]), 3), "slot": b["slot"], "lane": b["lane"],
                       "requests": b["n_requests"], "triangles": b["n_triangles"],
                       "t_form_s": round(b["t_form"], 4),
                       **{k: round(b[k], 3) for k in ("in_ms", "run_ms", "idle_ms", "out_ms")},
                       "host_meta_wait_ms": round(1e3 * (b["t_meta_seen"] - b["t_enqueued"]), 3),
                       "host_out_enqueue_ms": round(1e3 * (b["t_out_enqueued"] - b["t_meta_seen"]), 3),
                       "host_out_wait_ms": round(1e3 * (b["t_done"] - b["t_out_enqueued"]), 3),
                       "stream_start_delay_ms": round(1e3 * (b["t_stream_start"] - b["t_form"]), 3),
                       "meta_notice_delay_ms": round(1e3 * (b["t_meta_seen"] - b["t_meta_landed"]), 3),
                       "host_enqueue_ms": round(1e3 * (b["t_enqueued"] - b["t_form"]), 3)} for b in slow]
    return out


def host_info() -> dict:
    """The host the CPU baseline ran on: architecture, core count and what
    lscpu reports of the CPU model."""
    import platform

    info = {"machine": platform.machine(), "cores": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return info
    for line in out.splitlines():
        k, _, v = line.partition(":")
        if k.strip() in ("Model name", "Vendor ID", "Socket(s)", "Core(s) per socket", "CPU max MHz"):
            info[k.strip()] = v.strip()
    return info


def measure_served(small, large, seconds: float, base_seconds: float, slots: int, batch_tri: int, lane: int,
                   rank: int, ws: int, local: int):
    """A Poisson request trace of the served recipe through the serving loop
    (continuous batching), and the same loop with one slot and one mesh per
    batch (the plain one-mesh-at-a-time GPU path) on a trace of the same
    recipe.  Returns a dict of the measurements."""
    import numpy as np
    import torch

    from paper_2403_14723_gb300 import polylla

    pool = small + large
    hrs = [polylla.HostRequest(m) for m in pool]
    tri = np.array([m.n_triangles for m in pool], dtype=np.int64)
    r = SERVE_RECIPE

    def replay(srv, secs, seed):
        t, pick = serve_trace(secs, len(small), len(large), seed)
        rc, lat, infos = srv.replay([hrs[i] for i in pick], t)
        assert rc == 0, f"served requests failed: {polylla.STATUS.get(rc, rc)}"
        span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
        wait = np.array([i["t_admit"] - i["t_submit"] for i in infos])
        serve = np.array([i["t_done"] - i["t_admit"] for i in infos])
        t_first = min(i["t_submit"] for i in infos)
        return {"requests": len(t), "triangles": int(tri[pick].sum()), "span_s": span,
                "batch_trace": batch_trace([b for b in srv.batch_log() if b["t_form"] >= t_first]),
                "queue_ms": {"p50": 1e3 * float(np.percentile(wait, 50)), "p99": 1e3 * float(np.percentile(wait, 99))},
                "service_ms": {"p50": 1e3 * float(np.percentile(serve, 50)), "p99": 1e3 * float(np.percentile(serve, 99))},
                "tri_per_s": float(tri[pick].sum()) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_batch": float(np.mean([i["batch_meshes"] for i in infos])),
                "h2d_bytes": int(sum(16 * pool[i].n_vertices + 8 * pool[i].n_halfedges for i in pick)),
                "d2h_bytes": int(sum(4 * (2 * infos[k]["n_polygons"] + 1 + 2 * infos[k]["n_frontier"] + 6 * pool[i].n_triangles)
                                     for k, i in enumerate(pick)))}

    # the copy engines' rate on an idle link, from the pool's largest pinned request
    big = max(range(len(pool)), key=lambda i: pool[i].n_halfedges)
    src = hrs[big].inp["origin"]
    dev = torch.empty(src.shape, dtype=src.dtype, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        ev[0].record()
        dev.copy_(src, non_blocking=True)
        ev[1].record()
        hrs[big].out["next"][: src.shape[0]].copy_(dev, non_blocking=True)
        ev[2].record()
        torch.cuda.synchronize()
    nbytes = src.numel() * src.element_size()
    copy_check = {"bytes": nbytes, "h2d_gbs": nbytes / (ev[0].elapsed_time(ev[1]) * 1e6),
                  "d2h_gbs": nbytes / (ev[1].elapsed_time(ev[2]) * 1e6)}
    del dev
    with polylla.Server(memory_budget=r["budget"], n_slots=slots,
                        max_batch_triangles=batch_tri, lane_triangles=lane) as srv:
        replay(srv, 1.0, seed=1000 + rank)                     # warm-up, untimed
        dist_barrier(ws)
        st0 = srv.stats()
        with ClockSampler(local) as clk:
            main = replay(srv, seconds, seed=r["seed"] + rank)
        st = srv.stats()
    with polylla.Server(memory_budget=r["budget"], n_slots=1, max_batch_meshes=1, lane_triangles=-1) as one:
        replay(one, 0.5, seed=2000 + rank)
        base = replay(one, base_seconds, seed=r["seed"] + rank)
    value = main["tri_per_s"]
    if ws > 1:
        import torch.distributed as dist

        tot = torch.tensor([float(main["triangles"])], dtype=torch.float64, device="cuda")
        dist.all_reduce(tot)
        value = float(tot[0]) / dist_max(main["span_s"], ws)
    del hrs
    return {"main": main, "base": base, "value": value, "stats": st, "copy_check": copy_check,
            "batches": int(st["batches"] - st0["batches"]), "launches": int(st["launches"] - st0["launches"]),
            "clocks": clk.summary()}


def run_served(args):
    small, large = serve_pool()               # process pool, before any CUDA call
    import torch

    from paper_2403_14723_gb300 import build

    rank, ws, local = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(torch.device("cuda", local))
    build.build_library()
    res = measure_served(small, large, args.serve_seconds, args.serve_baseline_seconds, args.serve_slots,
                         args.serve_batch_triangles, args.serve_lane, rank, ws, local)
    main, base, st, value = res["main"], res["base"], res["stats"], res["value"]
    r = SERVE_RECIPE
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": main["requests"], "warmup": 1,
            "ms_per_step": 1e3 * main["span_s"] / main["requests"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/int32", "data": "synthetic",
            "config": {"workload": "served", "rate_req_per_s": r["rate"], "seconds": args.serve_seconds,
                       "requests": main["requests"], "triangles": main["triangles"],
                       "mix": f"{int(100 * (1 - r['p_large']))}% log-uniform {r['small']} triangles, "
                              f"{int(100 * r['p_large'])}% log-uniform {r['large']}; Delaunay and perturbed grids",
                       "pool": f"{len(small)} small + {len(large)} large seeded meshes in pinned host memory",
                       "memory_budget_bytes": r["budget"], "slots": st["n_slots"],
                       "max_batch_triangles": args.serve_batch_triangles,
                       "lane_triangles": st["lane_triangles"],
                       "slot_triangles": st["slot_triangles"], "device_bytes": st["device_bytes"],
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"]},
            "served": main, "server_stats": st, "copy_check": res["copy_check"], "batches": res["batches"],
            "one_mesh_at_a_time": dict(base, how="same server loop with one slot and one mesh per batch, "
                                                  f"{args.serve_baseline_seconds:g} s of the same recipe"),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": main["h2d_bytes"] // max(1, main["requests"]),
                    "d2h_bytes_per_step": main["d2h_bytes"] // max(1, main["requests"]),
                    "api": "polylla_server_replay: host meshes in, host results out, per request"},
            "roofline": None, "cpu_baseline": None,
            "gpu_launches": res["launches"], "clocks": res["clocks"], "kernel_digest": kernel_digest(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


class BackgroundPools:
    """The batched workload's meshes and the served workload's request pool,
    built in a spawned process pool while the caller measures the single
    mesh on the GPU (spawned workers hold no CUDA state)."""

    def __init__(self, n_batch: int):
        import concurrent.futures as cf
        import multiprocessing as mp

        from paper_2403_14723_gb300 import meshgen

        workers = max(1, min(16, (os.cpu_count() or 2) - 2))
        self.t0 = time.perf_counter()
        self.ex = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
        rb = BATCH_RECIPE
        bsizes = meshgen.batch_sizes(n_batch, rb["t_min"], rb["t_max"], rb["seed"])
        self.n_batch = n_batch
        self.batch_it = self.ex.map(meshgen._batch_member_args, [(i, int(t), rb["seed"]) for i, t in enumerate(bsizes)],
                                    chunksize=16)
        small_args, large_args = serve_pool_args()
        self.n_small = len(small_args)
        self.serve_it = self.ex.map(meshgen._batch_member_args, small_args + large_args, chunksize=4)
        self.workers = workers

    def batch(self):
        meshes = list(self.batch_it)
        return meshes, time.perf_counter() - self.t0

    def serve(self):
        ms = list(self.serve_it)
        return ms[: self.n_small], ms[self.n_small:], time.perf_counter() - self.t0

    def close(self):
        self.ex.shutdown(wait=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch_"):
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
