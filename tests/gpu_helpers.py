"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle array by array (all outputs are integer, so the
bar is bit-exact equality)."""
from __future__ import annotations

import numpy as np

from paper_2403_14723_gb300 import build, polylla


def gpu_run(mesh, generate_times: int = 1, max_rotation: int = 0, tuning: dict | None = None,
            as_benched: bool = False) -> dict:
    """Upload ``mesh``, run polylla_generate ``generate_times`` times (with
    the launch settings ``tuning`` overriding the current ones, if given; or,
    with ``as_benched``, as bench.py times it: on a side stream, autotuned,
    from a captured CUDA graph) and return every output as numpy arrays."""
    import torch

    build.build_library()
    dm = polylla.DeviceMesh.from_host(mesh)
    stream = torch.cuda.Stream() if as_benched else torch.cuda.current_stream()
    with torch.cuda.stream(stream), polylla.Polylla(dm, max_rotation=max_rotation, stream=stream) as p:
        if tuning:
            polylla.polylla_set_tuning(p.ctx, dict(polylla.polylla_get_tuning(p.ctx), **tuning))
        if as_benched:
            polylla.polylla_autotune(p.ctx, reps=2, stream=stream)
            polylla.polylla_capture_graph(p.ctx, stream)
            dm.next[:3 * mesh.n_triangles].fill_(-1)   # generate never reads interior next/prev
            dm.prev[:3 * mesh.n_triangles].fill_(-1)
        for _ in range(generate_times):
            p.generate(stream)
        out = p.polygons(stream)
        lab = p.labels(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        res = {
            "n_polygons": out["n_polygons"], "n_frontier": out["n_frontier"],
            "seeds": out["seeds"].cpu().numpy(), "offsets": out["offsets"].cpu().numpy(),
            "he_list": out["he_list"].cpu().numpy(), "v_list": out["v_list"].cpu().numpy(),
            "next": dm.next.cpu().numpy(), "prev": dm.prev.cpu().numpy(),
            "le": lab["longest_local"].cpu().numpy(), "flags": lab["flags"].cpu().numpy(),
            "tips": lab["tips"].cpu().numpy(), "chords": lab["chords"].cpu().numpy(),
        }
    return res


def oracle_labels(mesh, r):
    """Per-triangle views of the oracle's per-half-edge labels."""
    T = mesh.n_triangles
    HI = 3 * T
    le = np.argmax(r.longest[:HI].reshape(T, 3), axis=1).astype(np.uint8)
    f0 = r.frontier0[:HI].reshape(T, 3).astype(np.uint8)
    f1 = r.frontier1[:HI].reshape(T, 3).astype(np.uint8)
    seed = np.zeros(T, np.uint8)
    seed[r.seed_list // 3] = 1
    assert np.all(le[r.seed_list // 3] == r.seed_list % 3)
    return le, f0, f1, seed


def assert_parity(mesh, g: dict, r) -> None:
    """Bit-exact comparison of every stage's output with the oracle."""
    T = mesh.n_triangles
    le, f0, f1, seed = oracle_labels(mesh, r)
    assert np.array_equal(g["le"], le), f"stage 1 longest edge: {np.count_nonzero(g['le'] != le)} triangles differ"
    gf1 = np.stack([(g["flags"] >> k) & 1 for k in range(3)], axis=1).astype(np.uint8)
    gseed = (g["flags"] >> 6) & 1
    # tips: the same set of (frontier half-edge, chord) pairs, any order
    gp = sorted(zip(g["tips"].tolist(), g["chords"].tolist()))
    op = sorted(zip(r.tip_out.tolist(), r.chord.tolist()))
    assert gp == op, f"stage 5a tips/chords differ ({len(gp)} vs {len(op)})"
    assert np.array_equal(gf1, f1), "stage 5a frontier after repair differs"
    # stage 2: F0 = F1 without the chord half-edges
    gf0 = gf1.reshape(-1).copy()
    if len(g["chords"]):
        gf0[g["chords"]] = 0
        gf0[mesh.twin[g["chords"]]] = 0
    assert np.array_equal(gf0.reshape(T, 3), f0), "stage 2 frontier labels differ"
    assert np.array_equal(gseed, seed), "stage 3 seeds differ"
    # walk-start marks: only on frontier half-edges, and on every polygon seed
    gmark = np.stack([(g["flags"] >> (3 + k)) & 1 for k in range(3)], axis=1).reshape(-1).astype(bool)
    assert not np.any(gmark & ~gf1.reshape(-1).astype(bool)), "walk-start mark on a non-frontier half-edge"
    assert np.all(gmark[r.seeds]), "a polygon seed has no walk-start mark"
    assert np.array_equal(g["next"], r.next_out), f"next differs at {np.count_nonzero(g['next'] != r.next_out)} half-edges"
    assert np.array_equal(g["prev"], r.prev_out), f"prev differs at {np.count_nonzero(g['prev'] != r.prev_out)} half-edges"
    assert g["n_polygons"] == r.n_polygons, f"P {g['n_polygons']} vs {r.n_polygons}"
    assert g["n_frontier"] == r.he_list.shape[0]
    assert np.array_equal(g["seeds"], r.seeds), "seeds differ"
    assert np.array_equal(g["offsets"], r.offsets), "offsets differ"
    assert np.array_equal(g["he_list"], r.he_list), "he_list differs"
    assert np.array_equal(g["v_list"], r.v_list), "v_list differs"
