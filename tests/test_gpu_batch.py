"""Batches through the C ABI: one launch per stage over many meshes must give
every mesh exactly what the oracle gives it alone (bit-exact: links, seeds,
CSR, labels), also when replayed from a CUDA graph and after autotuning."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import build, meshgen, polylla
from tests.gpu_helpers import oracle_labels

pytestmark = pytest.mark.gpu


def _tip_meshes(n):
    out = []
    for s in range(80):
        m = meshgen.random_delaunay(150, seed=7000 + s)
        if oracle.run_mesh(m).stats["tips"] >= 1:
            out.append(m)
        if len(out) >= n:
            break
    return out


def _mix():
    ms = [
        meshgen.two_triangle_square(),
        meshgen.from_triangles([[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], name="one_triangle"),
        meshgen.exact_grid(5),
        meshgen.perturbed_grid(24, 0.3, seed=11),
        meshgen.random_delaunay(60, seed=100),
        meshgen.random_delaunay(2000, seed=1),
    ]
    ms += _tip_meshes(3)
    ms += meshgen.random_batch(20, t_min=100, t_max=20_000, seed=40)
    ms.insert(4, meshgen.exact_grid(2))
    return ms


def batch_run(meshes, graph=False, tune=False, generate_times=1, unaligned=False, tuning=None):
    import torch

    build.build_library()
    db = polylla.DeviceBatch.from_host(meshes)
    if unaligned:
        # origin and twin one entry past a 16-byte boundary: the listing kernel
        # cannot bulk-copy a tile's local origins and loads them one by one
        for name in ("origin", "twin"):
            a = getattr(db, name)
            buf = torch.empty(a.numel() + 1, dtype=a.dtype, device=a.device)
            buf[1:].copy_(a)
            setattr(db, name, buf[1:])
            assert getattr(db, name).data_ptr() % 16 == 4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = polylla.polylla_batch_create(db, stream=stream)
        try:
            if tune:
                polylla.polylla_autotune(ctx, reps=2, stream=stream)
            if tuning:
                polylla.polylla_set_tuning(ctx, dict(polylla.polylla_get_tuning(ctx), **tuning))
            if graph:
                polylla.polylla_capture_graph(ctx, stream)
            for _ in range(generate_times):
                polylla.polylla_generate(ctx, stream)
            out = polylla.polylla_get_polygons(ctx, stream)
            po = polylla.polylla_batch_polygon_offsets(ctx, len(meshes)).cpu().numpy()
            lab = polylla.polylla_get_labels(ctx, int(db.triangle_offset[-1]), stream)
            stream.synchronize()
            res = {k: out[k].cpu().numpy() for k in ("seeds", "offsets", "he_list", "v_list")}
            res.update(n_polygons=out["n_polygons"], n_frontier=out["n_frontier"], poly_offset=po,
                       next=db.next.cpu().numpy(), prev=db.prev.cpu().numpy(),
                       le=lab["longest_local"].cpu().numpy(), flags=lab["flags"].cpu().numpy(),
                       launches=polylla.polylla_launch_count(ctx))
        finally:
            polylla.polylla_destroy(ctx)
    return db, res


def assert_batch_parity(meshes, db, g):
    ho, to = db.halfedge_offset, db.triangle_offset
    po = g["poly_offset"]
    assert po[0] == 0 and po[-1] == g["n_polygons"]
    assert g["offsets"][g["n_polygons"]] == g["n_frontier"]
    for i, m in enumerate(meshes):
        r = oracle.run_mesh(m)
        tag = f"mesh {i} ({m.name}, T={m.n_triangles})"
        assert np.array_equal(g["next"][ho[i]:ho[i + 1]], r.next_out), f"{tag}: next"
        assert np.array_equal(g["prev"][ho[i]:ho[i + 1]], r.prev_out), f"{tag}: prev"
        le, _, f1, _ = oracle_labels(m, r)
        assert np.array_equal(g["le"][to[i]:to[i + 1]], le), f"{tag}: longest edges"
        gf1 = np.stack([(g["flags"][to[i]:to[i + 1]] >> k) & 1 for k in range(3)], axis=1)
        assert np.array_equal(gf1, f1), f"{tag}: frontier"
        p0, p1 = po[i], po[i + 1]
        assert p1 - p0 == r.n_polygons, f"{tag}: {p1 - p0} polygons vs {r.n_polygons}"
        assert np.array_equal(g["seeds"][p0:p1], r.seeds), f"{tag}: seeds"
        off = g["offsets"][p0:p1 + 1]
        assert np.array_equal(off - off[0], r.offsets), f"{tag}: offsets"
        assert np.array_equal(g["he_list"][off[0]:off[-1]], r.he_list), f"{tag}: he_list"
        assert np.array_equal(g["v_list"][off[0]:off[-1]], r.v_list), f"{tag}: v_list"


def test_batch_matches_oracle_per_mesh():
    meshes = _mix()
    db, g = batch_run(meshes)
    assert g["launches"] == 7
    assert_batch_parity(meshes, db, g)


def test_batch_with_unaligned_local_arrays():
    meshes = _mix()
    db, g = batch_run(meshes, unaligned=True)
    assert_batch_parity(meshes, db, g)


def test_batch_generate_twice_and_from_a_graph():
    meshes = _mix()
    db, g = batch_run(meshes, graph=True, generate_times=2)
    assert_batch_parity(meshes, db, g)


# every relink launch setting: one triangle per thread (64, 128 or 256 per
# CTA) runs the one-rotation-per-thread kernel, two or four per thread the
# kernel with per-warp rotation lists
RELINK_SETTINGS = [(64, 1), (128, 1), (256, 1), (256, 2), (256, 4)]


@pytest.mark.parametrize("tile,items", RELINK_SETTINGS)
def test_batch_every_relink_setting(tile, items):
    meshes = _mix()
    db, g = batch_run(meshes, tuning={"relink_tile": tile, "relink_items": items})
    assert_batch_parity(meshes, db, g)


def test_batch_after_autotune():
    meshes = meshgen.random_batch(12, t_min=1000, t_max=60_000, seed=41)
    db, g = batch_run(meshes, tune=True)
    assert_batch_parity(meshes, db, g)
    polylla.polylla_tuning_cache_clear()


def test_batch_rejects_out_of_range_local_index():
    import torch

    build.build_library()
    meshes = [meshgen.exact_grid(4), meshgen.random_delaunay(100, seed=3)]
    db = polylla.DeviceBatch.from_host(meshes)
    # a twin of mesh 0 pointing past its own half-edges (into mesh 1's range)
    db.twin[0] = int(meshes[0].n_halfedges)
    with pytest.raises(polylla.PolyllaError) as e:
        polylla.polylla_batch_create(db)
    assert e.value.status == -2
    torch.cuda.synchronize()


def test_single_mesh_graph_and_tuning_keep_results():
    import torch

    build.build_library()
    mesh = meshgen.perturbed_grid(200, 0.3, seed=12)
    r = oracle.run_mesh(mesh)
    dm = polylla.DeviceMesh.from_host(mesh)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with polylla.Polylla(dm, stream=stream) as p:
            t = polylla.polylla_autotune(p.ctx, reps=2, stream=stream)
            assert (t["relink_tile"], t["relink_items"]) in ((64, 1), (128, 1), (256, 1), (256, 2), (256, 4))
            assert (t["output_tile"], t["output_items"]) in ((1024, 2), (1024, 4), (2048, 2), (2048, 4),
                                                             (4096, 4))
            assert polylla.polylla_get_tuning(p.ctx) == t
            with pytest.raises(polylla.PolyllaError):
                polylla.polylla_set_tuning(p.ctx, dict(t, output_tile=3072))
            with pytest.raises(polylla.PolyllaError):
                polylla.polylla_set_tuning(p.ctx, dict(t, relink_items=3))
            polylla.polylla_capture_graph(p.ctx, stream)
            dm.next.fill_(-1)
            dm.prev.fill_(-1)
            p.generate(stream)
            out = p.polygons(stream)
            stream.synchronize()
            assert polylla.polylla_launch_count(p.ctx) == 7
            assert np.array_equal(dm.next.cpu().numpy()[:3 * mesh.n_triangles], r.next_out[:3 * mesh.n_triangles])
            assert np.array_equal(out["he_list"].cpu().numpy(), r.he_list)
            assert np.array_equal(out["seeds"].cpu().numpy(), r.seeds)
    polylla.polylla_tuning_cache_clear()


def test_batch_4096_full_size_matches_oracle():
    """The batched workload at full size (4,096 meshes, 111M triangles), in
    the launch configuration bench.py times (autotuned, from a CUDA graph):
    every mesh against its own oracle run."""
    import bench

    meshes = bench.batch_meshes(4096)
    db, g = batch_run(meshes, graph=True, tune=True)
    assert_batch_parity(meshes, db, g)
    polylla.polylla_tuning_cache_clear()


def test_unvalidated_batch_with_out_of_range_index_reports_invalid_mesh():
    import torch

    build.build_library()
    meshes = [meshgen.exact_grid(5), meshgen.random_delaunay(200, seed=4)]
    db = polylla.DeviceBatch.from_host(meshes)
    ctx = polylla.polylla_batch_create(db, validate=False)
    try:
        db.twin[meshes[0].n_halfedges + 3] = -12345      # a twin of mesh 1, out of range
        polylla.polylla_generate(ctx)
        with pytest.raises(polylla.PolyllaError) as e:
            polylla.polylla_get_polygons(ctx)
        assert e.value.status == -2
        torch.cuda.synchronize()
    finally:
        polylla.polylla_destroy(ctx)
