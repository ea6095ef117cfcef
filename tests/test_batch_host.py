"""Host-side checks of batches (no GPU).

The batched path rests on one claim: running the method once on the union
of independent meshes -- interior half-edges of all meshes first, in mesh
order, then all border half-edges, vertex ids shifted -- gives every mesh
exactly its own result.  The oracle (independent of the CUDA path) checks
that claim here on a numpy-built union; the GPU tests then compare the
batched CUDA path with per-mesh oracle runs.
"""
import numpy as np

import oracle
from paper_2403_14723_gb300 import meshgen, polylla


def union_of(meshes):
    """The union layout, built with numpy (test code, not the library's)."""
    T = np.array([m.n_triangles for m in meshes])
    H = np.array([m.n_halfedges for m in meshes])
    V = np.array([m.n_vertices for m in meshes])
    t_off = np.concatenate([[0], np.cumsum(T)])
    v_off = np.concatenate([[0], np.cumsum(V)])
    b_off = np.concatenate([[0], np.cumsum(H - 3 * T)])
    HI = 3 * int(t_off[-1])

    def remap(i, x):
        x = x.astype(np.int64)
        return np.where(x < 3 * T[i], 3 * t_off[i] + x, HI + b_off[i] + (x - 3 * T[i]))

    parts = {k: [None] * (2 * len(meshes)) for k in ("origin", "twin", "next", "prev")}
    for i, m in enumerate(meshes):
        n_int = 3 * m.n_triangles
        for k in ("twin", "next", "prev"):
            a = remap(i, getattr(m, k))
            parts[k][i] = a[:n_int]
            parts[k][len(meshes) + i] = a[n_int:]
        o = m.origin.astype(np.int64) + v_off[i]
        parts["origin"][i] = o[:n_int]
        parts["origin"][len(meshes) + i] = o[n_int:]
    u = meshgen.HalfEdgeMesh(
        coords=np.concatenate([m.coords for m in meshes]),
        **{k: np.concatenate(v).astype(np.int32) for k, v in parts.items()},
        n_triangles=int(t_off[-1]), name="union")
    return u, t_off, v_off


def test_union_gives_each_mesh_its_own_result():
    meshes = [meshgen.two_triangle_square(), meshgen.exact_grid(4),
              meshgen.random_delaunay(150, seed=7003), meshgen.perturbed_grid(9, 0.3, seed=5),
              meshgen.random_delaunay(400, seed=11)]
    u, t_off, v_off = union_of(meshes)
    ru = oracle.run_mesh(u)
    p = 0
    for i, m in enumerate(meshes):
        r = oracle.run_mesh(m)
        n = r.n_polygons
        seeds = ru.seeds[p:p + n]
        assert np.all((seeds >= 3 * t_off[i]) & (seeds < 3 * t_off[i + 1])), "polygons are ordered by mesh"
        assert np.array_equal(seeds - 3 * t_off[i], r.seeds)
        off = ru.offsets[p:p + n + 1]
        assert np.array_equal(off - off[0], r.offsets)
        assert np.array_equal(ru.he_list[off[0]:off[-1]] - 3 * t_off[i], r.he_list)
        assert np.array_equal(ru.v_list[off[0]:off[-1]] - v_off[i], r.v_list)
        lo, hi = 3 * t_off[i], 3 * t_off[i + 1]
        assert np.array_equal(ru.next_out[lo:hi] - lo, r.next_out[:3 * m.n_triangles])
        assert np.array_equal(ru.prev_out[lo:hi] - lo, r.prev_out[:3 * m.n_triangles])
        p += n
    assert p == ru.n_polygons


def test_batch_sizes_are_log_uniform_within_bounds():
    s = meshgen.batch_sizes(4096, 100, 200_000, seed=4)
    assert s.min() >= 100 and s.max() <= 200_000
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(np.log(np.median(s)) - 0.5 * (np.log(100) + np.log(200_000))) < 0.25
    assert np.array_equal(s, meshgen.batch_sizes(4096, 100, 200_000, seed=4))


def test_batch_members_alternate_generators_near_target_size():
    for i, t in enumerate([100, 1000, 5000, 20_000]):
        m = meshgen.batch_member(i, t, seed=4)
        assert 0.6 * t <= m.n_triangles <= 1.4 * t, (i, t, m.n_triangles)
        assert ("delaunay" in m.name) == (i % 2 == 0), m.name


def test_device_batch_offsets_on_cpu():
    meshes = [meshgen.exact_grid(3), meshgen.random_delaunay(50, seed=2)]
    db = polylla.DeviceBatch.from_host(meshes, device="cpu")
    assert db.n_meshes == 2
    assert list(db.triangle_offset) == [0, meshes[0].n_triangles, meshes[0].n_triangles + meshes[1].n_triangles]
    assert list(db.halfedge_offset) == [0, meshes[0].n_halfedges, meshes[0].n_halfedges + meshes[1].n_halfedges]
    assert list(db.vertex_offset) == [0, meshes[0].n_vertices, meshes[0].n_vertices + meshes[1].n_vertices]
    assert db.origin.numel() == db.halfedge_offset[-1]
