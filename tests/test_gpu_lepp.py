"""The Lepp primitive (Definition 1) through the C ABI against the oracle's
Lepp, bit for bit: every triangle's terminal seed and path length, and the
paths of query triangles (offsets and triangle lists), on small meshes, the
1M-point Delaunay mesh and the 4096 x 4096 grid; cut paths and bad queries
are reported, not faulted."""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import build, meshgen, polylla

pytestmark = pytest.mark.gpu

MESHES = [
    meshgen.two_triangle_square,
    lambda: meshgen.from_triangles([[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], name="one_triangle"),
    lambda: meshgen.exact_grid(9),
    lambda: meshgen.perturbed_grid(64, 0.3, seed=5),
    lambda: meshgen.random_delaunay(3000, seed=6),
    lambda: meshgen.workload("delaunay_1m"),
    lambda: meshgen.workload("pgrid_4096"),
]


def _run(mesh, queries=None, capacity=None):
    import torch

    build.build_library()
    dm = polylla.DeviceMesh.from_host(mesh)
    with polylla.Polylla(dm) as p:
        p.generate()
        term, length = polylla.polylla_lepp_terminal(p.ctx, mesh.n_triangles)
        out = {"terminal": term.cpu().numpy(), "length": length.cpu().numpy()}
        if queries is not None:
            q = torch.from_numpy(np.ascontiguousarray(queries, dtype=np.int32)).cuda()
            off, paths = polylla.polylla_lepp_paths(p.ctx, q, capacity)
            torch.cuda.synchronize()
            out["offsets"] = off.cpu().numpy()
            out["paths"] = paths.cpu().numpy()
        out["status"] = polylla.polylla_last_error(p.ctx)
    return out


@pytest.mark.parametrize("make", MESHES, ids=lambda f: getattr(f, "__name__", "mesh"))
def test_lepp_matches_oracle(make):
    mesh = make()
    r = oracle.run_mesh(mesh)
    want_t, want_l = oracle.lepp(mesh, r.longest)
    rng = np.random.default_rng(mesh.n_triangles)
    q = rng.integers(0, mesh.n_triangles, size=min(mesh.n_triangles, 3000))
    cap = int(want_l[q].sum())
    g = _run(mesh, q, cap)
    assert g["status"] == 0
    assert np.array_equal(g["terminal"], want_t), "terminal seeds differ"
    assert np.array_equal(g["length"], want_l), "path lengths differ"
    assert np.array_equal(np.diff(g["offsets"]), want_l[q]) and g["offsets"][0] == 0
    for i in range(0, len(q), max(1, len(q) // 300)):
        got = g["paths"][g["offsets"][i]: g["offsets"][i + 1]]
        assert np.array_equal(got, oracle.lepp_path(mesh, r.longest, int(q[i]))), f"path of triangle {q[i]}"


def test_lepp_paths_past_capacity_and_bad_query_are_reported():
    mesh = meshgen.random_delaunay(500, seed=8)
    r = oracle.run_mesh(mesh)
    _, want_l = oracle.lepp(mesh, r.longest)
    q = np.arange(50)
    g = _run(mesh, q, int(want_l[q].sum()) - 5)          # 5 entries short
    assert g["status"] == -6
    assert g["offsets"][-1] == int(want_l[q].sum())
    q = np.array([0, 1, mesh.n_triangles + 7, 2])         # one query outside the mesh
    g = _run(mesh, q, 100)
    assert g["status"] == -2
    assert g["offsets"][3] - g["offsets"][2] == 0
