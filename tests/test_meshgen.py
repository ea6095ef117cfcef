"""The synthetic input generators produce valid half-edge meshes of the
stated shapes (workload recipe), deterministically from their seeds."""
import numpy as np
import pytest

from paper_2403_14723_gb300 import meshgen


def _check_layout(m):
    H, T = m.n_halfedges, m.n_triangles
    HI = 3 * T
    idx = np.arange(H)
    assert m.origin.dtype == np.int32 and m.twin.dtype == np.int32
    assert np.all(m.twin[m.twin] == idx) and np.all(m.twin != idx)
    assert np.all(m.next[m.prev] == idx) and np.all(m.prev[m.next] == idx)
    t3 = (idx[:HI] // 3) * 3
    assert np.all(m.next[:HI] == t3 + (idx[:HI] + 1) % 3)
    assert np.all(m.prev[:HI] == t3 + (idx[:HI] + 2) % 3)
    assert np.all(m.origin[m.next] == m.origin[m.twin])       # target(e) = origin(next e)
    assert np.all(m.twin[HI:] < HI)                           # border halves pair with interior ones
    assert np.all(m.next[HI:] >= HI)
    tri = m.triangles()
    a, b, c = m.coords[tri[:, 0]], m.coords[tri[:, 1]], m.coords[tri[:, 2]]
    orient = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(orient > 0)
    # Euler for a triangulated disk: V - E + T = 1
    E = (HI - m.n_border) // 2 + m.n_border
    assert m.n_vertices - E + T == 1


@pytest.mark.parametrize("make", [
    lambda: meshgen.exact_grid(7),
    lambda: meshgen.perturbed_grid(40, 0.3, seed=3),
    lambda: meshgen.random_delaunay(2000, seed=1),
    lambda: meshgen.lattice_delaunay(150, 16, seed=4),
    meshgen.two_triangle_square,
])
def test_layout(make):
    _check_layout(make())


def test_workload_sizes():
    m = meshgen.workload("delaunay_2k")
    assert m.n_vertices == 2000 and 3900 <= m.n_triangles <= 4000
    g = meshgen.perturbed_grid(129, 0.3, seed=3)
    assert g.n_triangles == 2 * 128 * 128 and g.n_border == 4 * 128
    # unit square exactly: boundary vertices are not jittered
    assert g.coords.min() == 0.0 and g.coords.max() == 1.0


def test_deterministic():
    a = meshgen.random_delaunay(500, seed=9)
    b = meshgen.random_delaunay(500, seed=9)
    for f in ("coords", "origin", "twin", "next", "prev"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = meshgen.perturbed_grid(30, 0.3, seed=5)
    d = meshgen.perturbed_grid(30, 0.3, seed=5)
    assert np.array_equal(c.coords, d.coords) and np.array_equal(c.origin, d.origin)


def test_exact_grid_is_algorithm_15():
    s = 4
    m = meshgen.exact_grid(s)
    # faces (k, k+1, k+s+1) and (k, k+s+1, k+s) for every k with k mod s != s-1
    want = []
    for k in range(s * s - s):
        if k % s != s - 1:
            want += [[k, k + 1, k + s + 1], [k, k + s + 1, k + s]]
    assert m.triangles().tolist() == want
