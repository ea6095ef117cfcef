"""Pins of the oracle's Lepp (Definition 1) against things other than itself:
a brute-force chase over longest edges recomputed from the triangles' own
vertex lists, the recursion the definition implies (a path is one triangle
followed by its neighbour's path), the closed form of the paper's grid, and
the terminal-edge regions as components over non-frontier edges
(Definitions 2-3)."""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen
from tests import checks


def _meshes():
    out = [meshgen.two_triangle_square(), meshgen.exact_grid(6), meshgen.perturbed_grid(24, 0.3, seed=11),
           meshgen.from_triangles([[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], name="one_triangle")]
    for s in range(3):
        out.append(meshgen.random_delaunay(60 + 70 * s, seed=300 + s))
    try:
        out.append(meshgen.lattice_delaunay(120, 14, seed=201))
    except ValueError:
        pass
    return out


@pytest.mark.parametrize("mesh", _meshes(), ids=lambda m: m.name)
def test_lepp_terminal_matches_brute_force(mesh):
    pin_lepp_terminal(mesh)


def pin_lepp_terminal(mesh, lib=None):
    r = oracle.run_mesh(mesh, lib=lib)
    term, length = oracle.lepp(mesh, r.longest, lib=lib)
    le_bf = checks.brute_force_longest(mesh)
    assert np.array_equal(term, checks.lepp_terminal(mesh, le_bf))
    # regions grouped by terminal edge are the components over non-frontier edges
    comp = checks.components_over_nonfrontier(mesh, r.frontier0)
    pairs = set(zip(comp.tolist(), term.tolist()))
    assert len(pairs) == len(set(comp.tolist())) == len(set(term.tolist()))


@pytest.mark.parametrize("mesh", _meshes(), ids=lambda m: m.name)
def test_lepp_length_recursion_and_paths(mesh):
    pin_lepp_recursion(mesh)


def pin_lepp_recursion(mesh, lib=None):
    """length(t) is 1 on a border longest edge, 2 on a terminal edge, else
    1 + length of the neighbour across the longest edge; every path steps
    across the previous triangle's longest edge and ends on the terminal."""
    r = oracle.run_mesh(mesh, lib=lib)
    T = mesh.n_triangles
    HI = 3 * T
    term, length = oracle.lepp(mesh, r.longest, lib=lib)
    le = checks.brute_force_longest(mesh)
    for t in range(T):
        e = 3 * t + int(le[t])
        tw = int(mesh.twin[e])
        if tw >= HI:
            assert length[t] == 1 and term[t] == e
            continue
        n = tw // 3
        if 3 * n + int(le[n]) == tw:
            assert length[t] == 2 and term[t] == min(e, tw)
        else:
            assert length[t] == 1 + length[n] and term[t] == term[n]
    for t in range(0, T, max(1, T // 25)):
        path = oracle.lepp_path(mesh, r.longest, t, lib=lib)
        assert len(path) == length[t] and path[0] == t
        for a, b in zip(path[:-1], path[1:]):
            e = 3 * a + int(le[a])
            assert int(mesh.twin[e]) // 3 == b


@pytest.mark.parametrize("s", [2, 5, 9])
def test_lepp_exact_grid_closed_form(s):
    pin_lepp_grid(s)


def pin_lepp_grid(s, lib=None):
    """Algorithm 15's grid: every cell's diagonal is the longest edge of both
    its triangles, so every Lepp is the cell's two triangles and ends on the
    diagonal."""
    m = meshgen.exact_grid(s)
    r = oracle.run_mesh(m, lib=lib)
    term, length = oracle.lepp(m, r.longest, lib=lib)
    assert np.all(length == 2)
    assert len(set(term.tolist())) == (s - 1) ** 2
    for t in range(m.n_triangles):
        e = int(term[t])
        a, b = m.coords[m.origin[e]], m.coords[m.origin[m.twin[e]]]
        assert abs(a[0] - b[0]) == 1 and abs(a[1] - b[1]) == 1   # a diagonal of a unit cell
