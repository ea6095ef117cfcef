"""Pins of the CPU oracle against things other than itself.

Each test ties the oracle to something the paper or plain mathematics fixes:
a hand-derived worked example (paper Fig. 3), the closed form of the
paper's grid (Algorithm 15, whose rows have no repair work in Table 1),
brute force from Definitions 1-3, geometric (atan2) ordering of the edges
around each barrier tip, output invariants, and relabelling symmetry.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen
from tests import checks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_meshes():
    out = [meshgen.two_triangle_square(), meshgen.exact_grid(6), meshgen.perturbed_grid(24, 0.3, seed=11)]
    for s in range(3):
        out.append(meshgen.random_delaunay(60 + 70 * s, seed=100 + s))
    for s in range(3):
        try:
            out.append(meshgen.lattice_delaunay(120, 14, seed=200 + s))
        except ValueError:
            pass
    return out


# ---------------------------------------------------------------- Fig. 3

def pin_two_triangle_square(lib=None):
    g = json.load(open(os.path.join(GOLDEN, "two_triangle_square.json")))
    m = meshgen.from_triangles(g["triangles"], g["coords"])
    r = oracle.run_mesh(m, lib=lib)
    HI = 3 * m.n_triangles
    le_local = [int(np.nonzero(r.longest[3 * t: 3 * t + 3])[0][0]) for t in range(m.n_triangles)]
    assert le_local == g["longest_local"]
    assert r.frontier0[:HI].tolist() == g["frontier_interior"]
    assert r.seed_list.tolist() == g["seed_list"]
    assert r.next_out[:HI].tolist() == g["next_out_interior"]
    assert r.prev_out[:HI].tolist() == g["prev_out_interior"]
    assert r.seeds.tolist() == g["seeds"]
    assert r.offsets.tolist() == g["offsets"]
    assert r.he_list.tolist() == g["he_list"]
    assert r.v_list.tolist() == g["v_list"]


def test_two_triangle_square_matches_hand_derivation():
    pin_two_triangle_square()


# ---------------------------------------------------------------- Algorithm 15 closed form

@pytest.mark.parametrize("s", [2, 3, 5, 8, 33])
def test_exact_grid_closed_form(s):
    pin_exact_grid(s)


def pin_exact_grid(s, lib=None):
    """Every cell of the paper's grid is one terminal-edge region: the
    diagonal (length sqrt 2 against legs of 1) is the longest edge of both
    triangles, so there are (s-1)^2 square polygons, N_F = 2T frontier
    half-edges and no barrier tip (Table 1 grid rows: Rep = 0)."""
    m = meshgen.exact_grid(s)
    r = oracle.run_mesh(m, lib=lib)
    T = m.n_triangles
    assert T == 2 * (s - 1) ** 2
    tri = m.triangles()
    # the longest half-edge of triangle t joins the cell corners k and k+s+1
    for t in range(T):
        e = 3 * t + int(np.nonzero(r.longest[3 * t: 3 * t + 3])[0][0])
        a, b = int(m.origin[e]), int(m.origin[int(m.twin[e])])
        assert abs(a - b) == s + 1
        assert min(a, b) in tri[t]
    assert r.n_polygons == (s - 1) ** 2
    assert r.stats["tips"] == 0
    assert r.stats["frontier1"] == 2 * T
    assert np.all(np.diff(r.offsets) == 4)
    # each polygon is the unit square of one cell, counter-clockwise
    ar = checks.polygon_areas(m.coords, r.v_list, r.offsets)
    assert np.allclose(ar, 1.0, rtol=0, atol=0)
    cells = sorted(tuple(sorted(r.v_list[r.offsets[p]: r.offsets[p + 1]].tolist())) for p in range(r.n_polygons))
    want = sorted((k, k + 1, k + s, k + s + 1) for k in range(s * s - s) if k % s != s - 1)
    assert cells == want


# ---------------------------------------------------------------- Definitions 1-3

@pytest.mark.parametrize("mesh", _small_meshes(), ids=lambda m: m.name)
def test_labels_match_lepp_brute_force(mesh):
    pin_labels(mesh)


def pin_labels(mesh, lib=None):
    """Longest edges from the triangles' own vertex lists; terminal-edge
    regions by chasing each triangle's Lepp (Definition 1-2); the frontier
    labels must cut the mesh exactly into those regions (Definition 3), and
    Algorithm 4 must give one seed per region, on its terminal edge."""
    r = oracle.run_mesh(mesh, lib=lib)
    T = mesh.n_triangles
    HI = 3 * T
    le_bf = checks.brute_force_longest(mesh)
    le_or = np.array([np.nonzero(r.longest[3 * t: 3 * t + 3])[0] for t in range(T)])
    assert le_or.shape == (T, 1), "not exactly one longest edge per triangle"
    assert np.array_equal(le_or[:, 0], le_bf)
    assert not np.any(r.longest[HI:]), "a border half-edge is labelled longest"
    term = checks.lepp_terminal(mesh, le_bf)
    comp = checks.components_over_nonfrontier(mesh, r.frontier0)
    # regions (by terminal edge) == components over non-frontier edges
    pairs = set(zip(comp.tolist(), term.tolist()))
    assert len(pairs) == len(set(comp.tolist())) == len(set(term.tolist()))
    # one seed per region, lying on that region's terminal edge
    seed_ids = sorted(min(int(s), int(mesh.twin[s])) for s in r.seed_list)
    assert seed_ids == sorted(set(term.tolist()))
    assert np.all(np.diff(r.seed_list) > 0)
    # frontier labels are symmetric and include every border edge
    assert np.array_equal(r.frontier0, r.frontier0[mesh.twin])
    assert np.all(r.frontier0[HI:] == 1)
    assert np.all(r.frontier0[mesh.twin[HI:]] == 1)


@pytest.mark.parametrize("mesh", _small_meshes(), ids=lambda m: m.name)
def test_every_vertex_has_a_frontier_edge(mesh):
    """Under the strict (length, edge id) order the shortest edge at a vertex
    is never a longest edge, so every vertex has a frontier edge and every
    rotation of the traversal ends."""
    r = oracle.run_mesh(mesh)
    deg = np.bincount(mesh.origin[r.frontier0.astype(bool)], minlength=mesh.n_vertices)
    assert np.all(deg >= 1)


# ---------------------------------------------------------------- Algorithm 6 geometry

def _meshes_with_tips():
    out = []
    for s in range(40):
        m = meshgen.random_delaunay(80, seed=1000 + s)
        r = oracle.run_mesh(m)
        if r.stats["tips"]:
            out.append(m)
        if len(out) >= 6:
            break
    return out


@pytest.mark.parametrize("mesh", _meshes_with_tips(), ids=lambda m: m.name)
def test_tips_and_middle_edges_from_geometry(mesh):
    pin_tips(mesh)


def pin_tips(mesh, lib=None):
    """Barrier tips are exactly the vertices with one incident frontier edge
    (counted from the F0 labels), and each chord is the edge found after
    floor((d-1)/2)+1 clockwise steps from that frontier edge, where the
    clockwise order comes from atan2 of the neighbour directions."""
    r = oracle.run_mesh(mesh, lib=lib)
    HI = 3 * mesh.n_triangles
    f0 = r.frontier0.astype(bool)
    deg_f = np.bincount(mesh.origin[f0], minlength=mesh.n_vertices)
    tip_vertices = set(np.nonzero(deg_f == 1)[0].tolist())
    assert set(mesh.origin[r.tip_out].tolist()) == tip_vertices
    assert len(r.tip_out) == len(tip_vertices)
    for f, m_ in zip(r.tip_out.tolist(), r.chord.tolist()):
        assert f0[f] and f < HI
        fan = checks.cw_fan(mesh, f)
        d = len(fan)
        assert d >= 3
        rr = (d - 1) // 2 + 1
        assert fan[rr] == m_
        assert not f0[m_] and r.frontier1[m_] and r.frontier1[mesh.twin[m_]]
    # F1 adds exactly the chord edges
    added = np.nonzero(r.frontier1.astype(bool) & ~f0)[0]
    want = set(r.chord.tolist()) | set(mesh.twin[r.chord].tolist())
    assert set(added.tolist()) == want


# ---------------------------------------------------------------- output invariants

def _invariant_meshes():
    out = _small_meshes()
    out += [meshgen.random_delaunay(2000, seed=1), meshgen.perturbed_grid(64, 0.3, seed=3)]
    out += [meshgen.random_delaunay(500, seed=300 + s) for s in range(4)]
    return out


@pytest.mark.parametrize("mesh", _invariant_meshes(), ids=lambda m: m.name)
def test_output_invariants(mesh):
    pin_invariants(mesh)


def pin_invariants(mesh, lib=None):
    r = oracle.run_mesh(mesh, lib=lib)
    assert r.stats["completion"] == 0
    checks.check_output_invariants(
        mesh, r.frontier1, r.next_out, r.prev_out, r.seeds, r.offsets, r.he_list, r.v_list,
        n_seeds_alg4=len(r.seed_list), n_distinct_chords=r.stats["distinct_chords"])
    if mesh.n_triangles <= 5000:
        checks.check_triangle_coverage(mesh, r.frontier1, r.he_list, r.offsets)


def test_paper_polygon_count_matches_canonical_list():
    """The traversal and repair phases produce as many polygons as the
    canonical cycle list holds (no cycle is produced twice or missed)."""
    for mesh in _invariant_meshes():
        r = oracle.run_mesh(mesh)
        assert r.stats["traversal_polygons"] + r.stats["repair_polygons"] == r.n_polygons


# ---------------------------------------------------------------- relabelling symmetry

def _vertex_cycles(mesh, r):
    out = set()
    for p in range(r.n_polygons):
        pts = [tuple(mesh.coords[v]) for v in r.v_list[r.offsets[p]: r.offsets[p + 1]]]
        i = min(range(len(pts)), key=lambda k: pts[k])
        out.add(tuple(pts[i:] + pts[:i]))
    return out


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_relabelling_keeps_polygons(seed):
    pin_relabelling(seed)


def pin_relabelling(seed, lib=None):
    """On a tie-free mesh, permuting vertex ids, triangle order and the
    starting corner of each triangle leaves the polygons (as cycles of
    points) unchanged: the output depends on numbering only through the
    canonical order."""
    m = meshgen.random_delaunay(400, seed=seed)
    r = oracle.run_mesh(m, lib=lib)
    rng = np.random.default_rng(seed)
    tri = m.triangles().astype(np.int64)
    perm_v = rng.permutation(m.n_vertices)
    inv = np.empty_like(perm_v)
    inv[perm_v] = np.arange(perm_v.shape[0])
    coords2 = m.coords[perm_v]
    tri2 = inv[tri]
    tri2 = tri2[rng.permutation(tri2.shape[0])]
    rot = rng.integers(0, 3, size=tri2.shape[0])
    tri2 = np.take_along_axis(tri2, (rot[:, None] + np.arange(3)[None, :]) % 3, axis=1)
    m2 = meshgen.from_triangles(tri2, coords2)
    r2 = oracle.run_mesh(m2, lib=lib)
    assert r2.n_polygons == r.n_polygons
    assert _vertex_cycles(m2, r2) == _vertex_cycles(m, r)


def test_tie_free_relabel_changes_only_order():
    """Seeds are the smallest half-edge of each polygon, so reversing the
    triangle order changes seeds and order but not the polygons."""
    m = meshgen.random_delaunay(300, seed=5)
    r = oracle.run_mesh(m)
    tri = m.triangles()[::-1].copy()
    m2 = meshgen.from_triangles(tri, m.coords)
    r2 = oracle.run_mesh(m2)
    assert _vertex_cycles(m2, r2) == _vertex_cycles(m, r)
