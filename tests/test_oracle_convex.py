"""Pins of the oracle's convexification (post-processing of the Polylla mesh).

Section 4.2 of the paper keeps every half-edge of the triangulation so that
a later step can turn non-convex polygons into convex ones; it gives no
method, so the oracle follows reading R9 (chords at reflex corners, fewest
per corner, taken from the triangulation's own edges).  The pins check what
geometry and the reading fix, independently of the oracle's code:

* convexity, exactly: every corner of every output polygon turns by at
  most a half turn, in rational arithmetic on the float coordinates;
* chords are interior edges of the triangulation that were not frontier
  edges, both halves join the frontier, and nothing else changes there;
* the result is a planar subdivision of the domain: next/prev a
  permutation on the new frontier, canonical CSR, Euler V - E + P = 1,
  polygon areas summing to the domain's area, P2 = P1 + distinct chords,
  every triangle in exactly one polygon, every new polygon inside one
  Polylla polygon;
* fewest chords: at every reflex corner the number of chords equals the
  minimum over all subsets of the corner's interior edges (brute force over
  the fan ordered by angle, exact turn tests);
* a fixed point: convexifying a convex mesh adds no chord; exact grids
  (unit squares) get none.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen
from tests.checks import check_output_invariants, check_triangle_coverage, components_over_nonfrontier


def _exact_cross(coords, v, a, b) -> Fraction:
    """cross(a - v, b - v) for vertex ids, exactly."""
    vx, vy = Fraction(float(coords[v, 0])), Fraction(float(coords[v, 1]))
    ax, ay = Fraction(float(coords[a, 0])) - vx, Fraction(float(coords[a, 1])) - vy
    bx, by = Fraction(float(coords[b, 0])) - vx, Fraction(float(coords[b, 1])) - vy
    return ax * by - ay * bx


def _target(mesh, h) -> int:
    return int(mesh.origin[int(mesh.twin[h])])


def _corner_fan(mesh, e, x):
    """Interior half-edges leaving v = target(e) strictly inside the corner
    (twin(e) .. x clockwise), ordered by angle from the coordinates."""
    HI = 3 * mesh.n_triangles
    v = _target(mesh, e)
    vx, vy = mesh.coords[v]

    def ang(w):
        return math.atan2(mesh.coords[w, 1] - vy, mesh.coords[w, 0] - vx)

    a0 = ang(int(mesh.origin[e]))                 # direction of twin(e)
    cw = lambda w: (a0 - ang(w)) % (2 * math.pi)  # clockwise sweep from twin(e)
    ax = cw(_target(mesh, x))
    outs = [int(h) for h in np.nonzero(mesh.origin[:HI] == v)[0]]
    inside = [h for h in outs if 0 < cw(_target(mesh, h)) < ax]
    return v, sorted(inside, key=lambda h: cw(_target(mesh, h)))


def _min_chords(mesh, e, x) -> tuple[int, list]:
    """Fewest interior edges of the corner (e, x) that leave every part of
    it within a half turn (brute force over subsets, exact turn tests)."""
    v, fan = _corner_fan(mesh, e, x)
    ends = [int(mesh.origin[e])] + [_target(mesh, h) for h in fan] + [_target(mesh, x)]
    for k in range(len(fan) + 1):
        for sub in itertools.combinations(range(1, len(fan) + 1), k):
            pts = [ends[0]] + [ends[i] for i in sub] + [ends[-1]]
            if all(_exact_cross(mesh.coords, v, pts[i], pts[i + 1]) <= 0 for i in range(len(pts) - 1)):
                return k, fan
    raise AssertionError("no subset of the fan makes the corner convex")


def _distinct_edges(mesh, hs) -> int:
    return len({min(int(h), int(mesh.twin[h])) for h in hs})


def pin_convex(mesh, lib=None, minimal=True):
    base = oracle.run_mesh(mesh, lib=lib)
    c = oracle.convexify(mesh, base, lib=lib)
    T = mesh.n_triangles
    HI = 3 * T
    f1 = base.frontier1[:HI].astype(bool)
    f2 = c.frontier2[:HI].astype(bool)
    assert np.all(f2[f1]), "a frontier edge of the Polylla mesh was dropped"
    ch = c.chords
    assert np.all(ch < HI) and np.all(mesh.twin[ch] < HI), "a chord is not an interior edge"
    assert not np.any(f1[ch]), "a chord was a frontier edge already"
    halves = set(ch.tolist()) | set(mesh.twin[ch].tolist())
    assert set(np.nonzero(f2 & ~f1)[0].tolist()) == halves, "new frontier half-edges are not the chord halves"
    check_output_invariants(mesh, c.frontier2, c.next_out, c.prev_out, c.seeds, c.offsets, c.he_list, c.v_list,
                            n_seeds_alg4=base.n_polygons, n_distinct_chords=_distinct_edges(mesh, ch))
    comp2 = check_triangle_coverage(mesh, c.frontier2, c.he_list, c.offsets)
    comp1 = components_over_nonfrontier(mesh, base.frontier1)
    parent = {}
    for t in range(T):
        assert parent.setdefault(int(comp2[t]), int(comp1[t])) == int(comp1[t]), \
            "a convex polygon straddles two Polylla polygons"
    # exact convexity of every corner
    for p in range(c.n_polygons):
        hs = c.he_list[c.offsets[p]:c.offsets[p + 1]]
        for i, h in enumerate(hs):
            x = int(hs[(i + 1) % len(hs)])
            v = _target(mesh, int(h))
            assert _exact_cross(mesh.coords, v, int(mesh.origin[h]), _target(mesh, x)) <= 0, \
                f"reflex corner left at half-edge {int(h)}"
    # fewest chords at every reflex corner of the Polylla mesh
    if minimal:
        chosen = set(ch.tolist())
        for e in np.nonzero(f1)[0]:
            e = int(e)
            x = int(base.next_out[e])
            if _exact_cross(mesh.coords, _target(mesh, e), int(mesh.origin[e]), _target(mesh, x)) <= 0:
                continue
            k, fan = _min_chords(mesh, e, x)
            got = sum(1 for h in fan if h in chosen)
            assert got == k, f"corner at half-edge {e}: {got} chords, fewest is {k}"
    return base, c


def pin_fixed_point(mesh, lib=None):
    base = oracle.run_mesh(mesh, lib=lib)
    c = oracle.convexify(mesh, base, lib=lib)
    again = oracle.convexify(mesh, SimpleNamespace(frontier1=c.frontier2, next_out=c.next_out), lib=lib)
    assert again.chords.shape[0] == 0 and again.stats["reflex_corners"] == 0, "a convex mesh got chords"
    assert np.array_equal(again.he_list, c.he_list) and np.array_equal(again.seeds, c.seeds)


def pin_exact_grid(s: int, lib=None):
    mesh = meshgen.exact_grid(s)
    base = oracle.run_mesh(mesh, lib=lib)
    c = oracle.convexify(mesh, base, lib=lib)
    assert c.chords.shape[0] == 0 and c.n_polygons == (s - 1) ** 2
    assert np.array_equal(c.he_list, base.he_list)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_convex_pins_random_delaunay(seed):
    _, c = pin_convex(meshgen.random_delaunay(300, seed=400 + seed))
    assert c.stats["distinct_chords"] > 0


def test_convex_pins_perturbed_grid():
    _, c = pin_convex(meshgen.perturbed_grid(24, 0.3, seed=401))
    assert c.stats["distinct_chords"] > 0


def test_convex_pins_lattice_ties():
    for s in range(3):
        try:
            mesh = meshgen.lattice_delaunay(150, 16, seed=410 + s)
        except ValueError:
            continue
        pin_convex(mesh)
        return
    pytest.skip("no lattice mesh generated")


def test_convex_pins_larger_mesh_without_brute_force():
    pin_convex(meshgen.random_delaunay(3000, seed=420), minimal=False)


def test_convex_fixed_point_and_grid():
    pin_fixed_point(meshgen.random_delaunay(500, seed=430))
    pin_exact_grid(6)
