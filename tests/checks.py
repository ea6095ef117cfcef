"""Independent checks of a Polylla result (used to pin the oracle and to
check GPU output at sizes the oracle is not run on).

Nothing here calls the oracle or the library: every function takes plain
arrays and checks a property that the paper's definitions or plain geometry
fix (Definitions 1-3, the traversal of Section 5.2, the repair of Section
5.3), computed by a different route than the method itself.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------
# brute force from the definitions (tiny meshes; Python loops)
# --------------------------------------------------------------------------

def sq_len_py(coords, a, b) -> float:
    """Squared edge length with Python floats: IEEE binary64, each
    operation rounded (CPython never contracts to FMA)."""
    ax, ay = float(coords[a, 0]), float(coords[a, 1])
    bx, by = float(coords[b, 0]), float(coords[b, 1])
    dx = bx - ax
    dy = by - ay
    return dx * dx + dy * dy


def brute_force_longest(mesh) -> np.ndarray:
    """Per triangle, the local index k (0..2) of its longest edge, computed
    from the triangle's vertex list (not from half-edge queries); equal
    lengths go to the smaller edge id min(e, twin e)."""
    T = mesh.n_triangles
    tri = mesh.origin[: 3 * T].reshape(-1, 3)
    out = np.empty(T, np.int8)
    for t in range(T):
        best = None
        for k in range(3):
            e = 3 * t + k
            d = sq_len_py(mesh.coords, tri[t, k], tri[t, (k + 1) % 3])
            key = (d, -min(e, int(mesh.twin[e])))
            if best is None or key > best[0]:
                best = (key, k)
        out[t] = best[1]
    return out


def lepp_terminal(mesh, le_local: np.ndarray) -> np.ndarray:
    """Definition 1 by pointer chasing: for every triangle, follow the
    neighbour across the longest edge until the edge is terminal (the
    neighbour has the same longest edge) or on the border.  Returns, per
    triangle, the id min(e, twin e) of its terminal edge (Definition 2
    groups triangles by this id)."""
    T = mesh.n_triangles
    HI = 3 * T
    out = np.empty(T, np.int64)
    for t0 in range(T):
        t = t0
        for _ in range(T + 1):
            e = 3 * t + int(le_local[t])
            tw = int(mesh.twin[e])
            if tw >= HI:
                out[t0] = e
                break
            n = tw // 3
            if 3 * n + int(le_local[n]) == tw:
                out[t0] = min(e, tw)
                break
            t = n
        else:
            raise AssertionError("Lepp does not terminate")
    return out


def components_over_nonfrontier(mesh, frontier: np.ndarray) -> np.ndarray:
    """Connected components of triangles joined across non-frontier interior
    edges (flood fill).  Returns a component id per triangle."""
    T = mesh.n_triangles
    HI = 3 * T
    comp = np.full(T, -1, np.int64)
    c = 0
    for s in range(T):
        if comp[s] >= 0:
            continue
        stack = [s]
        comp[s] = c
        while stack:
            t = stack.pop()
            for k in range(3):
                e = 3 * t + k
                if frontier[e]:
                    continue
                tw = int(mesh.twin[e])
                if tw >= HI:
                    continue
                n = tw // 3
                if comp[n] < 0:
                    comp[n] = c
                    stack.append(n)
        c += 1
    return comp


def cw_fan(mesh, f: int) -> list:
    """Outgoing interior half-edges around origin(f), in clockwise angular
    order starting at f, from coordinates (atan2), not from rotation
    queries.  Valid for interior vertices."""
    HI = 3 * mesh.n_triangles
    v = int(mesh.origin[f])
    outs = [e for e in np.nonzero(mesh.origin[:HI] == v)[0]]
    def ang(e):
        w = int(mesh.origin[int(mesh.twin[e])]) if int(mesh.twin[e]) < len(mesh.origin) else None
        tx, ty = mesh.coords[w]
        return math.atan2(ty - mesh.coords[v, 1], tx - mesh.coords[v, 0])
    a0 = ang(f)
    # clockwise = decreasing angle, measured from f
    rel = sorted(outs, key=lambda e: ((a0 - ang(e)) % (2 * math.pi)))
    assert rel[0] == f
    return [int(e) for e in rel]


# --------------------------------------------------------------------------
# invariants of the output (any size; numpy)
# --------------------------------------------------------------------------

def polygon_areas(coords, v_list, offsets) -> np.ndarray:
    """Shoelace area of every polygon."""
    P = offsets.shape[0] - 1
    if P == 0:
        return np.zeros(0)
    lens = np.diff(offsets)
    pid = np.repeat(np.arange(P), lens)
    nxt_pos = np.arange(v_list.shape[0]) + 1
    last = offsets[1:] - 1
    nxt_pos[last] = offsets[:-1]
    a = coords[v_list]
    b = coords[v_list[nxt_pos]]
    cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    return 0.5 * np.bincount(pid, weights=cross, minlength=P)


def triangle_area_sum(mesh) -> float:
    t = mesh.triangles()
    a, b, c = mesh.coords[t[:, 0]], mesh.coords[t[:, 1]], mesh.coords[t[:, 2]]
    return float(0.5 * np.sum((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])))


def check_output_invariants(mesh, frontier1, next_out, prev_out, seeds, offsets, he_list, v_list,
                            n_seeds_alg4=None, n_distinct_chords=None, check_area=True,
                            check_euler=True) -> dict:
    """Assert the invariants of a Polylla polygon mesh; return some counts.

    * next_out is a permutation of the F1 frontier interior half-edges and
      prev_out its inverse; every other half-edge keeps its input links;
    * no half-edge is followed by its own twin (no barrier tip is left);
    * the CSR lists every frontier interior half-edge exactly once, each
      polygon from its smallest half-edge, polygons ascending, following
      next_out, with v_list = origin(he_list);
    * P = #seeds of Algorithm 4 + #distinct chords (each chord splits one
      polygon in two), when those counts are given;
    * Euler for the planar frontier graph: V - E_F + P = 1;
    * every polygon has positive area and the areas sum to the domain area.
    """
    T = mesh.n_triangles
    HI = 3 * T
    H = mesh.n_halfedges
    f1 = np.asarray(frontier1[:HI]).astype(bool)
    fr = np.nonzero(f1)[0]
    NF = fr.shape[0]
    # links
    nx = next_out[fr]
    assert np.all(nx >= 0) and np.all(nx < HI), "next_out leaves the interior half-edges"
    assert np.all(f1[nx]), "next_out reaches a non-frontier half-edge"
    assert np.unique(nx).shape[0] == NF, "next_out is not a permutation of the frontier half-edges"
    assert np.all(prev_out[nx] == fr), "prev_out is not the inverse of next_out"
    keep = np.ones(H, bool)
    keep[fr] = False
    assert np.all(next_out[keep] == mesh.next[keep]), "non-frontier next changed"
    assert np.all(prev_out[keep] == mesh.prev[keep]), "non-frontier prev changed"
    assert not np.any(nx == mesh.twin[fr]), "a barrier tip is left"
    # CSR
    P = seeds.shape[0]
    assert offsets.shape[0] == P + 1 and offsets[0] == 0 and offsets[-1] == NF
    assert he_list.shape[0] == NF and v_list.shape[0] == NF
    assert np.array_equal(np.sort(he_list), fr), "CSR does not list each frontier half-edge once"
    lens = np.diff(offsets)
    assert np.all(lens >= 3), "polygon with fewer than 3 sides"
    assert np.all(np.diff(seeds) > 0), "seeds not ascending"
    assert np.array_equal(he_list[offsets[:-1]], seeds), "polygon does not start at its seed"
    pid = np.repeat(np.arange(P), lens)
    assert np.all(he_list >= seeds[pid]), "seed is not the smallest half-edge of its polygon"
    nxt_pos = np.arange(NF) + 1
    nxt_pos[offsets[1:] - 1] = offsets[:-1]
    assert np.array_equal(next_out[he_list], he_list[nxt_pos]), "CSR order does not follow next_out"
    assert np.array_equal(v_list, mesh.origin[he_list]), "v_list != origin(he_list)"
    out = {"P": P, "NF": NF}
    if n_seeds_alg4 is not None and n_distinct_chords is not None:
        assert P == n_seeds_alg4 + n_distinct_chords, "P != regions + distinct chords"
    if check_euler:
        border_edges = H - HI
        E = (NF - border_edges) // 2 + border_edges   # interior frontier edges + border edges
        assert (NF - border_edges) % 2 == 0
        V = mesh.n_vertices
        out["euler"] = V - E + P
        assert V - E + P == 1, f"Euler V-E+P = {V - E + P} != 1"
    if check_area:
        ar = polygon_areas(mesh.coords, v_list, offsets)
        assert np.all(ar > 0), "polygon with non-positive area"
        tot = triangle_area_sum(mesh)
        assert abs(ar.sum() - tot) <= 1e-12 * max(1.0, abs(tot)) * max(1.0, math.log2(max(P, 2))), \
            f"area {ar.sum()} != {tot}"
    return out


def check_triangle_coverage(mesh, frontier1, he_list, offsets):
    """Every triangle lies in exactly one polygon: the components of
    triangles over non-F1 edges match the polygons one to one, and each
    polygon's half-edges bound exactly one component."""
    T = mesh.n_triangles
    comp = components_over_nonfrontier(mesh, frontier1)
    P = offsets.shape[0] - 1
    lens = np.diff(offsets)
    pid = np.repeat(np.arange(P), lens)
    tri_comp = comp[he_list // 3]
    # all half-edges of one polygon see one component
    first = tri_comp[offsets[:-1]]
    assert np.all(tri_comp == first[pid]), "a polygon touches two triangle components"
    # one polygon per component, and every component has one
    assert np.unique(first).shape[0] == P, "two polygons share a component"
    assert comp.max() + 1 == P, "a component has no polygon"
    return comp
