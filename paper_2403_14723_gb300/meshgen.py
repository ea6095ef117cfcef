"""Seeded synthetic triangulations in the half-edge layout the library consumes.

This module builds inputs only.  It holds none of the Polylla arithmetic
(no edge lengths, no labels, no rotations): it places points, triangulates
them, and lays the result out as half-edges.  Both the CUDA path and the
CPU oracle are fed from here, so the two never depend on each other for
their inputs.

Half-edge layout (one mesh, ``T`` triangles, ``H`` half-edges):

* interior half-edges ``[0, 3T)``: triangle ``t`` owns ``3t, 3t+1, 3t+2``,
  listed counter-clockwise; half-edge ``3t+k`` runs from vertex
  ``tri[t, k]`` to ``tri[t, (k+1) % 3]``.  Its ``next`` is
  ``3t + (k+1) % 3`` and its ``prev`` is ``3t + (k+2) % 3`` (the implicit
  face indexing of the paper's Section 4.2: "each three half-edges
  represent a face").
* border half-edges ``[3T, H)``: one per boundary edge, twin of the
  interior half-edge on that edge, running the other way; their
  ``next``/``prev`` walk the exterior face.
* ``coords`` is ``[V, 2]`` float64, interleaved ``x, y``.

Workloads (the synthetic stand-ins for the paper's datasets, Section 6.1):

* :func:`exact_grid` -- the paper's grid generator (Algorithm 15).
* :func:`perturbed_grid` -- a jittered ``s x s`` vertex grid on the unit
  square with a random diagonal per cell.
* :func:`random_delaunay` -- Delaunay triangulation of uniform random points
  in the unit square (the paper uses the Triangle program; here scipy's
  Qhull builds it, since Triangle is not available).
* :func:`lattice_delaunay` -- Delaunay triangulation of random points on a
  small integer lattice; integer coordinates make many squared edge lengths
  exactly equal, which exercises the longest-edge tie-break.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class HalfEdgeMesh:
    """A triangulation in the library's SoA half-edge layout (host arrays)."""

    coords: np.ndarray   # [V, 2] float64
    origin: np.ndarray   # [H] int32
    twin: np.ndarray     # [H] int32
    next: np.ndarray     # [H] int32
    prev: np.ndarray     # [H] int32
    n_triangles: int
    name: str = ""

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_halfedges(self) -> int:
        return int(self.origin.shape[0])

    @property
    def n_border(self) -> int:
        return self.n_halfedges - 3 * self.n_triangles

    def triangles(self) -> np.ndarray:
        """``[T, 3]`` vertex ids of each triangle (counter-clockwise)."""
        return self.origin[: 3 * self.n_triangles].reshape(-1, 3)


# --------------------------------------------------------------------------
# half-edge construction
# --------------------------------------------------------------------------

def _orient(coords: np.ndarray, tris: np.ndarray) -> np.ndarray:
    a = coords[tris[:, 0]]
    b = coords[tris[:, 1]]
    c = coords[tris[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def build_halfedges(tris: np.ndarray, coords: np.ndarray, name: str = "",
                    edge_ids: np.ndarray | None = None, n_edge_ids: int = 0) -> HalfEdgeMesh:
    """Lay out counter-clockwise triangles ``tris`` ([T, 3]) as half-edges.

    Twins are found by matching each directed edge ``(a, b)`` with ``(b, a)``.
    ``edge_ids`` (optional, one non-negative id per interior half-edge, equal
    for the two halves of an edge and below ``n_edge_ids``) lets a caller
    with a closed-form edge numbering skip the sort.  Boundary edges get a
    border half-edge appended at ``[3T, H)``.
    """
    tris = np.ascontiguousarray(tris, dtype=np.int64)
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    T = tris.shape[0]
    V = coords.shape[0]
    if T == 0:
        raise ValueError("a mesh needs at least one triangle")
    if tris.min() < 0 or tris.max() >= V:
        raise ValueError("triangle vertex out of range")
    if not np.all(_orient(coords, tris) > 0):
        raise ValueError("triangles must be counter-clockwise with positive area")
    HI = 3 * T
    org = tris.reshape(-1)
    dst = np.roll(tris, -1, axis=1).reshape(-1)
    twin_i = np.full(HI, -1, dtype=np.int64)
    if edge_ids is None:
        key = org * V + dst
        rkey = dst * V + org
        order = np.argsort(key, kind="stable")
        skey = key[order]
        if np.any(skey[1:] == skey[:-1]):
            raise ValueError("non-manifold input: a directed edge appears twice")
        pos = np.searchsorted(skey, rkey)
        posc = np.minimum(pos, HI - 1)
        found = skey[posc] == rkey
        twin_i[found] = order[posc[found]]
    else:
        eid = np.asarray(edge_ids, dtype=np.int64)
        lo = org < dst
        slot_lo = np.full(n_edge_ids, -1, dtype=np.int64)
        slot_hi = np.full(n_edge_ids, -1, dtype=np.int64)
        idx = np.arange(HI, dtype=np.int64)
        slot_lo[eid[lo]] = idx[lo]
        slot_hi[eid[~lo]] = idx[~lo]
        twin_i = np.where(lo, slot_hi[eid], slot_lo[eid])
    border_src = np.nonzero(twin_i < 0)[0]           # interior halves on the boundary
    NB = border_src.shape[0]
    H = HI + NB
    origin = np.empty(H, dtype=np.int64)
    twin = np.empty(H, dtype=np.int64)
    nxt = np.empty(H, dtype=np.int64)
    prv = np.empty(H, dtype=np.int64)
    origin[:HI] = org
    twin[:HI] = twin_i
    bid = HI + np.arange(NB, dtype=np.int64)
    twin[border_src] = bid
    twin[bid] = border_src
    origin[bid] = dst[border_src]                    # border half runs the other way
    t3 = (np.arange(HI, dtype=np.int64) // 3) * 3
    k = np.arange(HI, dtype=np.int64) % 3
    nxt[:HI] = t3 + (k + 1) % 3
    prv[:HI] = t3 + (k + 2) % 3
    if NB:
        out_border = np.full(V, -1, dtype=np.int64)
        borg = origin[bid]
        if np.unique(borg).shape[0] != NB:
            raise ValueError("boundary is not a simple closed curve (vertex with two border edges)")
        out_border[borg] = bid
        bdst = org[border_src]                       # target of a border half = origin of its twin
        nb = out_border[bdst]
        if np.any(nb < 0):
            raise ValueError("open boundary")
        nxt[bid] = nb
        prv[nb] = bid
    m = HalfEdgeMesh(
        coords=coords,
        origin=origin.astype(np.int32),
        twin=twin.astype(np.int32),
        next=nxt.astype(np.int32),
        prev=prv.astype(np.int32),
        n_triangles=T,
        name=name,
    )
    return m


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------

def exact_grid(s: int) -> HalfEdgeMesh:
    """The paper's grid (Algorithm 15) with ``s x s`` vertices.

    Vertex ``k = i*s + j`` has integer coordinates ``(i, j)``; the
    algorithm lists each cell's faces as ``(k, k+1, k+s+1)`` and
    ``(k, k+s+1, k+s)`` for ``k < s*s - s`` with ``k mod s != s-1``.
    Those lists are clockwise when ``(i, j)`` is read as ``(x, y)``, so the
    vertex is placed at ``x = j, y = i``, which makes the same lists
    counter-clockwise.  Every triangle is a right isosceles triangle with the
    cell diagonal as its unique longest edge.
    """
    if s < 2:
        raise ValueError("grid needs s >= 2")
    k = np.arange(s * s, dtype=np.int64)
    coords = np.stack([(k % s).astype(np.float64), (k // s).astype(np.float64)], axis=1)
    cells = np.arange(s * s - s, dtype=np.int64)
    cells = cells[cells % s != s - 1]
    tris = np.empty((2 * cells.shape[0], 3), dtype=np.int64)
    tris[0::2] = np.stack([cells, cells + 1, cells + s + 1], axis=1)
    tris[1::2] = np.stack([cells, cells + s + 1, cells + s], axis=1)
    return _grid_mesh(tris, coords, s, f"exact_grid_{s}")


def _grid_edge_ids(tris: np.ndarray, s: int) -> tuple[np.ndarray, int]:
    org = tris.reshape(-1)
    dst = np.roll(tris, -1, axis=1).reshape(-1)
    a = np.minimum(org, dst)
    d = np.maximum(org, dst) - a
    typ = np.select([d == 1, d == s, d == s + 1, d == s - 1], [0, 1, 2, 3], default=-1)
    if np.any(typ < 0):
        raise ValueError("not a grid edge")
    return a * 4 + typ, 4 * s * s


def _grid_mesh(tris: np.ndarray, coords: np.ndarray, s: int, name: str) -> HalfEdgeMesh:
    eid, n = _grid_edge_ids(tris, s)
    return build_halfedges(tris, coords, name=name, edge_ids=eid, n_edge_ids=n)


def perturbed_grid(s: int, jitter: float = 0.3, seed: int = 3) -> HalfEdgeMesh:
    """Jittered ``s x s`` vertex grid on the unit square.

    Vertex ``(i, j)`` (row ``i``, column ``j``, id ``i*s + j``) sits at
    ``(j*h, i*h)`` with ``h = 1/(s-1)``; every interior vertex is moved in x
    and in y independently by ``U[-jitter*h, +jitter*h]``; boundary vertices
    stay put, so the domain is exactly the unit square.  Each cell is cut
    along a diagonal picked by a fair coin.  If the picked diagonal would
    leave a triangle without positive area (possible at the extremes of the
    jitter), the cell takes the other diagonal, which is then always valid
    because the jittered cell is a simple quadrilateral.  Triangles are
    numbered cell by cell, row-major, two per cell.
    """
    if s < 2:
        raise ValueError("grid needs s >= 2")
    rng = np.random.default_rng(seed)
    h = 1.0 / (s - 1)
    k = np.arange(s * s, dtype=np.int64)
    i = k // s
    j = k % s
    x = j.astype(np.float64) * h
    y = i.astype(np.float64) * h
    x[j == s - 1] = 1.0
    y[i == s - 1] = 1.0
    jx = rng.uniform(-jitter * h, jitter * h, size=s * s)
    jy = rng.uniform(-jitter * h, jitter * h, size=s * s)
    interior = (i > 0) & (i < s - 1) & (j > 0) & (j < s - 1)
    x = np.where(interior, x + jx, x)
    y = np.where(interior, y + jy, y)
    coords = np.stack([x, y], axis=1)
    ci, cj = np.meshgrid(np.arange(s - 1, dtype=np.int64), np.arange(s - 1, dtype=np.int64), indexing="ij")
    c = (ci * s + cj).reshape(-1)
    coin = rng.integers(0, 2, size=c.shape[0]).astype(bool)
    # diagonal A: c -- c+s+1 ; diagonal B: c+1 -- c+s
    tA0 = np.stack([c, c + 1, c + s + 1], axis=1)
    tA1 = np.stack([c, c + s + 1, c + s], axis=1)
    tB0 = np.stack([c, c + 1, c + s], axis=1)
    tB1 = np.stack([c + 1, c + s + 1, c + s], axis=1)
    okA = (_orient(coords, tA0) > 0) & (_orient(coords, tA1) > 0)
    okB = (_orient(coords, tB0) > 0) & (_orient(coords, tB1) > 0)
    useA = np.where(coin, okA, ~okB)
    if not np.all(np.where(useA, okA, okB)):
        raise RuntimeError("jittered cell with no valid diagonal")
    tris = np.empty((2 * c.shape[0], 3), dtype=np.int64)
    tris[0::2] = np.where(useA[:, None], tA0, tB0)
    tris[1::2] = np.where(useA[:, None], tA1, tB1)
    return _grid_mesh(tris, coords, s, f"perturbed_grid_{s}")


# --------------------------------------------------------------------------
# Delaunay meshes
# --------------------------------------------------------------------------

def _hilbert_index(xy: np.ndarray, bits: int = 16) -> np.ndarray:
    """Hilbert curve index of points in ``[0, 1]^2`` quantised to ``2**bits``."""
    n = 1 << bits
    q = np.clip((xy * n).astype(np.int64), 0, n - 1)
    x = q[:, 0].copy()
    y = q[:, 1].copy()
    d = np.zeros(x.shape[0], dtype=np.int64)
    sft = n >> 1
    while sft > 0:
        rx = (x & sft) > 0
        ry = (y & sft) > 0
        d += sft * sft * ((3 * rx.astype(np.int64)) ^ ry.astype(np.int64))
        # rotate the quadrant
        flip = ~ry
        swap_x = flip & rx
        x = np.where(swap_x, n - 1 - x, x)
        y = np.where(swap_x, n - 1 - y, y)
        x2 = np.where(flip, y, x)
        y2 = np.where(flip, x, y)
        x, y = x2, y2
        sft >>= 1
    return d


def _delaunay(points: np.ndarray) -> np.ndarray:
    from scipy.spatial import Delaunay  # generator-only dependency

    return np.asarray(Delaunay(points).simplices, dtype=np.int64)


def _canonical_order(tris: np.ndarray, coords: np.ndarray) -> np.ndarray:
    """Orient every triangle CCW, start it at its smallest vertex id and sort
    the triangles lexicographically, so the layout does not depend on the
    triangulator's internal order."""
    tris = tris.copy()
    neg = _orient(coords, tris) < 0
    tris[neg] = tris[neg][:, ::-1]
    r = np.argmin(tris, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    tris = np.take_along_axis(tris, idx, axis=1)
    order = np.lexsort((tris[:, 2], tris[:, 1], tris[:, 0]))
    return tris[order]


def _drop_flat(tris: np.ndarray, coords: np.ndarray) -> np.ndarray:
    return tris[_orient(coords, tris) != 0]


def random_delaunay(n_points: int, seed: int) -> HalfEdgeMesh:
    """Delaunay triangulation of ``n_points`` uniform points in ``[0, 1)^2``.

    Points come from ``numpy.random.default_rng(seed).random((n, 2))`` and are
    numbered along a Hilbert curve (a mesh generator's spatially coherent
    vertex order); triangles are canonicalised by :func:`_canonical_order`.
    The boundary is the convex hull.
    """
    rng = np.random.default_rng(seed)
    pts = rng.random((n_points, 2))
    pts = pts[np.argsort(_hilbert_index(pts), kind="stable")]
    tris = _drop_flat(_delaunay(pts), pts)
    tris = _canonical_order(tris, pts)
    return build_halfedges(tris, pts, name=f"random_delaunay_{n_points}_s{seed}")


def lattice_delaunay(n_points: int, side: int, seed: int) -> HalfEdgeMesh:
    """Delaunay triangulation of ``n_points`` distinct random points of the
    integer lattice ``[0, side)^2`` (float64 coordinates holding integers).

    Many edges have exactly equal squared lengths, so the longest-edge
    tie-break decides the labels.  Qhull may return zero-area triangles for
    collinear lattice points on the hull; those are dropped and the seed is
    rejected (``ValueError``) if the remainder is not a valid triangulation.
    """
    rng = np.random.default_rng(seed)
    if n_points > side * side:
        raise ValueError("more points than lattice sites")
    flat = rng.choice(side * side, size=n_points, replace=False)
    pts = np.stack([(flat % side).astype(np.float64), (flat // side).astype(np.float64)], axis=1)
    tris = _drop_flat(_delaunay(pts), pts)
    used = np.unique(tris)
    remap = np.full(n_points, -1, dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    pts = pts[used]
    tris = remap[tris]
    tris = _canonical_order(tris, pts)
    return build_halfedges(tris, pts, name=f"lattice_delaunay_{n_points}_{side}_s{seed}")


def near_tie_delaunay(n_points: int, side: int, seed: int, ulps: int = 4) -> HalfEdgeMesh:
    """Lattice Delaunay mesh (see :func:`lattice_delaunay`) whose coordinates
    are then moved by a few units in the last place and scaled into
    ``[0, 1)``: squared edge lengths that were equal now differ only in
    their last bits, so a float32 screen of the longest edge cannot decide
    them and the exact float64 comparison must."""
    m = lattice_delaunay(n_points, side, seed)
    rng = np.random.default_rng(seed + 7)
    xy = m.coords / float(side) + 0.25
    bits = xy.view(np.int64) + rng.integers(-ulps, ulps + 1, size=xy.shape)
    xy = bits.view(np.float64)
    tri = m.triangles()
    if not np.all(_orient(xy, tri) > 0):
        raise ValueError("perturbation flipped a triangle")
    return build_halfedges(tri, xy, name=f"near_tie_delaunay_{n_points}_{side}_s{seed}")


def two_triangle_square() -> HalfEdgeMesh:
    """The two triangles of a unit square cut by a diagonal (paper Fig. 3):
    the diagonal is the shared longest edge, so the result is one 4-gon."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]])
    return build_halfedges(tris, coords, name="two_triangle_square")


def from_triangles(tris, coords, name: str = "") -> HalfEdgeMesh:
    """Build a mesh from explicit CCW triangles (used by hand-made fixtures)."""
    return build_halfedges(np.asarray(tris), np.asarray(coords, dtype=np.float64), name=name)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    # 2,000 uniform random points, Delaunay, convex-hull boundary
    "delaunay_2k": lambda: random_delaunay(2000, seed=1),
    # 1,000,000 uniform random points, Delaunay
    "delaunay_1m": lambda: random_delaunay(1_000_000, seed=2),
    # 4096 x 4096 perturbed grid, jitter +-0.3 cell, random diagonals
    "pgrid_4096": lambda: perturbed_grid(4096, 0.3, seed=3),
}


def batch_sizes(n_meshes: int, t_min: int, t_max: int, seed: int) -> np.ndarray:
    """Target triangle counts, log-uniform in ``[t_min, t_max]``."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(t_min), np.log(t_max), size=n_meshes)).round().astype(np.int64)


def batch_member(i: int, t_target: int, seed: int) -> HalfEdgeMesh:
    """Mesh ``i`` of a batch: even ``i`` Delaunay of uniform random points
    (about ``t_target / 2`` points), odd ``i`` a perturbed grid (jitter 0.3,
    about ``sqrt(t_target / 2) + 1`` vertices a side); seed ``seed + i``."""
    if i % 2 == 0:
        return random_delaunay(max(4, int(round(t_target / 2)) + 1), seed=seed + i)
    s = max(2, int(round(np.sqrt(t_target / 2.0))) + 1)
    return perturbed_grid(s, 0.3, seed=seed + i)


def _batch_member_args(args):
    return batch_member(*args)


def random_batch(n_meshes: int = 4096, t_min: int = 100, t_max: int = 200_000, seed: int = 4,
                 workers: int = 0) -> list[HalfEdgeMesh]:
    """A batch of independent triangulations: sizes log-uniform in
    ``[t_min, t_max]`` triangles, alternately Delaunay and perturbed grids.
    ``workers > 1`` builds the meshes in a spawned process pool."""
    sizes = batch_sizes(n_meshes, t_min, t_max, seed)
    args = [(i, int(t), seed) for i, t in enumerate(sizes)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp

        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_member_args, args, chunksize=16))
    return [batch_member(*a) for a in args]


def workload(name: str) -> HalfEdgeMesh:
    """Build one of the named synthetic workloads."""
    if name in WORKLOADS:
        return WORKLOADS[name]()
    if name.startswith("pgrid_"):
        return perturbed_grid(int(name.split("_")[1]), 0.3, seed=3)
    if name.startswith("grid_"):
        return exact_grid(int(name.split("_")[1]))
    if name.startswith("delaunay_n"):
        return random_delaunay(int(name[len("delaunay_n"):]), seed=2)
    raise KeyError(name)
