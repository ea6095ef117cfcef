"""Facts about the labels that the relink kernel's one-triangle-per-thread
design rests on, checked on the oracle's stage-2 frontier labels (F0) of
Delaunay meshes, perturbed and exact grids and lattice meshes with exact
ties (CPU only):

* the frontier label of an interior edge is the same on both halves
  (Definition 3 is symmetric in e and twin(e));
* a triangle has at most one frontier half-edge whose successor inside the
  triangle is not frontier, so at most one rotation (Section 4.2);
* every rotation (x = CW(x) = next(twin x) from the triangle's next, until
  frontier) ends at a frontier half-edge whose predecessor inside its own
  triangle is not frontier, so the slots a rotation writes are never the
  ones a triangle fills with its own links;
* the in-triangle links and the rotations give every frontier interior
  half-edge exactly one predecessor, so the links form cycles; they are
  the oracle's relinked next except where the repair points a link at a
  chord (Algorithm 6).
"""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen


def _meshes():
    out = [meshgen.random_delaunay(n, seed=s) for n, s in ((5, 1), (60, 2), (500, 3), (3000, 4))]
    out += [meshgen.perturbed_grid(s, 0.3, seed=s) for s in (2, 7, 40)]
    out += [meshgen.exact_grid(9)]
    for s in range(200, 210):
        try:
            out.append(meshgen.lattice_delaunay(300, 20, seed=s))
            break
        except ValueError:
            continue
    return out


def _nx(e):
    return 3 * (e // 3) + (e % 3 + 1) % 3


def _pv(e):
    return 3 * (e // 3) + (e % 3 + 2) % 3


@pytest.mark.parametrize("mesh", _meshes(), ids=lambda m: m.name)
def test_one_rotation_per_triangle_and_disjoint_prev_slots(mesh):
    r = oracle.run_mesh(mesh)
    T = mesh.n_triangles
    HI = 3 * T
    f0 = r.frontier0.astype(bool)
    twin = np.asarray(mesh.twin)
    # symmetric labels on interior edges
    e = np.arange(HI)
    inner = twin[:HI] < HI
    assert np.array_equal(f0[e[inner]], f0[twin[e[inner]]])
    # at most one frontier half-edge per triangle with a non-frontier successor
    f = f0[:HI].reshape(T, 3)
    succ = np.roll(f, -1, axis=1)                     # F of the next half-edge in the triangle
    pend = f & ~succ
    assert int(pend.sum(axis=1).max(initial=0)) <= 1
    # rotations end at frontier half-edges whose in-triangle predecessor is
    # not frontier; the links (in-triangle ones and rotations) give every
    # frontier interior half-edge exactly one predecessor
    preds = np.zeros(HI, np.int64)
    link = np.full(HI, -1, np.int64)
    for t in range(T):
        for k in range(3):
            x0 = 3 * t + k
            if not f0[x0]:
                continue
            x = _nx(x0)
            if f0[x]:
                preds[x] += 1
                link[x0] = x
                continue
            steps = 0
            while not f0[x]:
                x = _nx(int(twin[x]))
                steps += 1
                assert steps <= 64
            assert not f0[_pv(x)], f"rotation from {x0} ends at {x}, whose predecessor is frontier"
            preds[x] += 1
            link[x0] = x
    front = np.flatnonzero(f0[:HI])
    assert np.all(preds[front] == 1)
    assert np.all(preds[~f0[:HI]] == 0)
    nxo = r.next_out[front]
    kept = f0[nxo]                                     # links not redirected to a chord by the repair
    assert np.array_equal(link[front][kept], nxo[kept])
    n_chords = int(np.count_nonzero(r.frontier1[:HI].astype(bool) & ~f0[:HI]))
    assert np.count_nonzero(~kept) <= n_chords
    if r.stats["tips"] == 0:
        assert np.all(kept)
