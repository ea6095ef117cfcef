"""GPU parity of the convexification (polylla_convexify) with the oracle's.

All outputs are integer, so the bar is bit-exact equality: the frontier
after the chords (flags bits 0-2), next/prev of every half-edge, the chosen
chord half-edges (as a set: threads append them in any order) and the CSR
of the convex polygons.  The turn test is a binary64 cross product with
every operation rounded on its own on both sides, so both take the same
decision on every corner."""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import build, meshgen, polylla

pytestmark = pytest.mark.gpu


def gpu_convex(mesh, times: int = 1):
    import torch

    build.build_library()
    dm = polylla.DeviceMesh.from_host(mesh)
    with polylla.Polylla(dm) as p:
        p.generate()
        for _ in range(times):
            p.convexify()
        out = p.polygons()
        lab = p.labels()
        chords = polylla.polylla_convex_chords(p.ctx).cpu().numpy()
        torch.cuda.synchronize()
        return {
            "n_polygons": out["n_polygons"], "n_frontier": out["n_frontier"],
            "seeds": out["seeds"].cpu().numpy(), "offsets": out["offsets"].cpu().numpy(),
            "he_list": out["he_list"].cpu().numpy(), "v_list": out["v_list"].cpu().numpy(),
            "next": dm.next.cpu().numpy(), "prev": dm.prev.cpu().numpy(),
            "flags": lab["flags"].cpu().numpy(), "chords": chords,
        }


def assert_convex_parity(mesh, g, chords_too=True):
    r = oracle.run_mesh(mesh)
    c = oracle.convexify(mesh, r)
    T = mesh.n_triangles
    HI = 3 * T
    f2 = c.frontier2[:HI].reshape(T, 3).astype(np.uint8)
    gf = np.stack([(g["flags"] >> k) & 1 for k in range(3)], axis=1).astype(np.uint8)
    assert np.array_equal(gf, f2), "frontier after the chords differs"
    if chords_too:
        assert sorted(g["chords"].tolist()) == sorted(c.chords.tolist()), "chosen chords differ"
    assert np.array_equal(g["next"][:HI], c.next_out[:HI]), "next differs"
    assert np.array_equal(g["prev"][:HI], c.prev_out[:HI]), "prev differs"
    assert g["n_polygons"] == c.n_polygons and g["n_frontier"] == c.he_list.shape[0]
    for k in ("seeds", "offsets", "he_list", "v_list"):
        assert np.array_equal(g[k], getattr(c, k)), f"{k} differs"
    return c


@pytest.mark.parametrize("n, seed", [(60, 1), (300, 2), (2000, 3), (30000, 4)])
def test_convex_parity_random_delaunay(n, seed):
    mesh = meshgen.random_delaunay(n, seed=500 + seed)
    c = assert_convex_parity(mesh, gpu_convex(mesh))
    assert c.stats["distinct_chords"] > 0


@pytest.mark.parametrize("s", [24, 300])
def test_convex_parity_perturbed_grid(s):
    mesh = meshgen.perturbed_grid(s, 0.3, seed=510 + s)
    assert_convex_parity(mesh, gpu_convex(mesh))


def test_convex_parity_exact_grid_and_lattice():
    mesh = meshgen.exact_grid(33)
    c = assert_convex_parity(mesh, gpu_convex(mesh))
    assert c.chords.shape[0] == 0
    for s in range(3):
        try:
            lat = meshgen.lattice_delaunay(2000, 60, seed=520 + s)
        except ValueError:
            continue
        assert_convex_parity(lat, gpu_convex(lat))
        break


def test_convex_parity_near_ties():
    """Lattice coordinates moved by a few ulps: turn tests close to zero,
    where the float32 filter must defer to binary64."""
    done = 0
    for s in range(6):
        try:
            mesh = meshgen.near_tie_delaunay(3000, 80, seed=525 + s)
        except ValueError:
            continue
        assert_convex_parity(mesh, gpu_convex(mesh))
        done += 1
        if done == 2:
            break
    assert done > 0


def test_convex_twice_is_a_fixed_point_and_generate_restores():
    import torch

    mesh = meshgen.random_delaunay(5000, seed=530)
    g2 = gpu_convex(mesh, times=2)
    assert g2["chords"].shape[0] == 0                 # the second call finds every corner convex
    assert_convex_parity(mesh, g2, chords_too=False)
    # a generate after a convexify gives the plain Polylla mesh again
    r = oracle.run_mesh(mesh)
    dm = polylla.DeviceMesh.from_host(mesh)
    with polylla.Polylla(dm) as p:
        p.generate()
        p.convexify()
        p.generate()
        out = p.polygons()
        assert np.array_equal(out["he_list"].cpu().numpy(), r.he_list)
        assert np.array_equal(dm.next.cpu().numpy(), r.next_out)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["delaunay_1m", "pgrid_4096"])
def test_convex_parity_full_size(name):
    mesh = meshgen.workload(name)
    c = assert_convex_parity(mesh, gpu_convex(mesh))
    assert c.stats["left_reflex"] == 0


def test_convexify_rejects_batches():
    meshes = [meshgen.random_delaunay(100, seed=540 + i) for i in range(3)]
    db = polylla.DeviceBatch.from_host(meshes)
    ctx = polylla.polylla_batch_create(db)
    try:
        with pytest.raises(polylla.PolyllaError) as e:
            polylla.polylla_convexify(ctx)
        assert e.value.status == -1
    finally:
        polylla.polylla_destroy(ctx)
