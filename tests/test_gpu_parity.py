"""Parity of the sm_103a CUDA path with the CPU oracle, through the C ABI.

Every output is integer (labels, links, polygon lists), so the bar is
bit-exact equality of every array, stage by stage: longest edges (stage 1),
frontier labels (2), seeds (3), relinked next/prev (4), tips, chords and
repaired frontier (5a), and the CSR polygon output (5b-5d).
"""
import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import meshgen, polylla
from tests import checks
from tests.gpu_helpers import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


def _tip_meshes(n=4):
    out = []
    for s in range(60):
        m = meshgen.random_delaunay(200, seed=5000 + s)
        if oracle.run_mesh(m).stats["tips"] >= 2:
            out.append(m)
        if len(out) >= n:
            break
    return out


def _lattice(seed):
    for s in range(seed, seed + 10):
        try:
            return meshgen.lattice_delaunay(400, 24, seed=s)
        except ValueError:
            continue
    raise AssertionError("no lattice mesh")


def _near_tie(seed):
    for s in range(seed, seed + 10):
        try:
            return meshgen.near_tie_delaunay(3000, 60, seed=s)
        except ValueError:
            continue
    raise AssertionError("no near-tie mesh")


SMALL = [
    meshgen.two_triangle_square,
    lambda: meshgen.from_triangles([[0, 1, 2]], [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]], name="one_triangle"),
    lambda: meshgen.exact_grid(2),
    lambda: meshgen.exact_grid(5),
    lambda: meshgen.exact_grid(33),
    lambda: meshgen.perturbed_grid(24, 0.3, seed=11),
    lambda: meshgen.perturbed_grid(300, 0.3, seed=3),
    lambda: meshgen.random_delaunay(60, seed=100),
    lambda: meshgen.random_delaunay(2000, seed=1),       # the 2,000-point workload
    lambda: meshgen.random_delaunay(30_000, seed=7),
    lambda: _lattice(200),                                # exact ties everywhere
    lambda: _lattice(300),
    lambda: _near_tie(0),                                 # lengths equal up to a few ulps
    lambda: _near_tie(1),
]


@pytest.mark.parametrize("make", SMALL, ids=lambda f: getattr(f, "__name__", "mesh"))
def test_parity_small(make):
    mesh = make()
    g = gpu_run(mesh)
    r = oracle.run_mesh(mesh)
    assert_parity(mesh, g, r)


@pytest.mark.parametrize("mesh", _tip_meshes(), ids=lambda m: m.name)
def test_parity_with_barrier_tips(mesh):
    g = gpu_run(mesh)
    r = oracle.run_mesh(mesh)
    assert r.stats["tips"] >= 2
    assert_parity(mesh, g, r)


def test_parity_random_sweep():
    """Forty small meshes of random kinds and sizes (3-point to 600-point
    Delaunay meshes, 2x2 to 41x41 perturbed and exact grids, lattice meshes
    with exact ties), every array against the oracle."""
    rng = np.random.default_rng(2024)
    for i in range(40):
        kind = i % 4
        if kind == 0:
            mesh = meshgen.random_delaunay(int(rng.integers(3, 600)), seed=int(rng.integers(1 << 30)))
        elif kind == 1:
            mesh = meshgen.perturbed_grid(int(rng.integers(2, 42)), 0.3, seed=int(rng.integers(1 << 30)))
        elif kind == 2:
            mesh = meshgen.exact_grid(int(rng.integers(2, 42)))
        else:
            try:
                mesh = meshgen.lattice_delaunay(int(rng.integers(10, 300)), int(rng.integers(8, 30)),
                                                seed=int(rng.integers(1 << 30)))
            except ValueError:
                continue
        g = gpu_run(mesh)
        assert_parity(mesh, g, oracle.run_mesh(mesh))


@pytest.mark.parametrize("tile,items", [(64, 1), (128, 1), (256, 1), (256, 2), (256, 4)])
def test_parity_every_relink_setting(tile, items):
    """Every relink launch setting (triangles per CTA, per thread) gives the
    oracle's arrays on meshes with barrier tips, exact ties and a ragged
    last CTA."""
    for mesh in [meshgen.random_delaunay(3000, seed=77), meshgen.perturbed_grid(61, 0.3, seed=5),
                 _lattice(500), _near_tie(2)] + _tip_meshes(2):
        g = gpu_run(mesh, tuning={"relink_tile": tile, "relink_items": items})
        assert_parity(mesh, g, oracle.run_mesh(mesh))


def test_parity_generate_is_repeatable():
    """generate never reads the input next/prev of interior half-edges, so a
    second and third call on the rewritten arrays give the same result."""
    mesh = meshgen.random_delaunay(5000, seed=21)
    g = gpu_run(mesh, generate_times=3)
    assert_parity(mesh, g, oracle.run_mesh(mesh))


def test_parity_delaunay_1m():
    """1,000,000 uniform random points (Delaunay): every array, full size."""
    mesh = meshgen.workload("delaunay_1m")
    g = gpu_run(mesh)
    r = oracle.run_mesh(mesh)
    assert r.stats["tips"] > 1000
    assert_parity(mesh, g, r)


def test_parity_perturbed_grid_4096():
    """The 4096 x 4096 perturbed grid (33.5M triangles): every array, full
    size, plus the output invariants; then again in the launch
    configuration bench.py times (autotuned, from a CUDA graph, on a side
    stream)."""
    mesh = meshgen.workload("pgrid_4096")
    g = gpu_run(mesh)
    r = oracle.run_mesh(mesh)
    assert_parity(mesh, g, r)
    checks.check_output_invariants(
        mesh, r.frontier1, g["next"], g["prev"], g["seeds"], g["offsets"], g["he_list"], g["v_list"],
        n_seeds_alg4=len(r.seed_list), n_distinct_chords=r.stats["distinct_chords"])
    del g
    try:
        g = gpu_run(mesh, as_benched=True)
    finally:
        polylla.polylla_tuning_cache_clear()
    assert_parity(mesh, g, r)


def test_rejects_corrupt_mesh():
    import torch

    mesh = meshgen.random_delaunay(300, seed=2)
    dm = polylla.DeviceMesh.from_host(mesh)
    dm.twin[5] = dm.twin[6]                    # twin is no longer an involution
    with pytest.raises(polylla.PolyllaError) as ei:
        polylla.polylla_create(dm)
    assert ei.value.status == -2
    dm2 = polylla.DeviceMesh.from_host(mesh)
    dm2.next[4] = 7                            # interior next off the triangle layout
    with pytest.raises(polylla.PolyllaError):
        polylla.polylla_create(dm2)
    dm3 = polylla.DeviceMesh.from_host(mesh)
    dm3.coords[3, 0] = float("nan")
    with pytest.raises(polylla.PolyllaError):
        polylla.polylla_create(dm3)
    torch.cuda.synchronize()


def test_rotation_cap_reports_nonterminating():
    """A rotation cap of 1 is too small for a Delaunay mesh: generate must
    stop and report the status, not hang or fault."""
    mesh = meshgen.random_delaunay(3000, seed=4)
    dm = polylla.DeviceMesh.from_host(mesh)
    ctx = polylla.polylla_create(dm, max_rotation=1)
    try:
        polylla.polylla_generate(ctx)
        with pytest.raises(polylla.PolyllaError) as ei:
            polylla.polylla_get_polygons(ctx)
        assert ei.value.status == -5
        assert polylla.polylla_last_error(ctx) == -5
    finally:
        polylla.polylla_destroy(ctx)


def test_host_buffer_path_matches_device_path():
    import torch

    mesh = meshgen.random_delaunay(20_000, seed=8)
    r = oracle.run_mesh(mesh)
    T, H, V = mesh.n_triangles, mesh.n_halfedges, mesh.n_vertices
    ctx = polylla.polylla_create_host(V, T, H)
    try:
        hin = {k: torch.from_numpy(getattr(mesh, k)).pin_memory() for k in ("coords", "origin", "twin", "next", "prev")}
        hout = {"seeds": torch.empty(T, dtype=torch.int32).pin_memory(),
                "offsets": torch.empty(T + 1, dtype=torch.int32).pin_memory(),
                "he_list": torch.empty(3 * T, dtype=torch.int32).pin_memory(),
                "v_list": torch.empty(3 * T, dtype=torch.int32).pin_memory(),
                "next": torch.empty(H, dtype=torch.int32).pin_memory(),
                "prev": torch.empty(H, dtype=torch.int32).pin_memory()}
        for validate in (True, False):
            P, NF = polylla.polylla_generate_host(ctx, hin, hout, validate=validate)
            assert P == r.n_polygons and NF == r.he_list.shape[0]
            assert np.array_equal(hout["seeds"][:P].numpy(), r.seeds)
            assert np.array_equal(hout["offsets"][:P + 1].numpy(), r.offsets)
            assert np.array_equal(hout["he_list"][:NF].numpy(), r.he_list)
            assert np.array_equal(hout["v_list"][:NF].numpy(), r.v_list)
            assert np.array_equal(hout["next"].numpy(), r.next_out)
            assert np.array_equal(hout["prev"].numpy(), r.prev_out)
    finally:
        polylla.polylla_destroy(ctx)


def test_stage_timing_and_launch_count():
    mesh = meshgen.random_delaunay(20_000, seed=9)
    dm = polylla.DeviceMesh.from_host(mesh)
    with polylla.Polylla(dm) as p:
        polylla.polylla_set_timing(p.ctx, True)
        p.generate()
        t = polylla.polylla_get_stage_times(p.ctx)
        assert list(t) == ["longest_edge", "label_relink", "chords", "chord_links", "poly_count", "tile_scan",
                           "poly_list", "batch_meta"]
        assert all(v >= 0 for v in t.values())
        assert t["batch_meta"] == 0
        assert polylla.polylla_launch_count(p.ctx) == 7
