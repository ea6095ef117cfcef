"""polylla_generate_noalloc: the no-allocation entry point.

It exists for callers that cannot call cudaMalloc: a serving loop that must
not allocate once it runs (an allocation can block on, or fail against,
memory that other work holds), or a process whose device memory belongs to
another allocator.  The library keeps the call's scratch in one static
device array of fixed size, and the caller supplies the mesh and the output
buffers.  These tests call it through the C ABI and check its result, bit
for bit and on two calls in a row, against the context-based entry point
(polylla_create / polylla_generate / polylla_get_polygons) and, on a mesh
just under the array's limit with many barrier tips, against the oracle.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2403_14723_gb300 import build, meshgen, polylla

pytestmark = pytest.mark.gpu


def _context_result(mesh):
    import torch

    dm = polylla.DeviceMesh.from_host(mesh)
    with polylla.Polylla(dm) as p:
        p.generate()
        out = p.polygons()
        res = {k: out[k].cpu().numpy() for k in ("seeds", "offsets", "he_list", "v_list")}
        res["n_polygons"], res["n_frontier"] = out["n_polygons"], out["n_frontier"]
        res["next"], res["prev"] = dm.next.cpu().numpy(), dm.prev.cpu().numpy()
    torch.cuda.synchronize()
    return res


def _oracle_result(mesh):
    r = oracle.run_mesh(mesh)
    return {"seeds": r.seeds, "offsets": r.offsets, "he_list": r.he_list, "v_list": r.v_list,
            "n_polygons": r.n_polygons, "n_frontier": int(r.he_list.shape[0]),
            "next": r.next_out, "prev": r.prev_out, "tips": r.stats["tips"]}


def _noalloc_call(lib, mesh, dm, outs, stream):
    T = mesh.n_triangles
    m = polylla.polylla_mesh(
        mesh.n_vertices, T, mesh.n_halfedges,
        ctypes.c_void_p(dm.coords.data_ptr()), ctypes.c_void_p(dm.origin.data_ptr()),
        ctypes.c_void_p(dm.twin.data_ptr()), ctypes.c_void_p(dm.next.data_ptr()),
        ctypes.c_void_p(dm.prev.data_ptr()))
    rc = lib.polylla_generate_noalloc(
        ctypes.byref(m), *(ctypes.c_void_p(outs[k].data_ptr()) for k in ("seeds", "offsets", "he_list", "v_list",
                                                                           "status")),
        ctypes.c_void_p(stream.cuda_stream))
    return rc


def _check_twice(mesh, want):
    """Two no-allocation calls in a row on fresh output buffers filled with
    junk, each compared with ``want`` array by array."""
    import torch

    build.build_library()
    lib = polylla.load_library()
    T = mesh.n_triangles
    assert T <= polylla.POLYLLA_NOALLOC_MAX_TRIANGLES
    dm = polylla.DeviceMesh.from_host(mesh)
    stream = torch.cuda.current_stream()
    outs = {"seeds": torch.empty(T, dtype=torch.int32, device="cuda"),
            "offsets": torch.empty(T + 1, dtype=torch.int32, device="cuda"),
            "he_list": torch.empty(3 * T, dtype=torch.int32, device="cuda"),
            "v_list": torch.empty(3 * T, dtype=torch.int32, device="cuda"),
            "status": torch.empty(3, dtype=torch.int32, device="cuda")}
    for call in range(2):
        for t in outs.values():
            t.fill_(-7)                                # stale contents must not matter
        assert _noalloc_call(lib, mesh, dm, outs, stream) == 0
        torch.cuda.synchronize()
        P, NF, err = outs["status"].cpu().tolist()
        assert err == 0, f"call {call}: device error bits {err}"
        assert P == want["n_polygons"] and NF == want["n_frontier"]
        assert np.array_equal(outs["seeds"][:P].cpu().numpy(), want["seeds"])
        assert np.array_equal(outs["offsets"][:P + 1].cpu().numpy(), want["offsets"])
        assert np.array_equal(outs["he_list"][:NF].cpu().numpy(), want["he_list"])
        assert np.array_equal(outs["v_list"][:NF].cpu().numpy(), want["v_list"])
        assert np.array_equal(dm.next.cpu().numpy(), want["next"])
        assert np.array_equal(dm.prev.cpu().numpy(), want["prev"])


def test_noalloc_matches_context_entry_point_twice():
    mesh = meshgen.random_delaunay(4000, seed=31)     # ~7,970 triangles, with barrier tips
    _check_twice(mesh, _context_result(mesh))


def test_noalloc_at_its_limit_matches_oracle_twice():
    """A Delaunay mesh just under POLYLLA_NOALLOC_MAX_TRIANGLES: the static
    label, tip and chord regions and the output tiles' look-back words are
    used up to (nearly) their full size, with thousands of barrier tips."""
    mesh = meshgen.random_delaunay(65_500, seed=33)
    T = mesh.n_triangles
    assert 0.99 * polylla.POLYLLA_NOALLOC_MAX_TRIANGLES < T <= polylla.POLYLLA_NOALLOC_MAX_TRIANGLES
    want = _oracle_result(mesh)
    assert want["tips"] > 1000
    _check_twice(mesh, want)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import torch

    build.build_library()
    lib = polylla.load_library()
    T = polylla.POLYLLA_NOALLOC_MAX_TRIANGLES + 1
    dummy = torch.empty(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    m = polylla.polylla_mesh(T + 2, T, 3 * T + 3, p, p, p, p, p)
    rc = lib.polylla_generate_noalloc(ctypes.byref(m), p, p, p, p, p, ctypes.c_void_p(0))
    assert rc == -8
    assert lib.polylla_status_string(rc).startswith(b"mesh larger than the available capacity")
