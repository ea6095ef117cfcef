"""Thin Python binding of libpolylla (``include/polylla.h``).

Argument marshalling only: every step of the method runs in the CUDA
library.  Device arrays are torch CUDA tensors (PyTorch supplies device
memory and streams); functions keep the C names.  If the library has not
been built, or no CUDA device is usable, calls raise -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

POLYLLA_OK = 0
STATUS = {
    0: "ok", -1: "invalid argument", -2: "invalid mesh layout", -3: "out of device memory",
    -4: "CUDA error", -5: "rotation or cycle walk did not terminate",
    -6: "internal list capacity exceeded", -7: "device wait timed out",
    -8: "mesh larger than the no-allocation scratch",
}
POLYLLA_NOALLOC_MAX_TRIANGLES = 131072


class PolyllaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")


class polylla_mesh(ctypes.Structure):
    _fields_ = [
        ("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32), ("n_halfedges", ctypes.c_int32),
        ("coords", ctypes.c_void_p), ("origin", ctypes.c_void_p), ("twin", ctypes.c_void_p),
        ("next", ctypes.c_void_p), ("prev", ctypes.c_void_p),
    ]


class polylla_options(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int32), ("max_rotation", ctypes.c_int32)]


class polylla_polygons(ctypes.Structure):
    _fields_ = [
        ("n_polygons", ctypes.c_int32), ("n_frontier", ctypes.c_int32),
        ("seeds", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
        ("he_list", ctypes.c_void_p), ("v_list", ctypes.c_void_p),
    ]


class polylla_labels(ctypes.Structure):
    _fields_ = [
        ("longest_local", ctypes.c_void_p), ("flags", ctypes.c_void_p),
        ("tips", ctypes.c_void_p), ("chords", ctypes.c_void_p), ("n_tips", ctypes.c_int32),
    ]


class polylla_host_mesh(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_void_p), ("origin", ctypes.c_void_p), ("twin", ctypes.c_void_p),
                ("next", ctypes.c_void_p), ("prev", ctypes.c_void_p)]


class polylla_host_result(ctypes.Structure):
    _fields_ = [("seeds", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("he_list", ctypes.c_void_p),
                ("v_list", ctypes.c_void_p), ("next", ctypes.c_void_p), ("prev", ctypes.c_void_p),
                ("n_polygons", ctypes.c_int32), ("n_frontier", ctypes.c_int32)]


class polylla_batch(ctypes.Structure):
    _fields_ = [("n_meshes", ctypes.c_int32),
                ("vertex_offset", ctypes.c_void_p), ("triangle_offset", ctypes.c_void_p),
                ("halfedge_offset", ctypes.c_void_p),
                ("coords", ctypes.c_void_p), ("origin", ctypes.c_void_p), ("twin", ctypes.c_void_p),
                ("next", ctypes.c_void_p), ("prev", ctypes.c_void_p)]


class polylla_tuning(ctypes.Structure):
    _fields_ = [("relink_tile", ctypes.c_int32), ("relink_items", ctypes.c_int32),
                ("longest_edge_blocks", ctypes.c_int32), ("longest_edge_items", ctypes.c_int32),
                ("output_tile", ctypes.c_int32), ("output_items", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class polylla_server_options(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("max_batch_meshes", ctypes.c_int32), ("max_rotation", ctypes.c_int32),
                ("max_batch_triangles", ctypes.c_int32), ("lane_triangles", ctypes.c_int32)]


class polylla_request(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32), ("n_halfedges", ctypes.c_int32),
                ("mesh", polylla_host_mesh), ("result", polylla_host_result)]


class polylla_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_polygons", ctypes.c_int32), ("n_frontier", ctypes.c_int32),
                ("batch_meshes", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class polylla_server_stats(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("slot_triangles", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("requests_done", ctypes.c_int64), ("busy_seconds", ctypes.c_double),
                ("mean_in_ms", ctypes.c_double), ("mean_run_ms", ctypes.c_double), ("mean_out_ms", ctypes.c_double),
                ("max_batch_ms", ctypes.c_double), ("max_batch_triangles", ctypes.c_int64),
                ("max_batch_requests", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("lane_batches", ctypes.c_int64), ("lane_triangles", ctypes.c_int32),
                ("lane_slot_triangles", ctypes.c_int32)]


class polylla_server_plan(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("slot_triangles", ctypes.c_int32), ("lane_triangles", ctypes.c_int32),
                ("lane_slot_triangles", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class polylla_batch_record(ctypes.Structure):
    _fields_ = [("t_form", ctypes.c_double), ("t_enqueued", ctypes.c_double), ("t_meta_seen", ctypes.c_double),
                ("t_out_enqueued", ctypes.c_double), ("t_done", ctypes.c_double), ("in_ms", ctypes.c_float),
                ("run_ms", ctypes.c_float), ("idle_ms", ctypes.c_float), ("out_ms", ctypes.c_float),
                ("n_triangles", ctypes.c_int64), ("n_requests", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("lane", ctypes.c_int32), ("t_stream_start", ctypes.c_double), ("t_meta_landed", ctypes.c_double)]


# every function the header declares, with its ctypes signature
_SIGNATURES = {
    "polylla_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(polylla_mesh),
                                      ctypes.POINTER(polylla_options), ctypes.c_void_p]),
    "polylla_generate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polylla_get_polygons": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_polygons), ctypes.c_void_p]),
    "polylla_last_error": (ctypes.c_int, [ctypes.c_void_p]),
    "polylla_cuda_error": (ctypes.c_int, [ctypes.c_void_p]),
    "polylla_destroy": (None, [ctypes.c_void_p]),
    "polylla_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "polylla_get_labels": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_labels), ctypes.c_void_p]),
    "polylla_create_host": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.POINTER(polylla_options)]),
    "polylla_generate_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_host_mesh),
                                             ctypes.POINTER(polylla_host_result), ctypes.c_int32, ctypes.c_void_p]),
    "polylla_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "polylla_get_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "polylla_stage_count": (ctypes.c_int, []),
    "polylla_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "polylla_launch_count": (ctypes.c_int, [ctypes.c_void_p]),
    "polylla_generate_noalloc": (ctypes.c_int, [ctypes.POINTER(polylla_mesh), ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "polylla_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(polylla_batch),
                                            ctypes.POINTER(polylla_options), ctypes.c_void_p]),
    "polylla_batch_polygon_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "polylla_capture_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polylla_release_graph": (ctypes.c_int, [ctypes.c_void_p]),
    "polylla_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_tuning)]),
    "polylla_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_tuning)]),
    "polylla_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(polylla_tuning),
                                        ctypes.c_void_p]),
    "polylla_tuning_cache_clear": (ctypes.c_int, []),
    "polylla_lepp_terminal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "polylla_convexify": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "polylla_convex_chords": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "polylla_lepp_paths": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "polylla_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(polylla_server_options)]),
    "polylla_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_request),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "polylla_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(polylla_request_info)]),
    "polylla_server_replay": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(polylla_request),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(polylla_request_info)]),
    "polylla_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_server_stats)]),
    "polylla_server_plan_slots": (ctypes.c_int, [ctypes.POINTER(polylla_server_options),
                                                 ctypes.POINTER(polylla_server_plan)]),
    "polylla_server_get_batch_log": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(polylla_batch_record),
                                                    ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                    ctypes.POINTER(ctypes.c_int64)]),
    "polylla_server_destroy": (None, [ctypes.c_void_p]),
}

_lib = None


def load_library(path: str | None = None):
    """Load libpolylla.so (built by ``build.build_library``); raise if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    so = path or _build.library_path()
    if not os.path.exists(so):
        raise RuntimeError(f"libpolylla is not built ({so} missing); run paper_2403_14723_gb300.build.build_library()")
    lib = ctypes.CDLL(so)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != POLYLLA_OK:
        raise PolyllaError(rc, where)


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, n):
    import torch

    if not t.is_cuda:
        raise ValueError("device array expected (torch CUDA tensor)")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"expected contiguous {dtype} tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


class _CudaArray:
    """Zero-copy view of context-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3, "strides": None,
        }


def _view(ptr, n, typestr, dtype):
    import torch

    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(int(ptr), int(n), typestr), device="cuda")


@dataclass
class DeviceMesh:
    """The five device arrays of one mesh (torch CUDA tensors)."""

    coords: "object"   # [V, 2] float64
    origin: "object"   # [H] int32
    twin: "object"
    next: "object"
    prev: "object"
    n_triangles: int

    @classmethod
    def from_host(cls, mesh, device="cuda"):
        import torch

        return cls(
            coords=torch.from_numpy(mesh.coords).to(device).contiguous(),
            origin=torch.from_numpy(mesh.origin).to(device),
            twin=torch.from_numpy(mesh.twin).to(device),
            next=torch.from_numpy(mesh.next).to(device),
            prev=torch.from_numpy(mesh.prev).to(device),
            n_triangles=int(mesh.n_triangles),
        )


def polylla_create(mesh: DeviceMesh, validate: bool = True, max_rotation: int = 0, stream=None) -> int:
    """Create a context on a device mesh; returns the context handle."""
    import torch

    lib = load_library()
    V = mesh.coords.shape[0]
    H = mesh.origin.numel()
    m = polylla_mesh(V, int(mesh.n_triangles), H,
                     _dev_ptr(mesh.coords.view(-1), torch.float64, 2 * V),
                     _dev_ptr(mesh.origin, torch.int32, H), _dev_ptr(mesh.twin, torch.int32, H),
                     _dev_ptr(mesh.next, torch.int32, H), _dev_ptr(mesh.prev, torch.int32, H))
    opt = polylla_options(1 if validate else 0, int(max_rotation))
    ctx = ctypes.c_void_p()
    _check(lib.polylla_create(ctypes.byref(ctx), ctypes.byref(m), ctypes.byref(opt), _stream_ptr(stream)),
           "polylla_create")
    return ctx.value


def polylla_generate(ctx: int, stream=None) -> None:
    _check(load_library().polylla_generate(ctypes.c_void_p(ctx), _stream_ptr(stream)), "polylla_generate")


def polylla_get_polygons(ctx: int, stream=None) -> dict:
    """Return ``{n_polygons, n_frontier, seeds, offsets, he_list, v_list}``
    with zero-copy int32 CUDA tensors over the context's buffers."""
    import torch

    out = polylla_polygons()
    _check(load_library().polylla_get_polygons(ctypes.c_void_p(ctx), ctypes.byref(out), _stream_ptr(stream)),
           "polylla_get_polygons")
    P, NF = out.n_polygons, out.n_frontier
    return {
        "n_polygons": P, "n_frontier": NF,
        "seeds": _view(out.seeds, P, "<i4", torch.int32),
        "offsets": _view(out.offsets, P + 1, "<i4", torch.int32),
        "he_list": _view(out.he_list, NF, "<i4", torch.int32),
        "v_list": _view(out.v_list, NF, "<i4", torch.int32),
    }


def polylla_get_labels(ctx: int, n_triangles: int, stream=None) -> dict:
    import torch

    out = polylla_labels()
    _check(load_library().polylla_get_labels(ctypes.c_void_p(ctx), ctypes.byref(out), _stream_ptr(stream)),
           "polylla_get_labels")
    return {
        "longest_local": _view(out.longest_local, n_triangles, "|u1", torch.uint8),
        "flags": _view(out.flags, n_triangles, "|u1", torch.uint8),
        "tips": _view(out.tips, out.n_tips, "<i4", torch.int32),
        "chords": _view(out.chords, out.n_tips, "<i4", torch.int32),
        "n_tips": out.n_tips,
    }


def polylla_last_error(ctx: int) -> int:
    return load_library().polylla_last_error(ctypes.c_void_p(ctx))


def polylla_cuda_error(ctx: int) -> int:
    return load_library().polylla_cuda_error(ctypes.c_void_p(ctx))


def polylla_destroy(ctx: int) -> None:
    if ctx:
        load_library().polylla_destroy(ctypes.c_void_p(ctx))


def polylla_status_string(status: int) -> str:
    return load_library().polylla_status_string(int(status)).decode()


def polylla_set_timing(ctx: int, enable: bool) -> None:
    _check(load_library().polylla_set_timing(ctypes.c_void_p(ctx), 1 if enable else 0), "polylla_set_timing")


def polylla_get_stage_times(ctx: int) -> dict:
    lib = load_library()
    n = lib.polylla_stage_count()
    buf = (ctypes.c_float * n)()
    k = lib.polylla_get_stage_times(ctypes.c_void_p(ctx), buf, n)
    if k < 0:
        raise PolyllaError(k, "polylla_get_stage_times")
    return {lib.polylla_stage_name(i).decode(): float(buf[i]) for i in range(k)}


def polylla_stage_count() -> int:
    return load_library().polylla_stage_count()


def polylla_stage_name(i: int) -> str:
    return load_library().polylla_stage_name(int(i)).decode()


def polylla_launch_count(ctx: int) -> int:
    return load_library().polylla_launch_count(ctypes.c_void_p(ctx))


def polylla_create_host(n_vertices: int, n_triangles: int, n_halfedges: int, max_rotation: int = 0) -> int:
    lib = load_library()
    opt = polylla_options(0, int(max_rotation))
    ctx = ctypes.c_void_p()
    _check(lib.polylla_create_host(ctypes.byref(ctx), int(n_vertices), int(n_triangles), int(n_halfedges),
                                   ctypes.byref(opt)), "polylla_create_host")
    return ctx.value


def polylla_generate_host(ctx: int, host_in: dict, host_out: dict, validate: bool = False, stream=None) -> tuple:
    """Host-buffer path.  ``host_in``: coords/origin/twin/next/prev CPU
    tensors (pinned for speed); ``host_out``: seeds/offsets/he_list/v_list/
    next/prev CPU int32 tensors of the documented capacities.  Returns
    ``(n_polygons, n_frontier)``."""
    lib = load_library()
    hm = polylla_host_mesh(*(ctypes.c_void_p(host_in[k].data_ptr()) for k in ("coords", "origin", "twin", "next", "prev")))
    hr = polylla_host_result(*(ctypes.c_void_p(host_out[k].data_ptr())
                               for k in ("seeds", "offsets", "he_list", "v_list", "next", "prev")), 0, 0)
    _check(lib.polylla_generate_host(ctypes.c_void_p(ctx), ctypes.byref(hm), ctypes.byref(hr),
                                     1 if validate else 0, _stream_ptr(stream)), "polylla_generate_host")
    return hr.n_polygons, hr.n_frontier


def polylla_generate_noalloc(mesh: DeviceMesh, seeds, offsets, he_list, v_list, status3, stream=None) -> None:
    """The whole method with no allocation in the library: the caller
    passes device tensors for the outputs (int32, capacities T, T+1, 3T, 3T)
    and a device int32[3] that receives P, N_F and the device error bits.
    Does not synchronize."""
    import torch

    lib = load_library()
    V = mesh.coords.shape[0]
    H = mesh.origin.numel()
    T = int(mesh.n_triangles)
    m = polylla_mesh(V, T, H,
                     _dev_ptr(mesh.coords.view(-1), torch.float64, 2 * V),
                     _dev_ptr(mesh.origin, torch.int32, H), _dev_ptr(mesh.twin, torch.int32, H),
                     _dev_ptr(mesh.next, torch.int32, H), _dev_ptr(mesh.prev, torch.int32, H))
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (seeds, offsets, he_list, v_list, status3)]
    for t, n in zip((seeds, offsets, he_list, v_list, status3), (T, T + 1, 3 * T, 3 * T, 3)):
        if not t.is_cuda or t.dtype != torch.int32 or t.numel() < n:
            raise ValueError(f"device int32 tensor of at least {n} elements expected")
    _check(lib.polylla_generate_noalloc(ctypes.byref(m), *ptrs, _stream_ptr(stream)), "polylla_generate_noalloc")


def polylla_capture_graph(ctx: int, stream=None) -> None:
    """Record one generate into a CUDA graph that later generates launch
    (the stream must be a non-default torch stream)."""
    _check(load_library().polylla_capture_graph(ctypes.c_void_p(ctx), _stream_ptr(stream)), "polylla_capture_graph")


def polylla_release_graph(ctx: int) -> None:
    _check(load_library().polylla_release_graph(ctypes.c_void_p(ctx)), "polylla_release_graph")


def polylla_get_tuning(ctx: int) -> dict:
    t = polylla_tuning()
    _check(load_library().polylla_get_tuning(ctypes.c_void_p(ctx), ctypes.byref(t)), "polylla_get_tuning")
    return t.as_dict()


def polylla_set_tuning(ctx: int, tuning: dict) -> None:
    t = polylla_tuning(**{k: int(v) for k, v in tuning.items()})
    _check(load_library().polylla_set_tuning(ctypes.c_void_p(ctx), ctypes.byref(t)), "polylla_set_tuning")


def polylla_autotune(ctx: int, reps: int = 5, stream=None) -> dict:
    t = polylla_tuning()
    _check(load_library().polylla_autotune(ctypes.c_void_p(ctx), int(reps), ctypes.byref(t), _stream_ptr(stream)),
           "polylla_autotune")
    return t.as_dict()


def polylla_tuning_cache_clear() -> None:
    _check(load_library().polylla_tuning_cache_clear(), "polylla_tuning_cache_clear")


@dataclass
class DeviceBatch:
    """Concatenated device arrays of a batch of meshes plus host prefix sums
    (see ``polylla_batch`` in the header)."""

    coords: "object"           # [V_total, 2] float64
    origin: "object"           # [H_total] int32, local indices per mesh
    twin: "object"
    next: "object"
    prev: "object"
    vertex_offset: "object"    # host numpy int32 [n+1]
    triangle_offset: "object"
    halfedge_offset: "object"

    @property
    def n_meshes(self) -> int:
        return len(self.triangle_offset) - 1

    @classmethod
    def from_host(cls, meshes, device="cuda"):
        """Concatenate host meshes (``meshgen.HalfEdgeMesh``) into one batch."""
        import numpy as np
        import torch

        def cat(name):
            return torch.from_numpy(np.concatenate([getattr(m, name) for m in meshes])).to(device).contiguous()

        def prefix(vals):
            out = np.zeros(len(vals) + 1, dtype=np.int64)
            np.cumsum(vals, out=out[1:])
            if out[-1] >= 2 ** 31:
                raise ValueError("batch exceeds int32 indexing")
            return out.astype(np.int32)

        return cls(coords=cat("coords"), origin=cat("origin"), twin=cat("twin"), next=cat("next"), prev=cat("prev"),
                   vertex_offset=prefix([m.n_vertices for m in meshes]),
                   triangle_offset=prefix([m.n_triangles for m in meshes]),
                   halfedge_offset=prefix([m.n_halfedges for m in meshes]))


def polylla_batch_create(batch: DeviceBatch, validate: bool = True, max_rotation: int = 0, stream=None) -> int:
    import numpy as np
    import torch

    lib = load_library()
    V = int(batch.vertex_offset[-1])
    H = int(batch.halfedge_offset[-1])
    offs = [np.ascontiguousarray(a, dtype=np.int32) for a in
            (batch.vertex_offset, batch.triangle_offset, batch.halfedge_offset)]
    b = polylla_batch(batch.n_meshes, *(ctypes.c_void_p(a.ctypes.data) for a in offs),
                      _dev_ptr(batch.coords.view(-1), torch.float64, 2 * V),
                      _dev_ptr(batch.origin, torch.int32, H), _dev_ptr(batch.twin, torch.int32, H),
                      _dev_ptr(batch.next, torch.int32, H), _dev_ptr(batch.prev, torch.int32, H))
    opt = polylla_options(1 if validate else 0, int(max_rotation))
    ctx = ctypes.c_void_p()
    _check(lib.polylla_batch_create(ctypes.byref(ctx), ctypes.byref(b), ctypes.byref(opt), _stream_ptr(stream)),
           "polylla_batch_create")
    return ctx.value


def polylla_batch_polygon_offsets(ctx: int, n_meshes: int):
    """Device int32 view [n+1]: mesh i owns polygons [off[i], off[i+1])."""
    import torch

    p = ctypes.c_void_p()
    _check(load_library().polylla_batch_polygon_offsets(ctypes.c_void_p(ctx), ctypes.byref(p)),
           "polylla_batch_polygon_offsets")
    return _view(p.value, n_meshes + 1, "<i4", torch.int32)


def polylla_convexify(ctx: int, stream=None) -> None:
    """Split every reflex corner of the last generate's polygons with the
    fewest triangulation edges (see include/polylla.h); the convex polygons
    then come from polylla_get_polygons."""
    _check(load_library().polylla_convexify(ctypes.c_void_p(ctx), _stream_ptr(stream)), "polylla_convexify")


def polylla_convex_chords(ctx: int, stream=None):
    """The half-edges the last convexify chose (device int32 tensor)."""
    import torch

    p = ctypes.c_void_p()
    n = ctypes.c_int32()
    _check(load_library().polylla_convex_chords(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(n),
                                                _stream_ptr(stream)), "polylla_convex_chords")
    if n.value == 0:
        return torch.empty(0, dtype=torch.int32, device="cuda")
    return _view(p.value, n.value, "<i4", torch.int32)


def polylla_lepp_terminal(ctx: int, n_triangles: int, with_length: bool = True, stream=None):
    """Lepp terminal seed (and path length) of every triangle, after a
    generate: device int32 tensors ``(terminal, length or None)``."""
    import torch

    term = torch.empty(n_triangles, dtype=torch.int32, device="cuda")
    length = torch.empty(n_triangles, dtype=torch.int32, device="cuda") if with_length else None
    _check(load_library().polylla_lepp_terminal(
        ctypes.c_void_p(ctx), ctypes.c_void_p(term.data_ptr()),
        ctypes.c_void_p(length.data_ptr()) if length is not None else None, _stream_ptr(stream)),
        "polylla_lepp_terminal")
    return term, length


def polylla_lepp_paths(ctx: int, tri, capacity: int, stream=None):
    """Lepp paths of the query triangles ``tri`` (device int32 tensor):
    ``(offsets [n+1], paths [capacity])`` device int32 tensors."""
    import torch

    n = tri.numel()
    offsets = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    paths = torch.empty(max(int(capacity), 1), dtype=torch.int32, device="cuda")
    _check(load_library().polylla_lepp_paths(
        ctypes.c_void_p(ctx), _dev_ptr(tri, torch.int32, n), int(n), ctypes.c_void_p(offsets.data_ptr()),
        ctypes.c_void_p(paths.data_ptr()), int(capacity), _stream_ptr(stream)), "polylla_lepp_paths")
    return offsets, paths


class HostRequest:
    """A mesh in host memory plus result buffers of the capacities a request
    needs (T, T+1, 3T, 3T, H, H); pinned unless ``pinned=False``."""

    def __init__(self, mesh, pinned: bool = True):
        import torch

        self.mesh = mesh
        T, H = int(mesh.n_triangles), int(mesh.n_halfedges)
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t.clone())
        self.inp = {k: pin(torch.from_numpy(getattr(mesh, k)).contiguous())
                    for k in ("coords", "origin", "twin", "next", "prev")}
        self.out = {"seeds": pin(torch.empty(T, dtype=torch.int32)),
                    "offsets": pin(torch.empty(T + 1, dtype=torch.int32)),
                    "he_list": pin(torch.empty(3 * T, dtype=torch.int32)),
                    "v_list": pin(torch.empty(3 * T, dtype=torch.int32)),
                    "next": pin(torch.empty(H, dtype=torch.int32)),
                    "prev": pin(torch.empty(H, dtype=torch.int32))}
        self.req = polylla_request(
            int(mesh.n_vertices), T, H,
            polylla_host_mesh(*(ctypes.c_void_p(self.inp[k].data_ptr())
                                for k in ("coords", "origin", "twin", "next", "prev"))),
            polylla_host_result(*(ctypes.c_void_p(self.out[k].data_ptr())
                                  for k in ("seeds", "offsets", "he_list", "v_list", "next", "prev")), 0, 0))

    def result(self, info: dict) -> dict:
        """Numpy copies of the outputs, trimmed to the request's P and N_F."""
        P, NF = info["n_polygons"], info["n_frontier"]
        return {"seeds": self.out["seeds"][:P].numpy().copy(), "offsets": self.out["offsets"][:P + 1].numpy().copy(),
                "he_list": self.out["he_list"][:NF].numpy().copy(), "v_list": self.out["v_list"][:NF].numpy().copy(),
                "next": self.out["next"].numpy().copy(), "prev": self.out["prev"].numpy().copy()}


def server_plan(memory_budget: int, n_slots: int = 3, max_batch_meshes: int = 0, max_rotation: int = 0,
                max_batch_triangles: int = 0, lane_triangles: int = 0) -> dict:
    """The slots a Server with these options would allocate (no GPU needed)."""
    opt = polylla_server_options(int(memory_budget), int(n_slots), int(max_batch_meshes), int(max_rotation),
                                 int(max_batch_triangles), int(lane_triangles))
    out = polylla_server_plan()
    _check(load_library().polylla_server_plan_slots(ctypes.byref(opt), ctypes.byref(out)), "polylla_server_plan_slots")
    return {k: getattr(out, k) for k, _ in polylla_server_plan._fields_}


def _info_dict(info: polylla_request_info) -> dict:
    return {k: getattr(info, k) for k, _ in polylla_request_info._fields_}


class Server:
    """The serving loop (``polylla_server_*``): continuous batching of host
    requests on the current device."""

    def __init__(self, memory_budget: int, n_slots: int = 3, max_batch_meshes: int = 0, max_rotation: int = 0,
                 max_batch_triangles: int = 0, lane_triangles: int = 0):
        lib = load_library()
        opt = polylla_server_options(int(memory_budget), int(n_slots), int(max_batch_meshes), int(max_rotation),
                                     int(max_batch_triangles), int(lane_triangles))
        h = ctypes.c_void_p()
        _check(lib.polylla_server_create(ctypes.byref(h), ctypes.byref(opt)), "polylla_server_create")
        self.h = h.value

    def submit(self, r: HostRequest) -> int:
        t = ctypes.c_int64()
        _check(load_library().polylla_server_submit(ctypes.c_void_p(self.h), ctypes.byref(r.req), ctypes.byref(t)),
               "polylla_server_submit")
        return t.value

    def wait(self, ticket: int) -> dict:
        info = polylla_request_info()
        load_library().polylla_server_wait(ctypes.c_void_p(self.h), int(ticket), ctypes.byref(info))
        return _info_dict(info)

    def replay(self, requests, arrival_s) -> tuple:
        """Open-loop replay (native): returns (status, latencies [s], infos)."""
        import numpy as np

        n = len(requests)
        arr = (polylla_request * n)(*[r.req for r in requests])
        at = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(n, dtype=np.float64)
        infos = (polylla_request_info * n)()
        rc = load_library().polylla_server_replay(
            ctypes.c_void_p(self.h), n, arr, at.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), infos)
        return rc, lat, [_info_dict(i) for i in infos]

    def stats(self) -> dict:
        st = polylla_server_stats()
        _check(load_library().polylla_server_get_stats(ctypes.c_void_p(self.h), ctypes.byref(st)),
               "polylla_server_get_stats")
        return {k: getattr(st, k) for k, _ in polylla_server_stats._fields_}

    def batch_log(self, capacity: int = 65536) -> list:
        """The most recent completed batches, oldest first (one dict each)."""
        recs = (polylla_batch_record * capacity)()
        n = ctypes.c_int32()
        tot = ctypes.c_int64()
        _check(load_library().polylla_server_get_batch_log(ctypes.c_void_p(self.h), recs, capacity, ctypes.byref(n),
                                                           ctypes.byref(tot)), "polylla_server_get_batch_log")
        return [{k: getattr(recs[i], k) for k, _ in polylla_batch_record._fields_} for i in range(n.value)]

    def close(self):
        if self.h:
            load_library().polylla_server_destroy(ctypes.c_void_p(self.h))
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Polylla:
    """Owns one context on a device mesh (convenience wrapper)."""

    def __init__(self, mesh: DeviceMesh, validate: bool = True, max_rotation: int = 0, stream=None):
        self.mesh = mesh
        self.ctx = polylla_create(mesh, validate=validate, max_rotation=max_rotation, stream=stream)

    def generate(self, stream=None):
        polylla_generate(self.ctx, stream)

    def polygons(self, stream=None) -> dict:
        return polylla_get_polygons(self.ctx, stream)

    def labels(self, stream=None) -> dict:
        return polylla_get_labels(self.ctx, self.mesh.n_triangles, stream)

    def convexify(self, stream=None) -> None:
        polylla_convexify(self.ctx, stream)

    def close(self):
        polylla_destroy(self.ctx)
        self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.ctx:
                self.close()
        except Exception:
            pass
