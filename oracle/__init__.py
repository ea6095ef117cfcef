"""CPU oracle for the Polylla method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2403_14723_gb300`` never imports it, and this package imports
nothing from the library: it takes plain arrays.

The arithmetic lives in ``polylla_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so every binary64 operation is rounded on its own); this
file builds it with gcc and marshals numpy arrays through ctypes.

Parity pins (tests that tie the oracle to something other than itself) are
in ``tests/test_oracle_pins.py``; every function here is pinned there.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polylla_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lib = None

STAT_NAMES = (
    "seeds", "tips", "polygons", "frontier1", "nonsimple", "completion",
    "repair_polygons", "traversal_polygons", "distinct_chords", "frontier0",
)
TIME_NAMES = ("longest_edge", "frontier", "seeds", "traversal", "repair", "output")

ERRORS = {-1: "out of memory", -2: "non-terminating rotation or walk", -3: "output links are not cycles"}


def _so_path() -> str:
    with open(_SRC, "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()[:12]
    import platform

    return os.path.join(_BUILD, f"liboracle_{platform.machine()}_{digest}.so")


def build() -> str:
    """Compile the oracle with gcc (idempotent); return the shared object path."""
    so = _so_path()
    if not os.path.exists(so):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    f64p = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_polylla.restype = ctypes.c_int
    lib.oracle_polylla.argtypes = [
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, f64p,
        i32p, i32p, i32p, i32p,
        u8p, u8p, u8p,
        i32p, i32p, i32p,
        i32p, i32p,
        i32p, i32p, i32p, i32p,
        i64p, f64p,
    ]
    lib.oracle_lepp.restype = ctypes.c_int
    lib.oracle_lepp.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_lepp_path.restype = ctypes.c_int32
    lib.oracle_lepp_path.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8),
                                     ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    lib.oracle_convexify.restype = ctypes.c_int
    lib.oracle_convexify.argtypes = [
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, f64p,
        i32p, i32p, i32p, i32p,
        u8p, i32p,
        u8p, i32p, i32p,
        i32p, i32p,
        i32p, i32p, i32p, i32p,
        i64p,
    ]
    lib.oracle_stats_count.restype = ctypes.c_int
    assert lib.oracle_stats_count() == len(STAT_NAMES)
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(so_path: str):
    """Bind another build of the oracle source (the mutation tests compile
    deliberately broken copies to show that the pins catch them)."""
    return _bind(ctypes.CDLL(so_path))


@dataclass
class OracleResult:
    """Everything the oracle computes for one mesh (host numpy arrays)."""

    longest: np.ndarray      # [H] uint8, 1 on the longest half-edge of each triangle
    frontier0: np.ndarray    # [H] uint8, frontier labels of the label phase
    frontier1: np.ndarray    # [H] uint8, after the repair chords
    seed_list: np.ndarray    # seeds of Algorithm 4, ascending
    tip_out: np.ndarray      # per repaired tip: the F0 half-edge leaving it
    chord: np.ndarray        # per repaired tip: the chord half-edge leaving it
    next_out: np.ndarray     # [H] int32
    prev_out: np.ndarray     # [H] int32
    seeds: np.ndarray        # [P] smallest half-edge of each polygon, ascending
    offsets: np.ndarray      # [P+1]
    he_list: np.ndarray      # [N_F] half-edges of each polygon from its seed
    v_list: np.ndarray       # [N_F] origin of each listed half-edge
    stats: dict = field(default_factory=dict)
    times: dict = field(default_factory=dict)

    @property
    def n_polygons(self) -> int:
        return int(self.seeds.shape[0])


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def run(coords, origin, twin, next, prev, n_triangles: int, lib=None) -> OracleResult:
    """Run the sequential method on one mesh given as plain arrays.

    ``coords`` [V, 2] float64; ``origin/twin/next/prev`` [H] int32;
    interior half-edges are ``[0, 3*n_triangles)``.
    """
    lib = lib if lib is not None else _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    origin = np.ascontiguousarray(origin, dtype=np.int32)
    twin = np.ascontiguousarray(twin, dtype=np.int32)
    nxt = np.ascontiguousarray(next, dtype=np.int32)
    prv = np.ascontiguousarray(prev, dtype=np.int32)
    V = coords.shape[0]
    H = origin.shape[0]
    T = int(n_triangles)
    HI = 3 * T
    longest = np.zeros(H, np.uint8)
    f0 = np.zeros(H, np.uint8)
    f1 = np.zeros(H, np.uint8)
    seed_list = np.zeros(max(H, 1), np.int32)
    tip_out = np.zeros(max(V, 1), np.int32)
    chord = np.zeros(max(V, 1), np.int32)
    next_out = np.zeros(H, np.int32)
    prev_out = np.zeros(H, np.int32)
    seeds = np.zeros(max(T, 1), np.int32)
    offsets = np.zeros(T + 1, np.int32)
    he_list = np.zeros(max(HI, 1), np.int32)
    v_list = np.zeros(max(HI, 1), np.int32)
    stats = np.zeros(len(STAT_NAMES), np.int64)
    times = np.zeros(len(TIME_NAMES), np.float64)
    rc = lib.oracle_polylla(
        V, T, H, _ptr(coords, ctypes.c_double),
        _ptr(origin, ctypes.c_int32), _ptr(twin, ctypes.c_int32),
        _ptr(nxt, ctypes.c_int32), _ptr(prv, ctypes.c_int32),
        _ptr(longest, ctypes.c_uint8), _ptr(f0, ctypes.c_uint8), _ptr(f1, ctypes.c_uint8),
        _ptr(seed_list, ctypes.c_int32), _ptr(tip_out, ctypes.c_int32), _ptr(chord, ctypes.c_int32),
        _ptr(next_out, ctypes.c_int32), _ptr(prev_out, ctypes.c_int32),
        _ptr(seeds, ctypes.c_int32), _ptr(offsets, ctypes.c_int32),
        _ptr(he_list, ctypes.c_int32), _ptr(v_list, ctypes.c_int32),
        _ptr(stats, ctypes.c_int64), _ptr(times, ctypes.c_double),
    )
    if rc != 0:
        raise RuntimeError(f"oracle failed: {ERRORS.get(rc, rc)}")
    st = {n: int(v) for n, v in zip(STAT_NAMES, stats)}
    P = st["polygons"]
    NF = st["frontier1"]
    ntips = st["tips"]
    return OracleResult(
        longest=longest, frontier0=f0, frontier1=f1,
        seed_list=seed_list[: st["seeds"]].copy(),
        tip_out=tip_out[:ntips].copy(), chord=chord[:ntips].copy(),
        next_out=next_out, prev_out=prev_out,
        seeds=seeds[:P].copy(), offsets=offsets[: P + 1].copy(),
        he_list=he_list[:NF].copy(), v_list=v_list[:NF].copy(),
        stats=st, times={n: float(v) for n, v in zip(TIME_NAMES, times)},
    )


def lepp(mesh, longest: np.ndarray, lib=None):
    """Lepp of every triangle (Definition 1) from the label phase's longest
    edges: ``(terminal [T], length [T])``, terminal = the seed half-edge of
    the terminal edge the path ends on, length = triangles in the path."""
    lib = lib if lib is not None else _load()
    T = int(mesh.n_triangles)
    twin = np.ascontiguousarray(mesh.twin, dtype=np.int32)
    lg = np.ascontiguousarray(longest, dtype=np.uint8)
    term = np.zeros(max(T, 1), np.int32)
    length = np.zeros(max(T, 1), np.int32)
    rc = lib.oracle_lepp(T, int(twin.shape[0]), _ptr(twin, ctypes.c_int32), _ptr(lg, ctypes.c_uint8),
                         _ptr(term, ctypes.c_int32), _ptr(length, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError(f"oracle failed: {ERRORS.get(rc, rc)}")
    return term[:T].copy(), length[:T].copy()


def lepp_path(mesh, longest: np.ndarray, t0: int, lib=None) -> np.ndarray:
    """The triangles of Lepp(t0), in order."""
    lib = lib if lib is not None else _load()
    twin = np.ascontiguousarray(mesh.twin, dtype=np.int32)
    lg = np.ascontiguousarray(longest, dtype=np.uint8)
    cap = int(mesh.n_triangles) + 1
    path = np.zeros(cap, np.int32)
    n = lib.oracle_lepp_path(int(mesh.n_triangles), _ptr(twin, ctypes.c_int32), _ptr(lg, ctypes.c_uint8), int(t0),
                             _ptr(path, ctypes.c_int32), cap)
    if n < 0:
        raise RuntimeError("oracle Lepp path longer than the mesh")
    return path[:n].copy()


def run_mesh(mesh, lib=None) -> OracleResult:
    """Convenience: run on any object with ``coords, origin, twin, next, prev,
    n_triangles`` attributes."""
    return run(mesh.coords, mesh.origin, mesh.twin, mesh.next, mesh.prev, mesh.n_triangles, lib=lib)


@dataclass
class ConvexResult:
    """The convexified mesh (reading R9 of the oracle source): every
    polygon of ``base`` split at its reflex corners by chords that are
    existing interior edges of the triangulation."""

    frontier2: np.ndarray   # [H] uint8, F1 plus both halves of every chord
    next_out: np.ndarray    # [H] int32, the relink under F2
    prev_out: np.ndarray    # [H] int32
    chords: np.ndarray      # chosen half-edges, each leaving its corner's vertex
    seeds: np.ndarray       # [P2]
    offsets: np.ndarray     # [P2+1]
    he_list: np.ndarray     # [N_F2]
    v_list: np.ndarray      # [N_F2]
    stats: dict = field(default_factory=dict)

    @property
    def n_polygons(self) -> int:
        return int(self.seeds.shape[0])


CONVEX_STAT_NAMES = ("polygons", "frontier", "reflex_corners", "left_reflex", "distinct_chords")


def convexify(mesh, base: OracleResult, lib=None) -> ConvexResult:
    """Convexify the Polylla mesh ``base`` (the result of ``run_mesh`` on
    ``mesh``): chords at every reflex corner, relink, canonical CSR."""
    lib = lib if lib is not None else _load()
    coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    origin = np.ascontiguousarray(mesh.origin, dtype=np.int32)
    twin = np.ascontiguousarray(mesh.twin, dtype=np.int32)
    nxt = np.ascontiguousarray(mesh.next, dtype=np.int32)
    prv = np.ascontiguousarray(mesh.prev, dtype=np.int32)
    V, H, T = coords.shape[0], origin.shape[0], int(mesh.n_triangles)
    HI = 3 * T
    f1 = np.ascontiguousarray(base.frontier1, dtype=np.uint8)
    n1 = np.ascontiguousarray(base.next_out, dtype=np.int32)
    f2 = np.zeros(H, np.uint8)
    n2 = np.zeros(H, np.int32)
    p2 = np.zeros(H, np.int32)
    chords = np.zeros(max(HI, 1), np.int32)
    n_chords = np.zeros(1, np.int32)
    seeds = np.zeros(max(T, 1), np.int32)
    offsets = np.zeros(T + 1, np.int32)
    he_list = np.zeros(max(HI, 1), np.int32)
    v_list = np.zeros(max(HI, 1), np.int32)
    stats = np.zeros(len(CONVEX_STAT_NAMES), np.int64)
    rc = lib.oracle_convexify(
        V, T, H, _ptr(coords, ctypes.c_double),
        _ptr(origin, ctypes.c_int32), _ptr(twin, ctypes.c_int32), _ptr(nxt, ctypes.c_int32), _ptr(prv, ctypes.c_int32),
        _ptr(f1, ctypes.c_uint8), _ptr(n1, ctypes.c_int32),
        _ptr(f2, ctypes.c_uint8), _ptr(n2, ctypes.c_int32), _ptr(p2, ctypes.c_int32),
        _ptr(chords, ctypes.c_int32), _ptr(n_chords, ctypes.c_int32),
        _ptr(seeds, ctypes.c_int32), _ptr(offsets, ctypes.c_int32),
        _ptr(he_list, ctypes.c_int32), _ptr(v_list, ctypes.c_int32),
        _ptr(stats, ctypes.c_int64),
    )
    if rc != 0:
        raise RuntimeError(f"oracle failed: {ERRORS.get(rc, rc)}")
    st = {n: int(v) for n, v in zip(CONVEX_STAT_NAMES, stats)}
    P, NF = st["polygons"], st["frontier"]
    return ConvexResult(frontier2=f2, next_out=n2, prev_out=p2, chords=chords[: int(n_chords[0])].copy(),
                        seeds=seeds[:P].copy(), offsets=offsets[: P + 1].copy(),
                        he_list=he_list[:NF].copy(), v_list=v_list[:NF].copy(), stats=st)
