"""The certified float32 filters of the kernels, restated in numpy and
searched for counterexamples on the CPU.

Two binary64 decisions of the method run first through a float32 filter on
the GPU, which answers only when its error bound proves the answer:

* the longest edge of a triangle (Algorithm 2 / 8, reading 2): the argmax
  of the squared lengths fl(fl(dx dx) + fl(dy dy)), dx = fl(xb - xa), all
  in binary64 without FMA; the filter must answer only when that argmax
  is unique and is its answer;
* the turn test of the convexification (reading 17): the sign of
  fl(fl(ux wy) - fl(uy wx)) with u = a - v, w = b - v in binary64; the
  filter must answer only with that sign, and never when it is zero.

The model below follows the filters' arithmetic (coordinates truncated to
float32 by bit manipulation, differences, products and sums in float32
rounded to nearest, the same bounds) and is checked against the binary64
definitions on adversarial inputs: lattice triangles with exact ties moved
by a few ulps, near-isosceles triangles, tiny triangles far from the
origin, magnitudes across the filter's range and its edges, nearly
collinear corners.  It is a restatement for testing, not the kernels' code;
the GPU parity tests compare the kernels themselves with the oracle on
near-tie meshes.
"""
import numpy as np

U = np.float32(2.0 ** -24)


def trunc_to_f32(v):
    """v (float64 array) truncated to float32 by bit manipulation: the sign,
    the exponent rebiased, the top 23 significand bits; bad where |v| lies
    outside [2^-126, 2^61) (zero included)."""
    bits = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint32)
    lo = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    mag = hi & np.uint32(0x7FFFFFFF)
    bad = (mag - np.uint32(897 << 20)) >= np.uint32((1084 - 897) << 20)
    f = ((hi << np.uint32(3)) | (lo >> np.uint32(29))) - np.uint32(384 << 23)
    f |= hi & np.uint32(0x80000000)
    return f.view(np.float32), bad


def fma32(a, b, c):
    """float32 fused multiply-add (the product is exact in float64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def edge32(ax, ay, bx, by):
    dx = bx - ax
    dy = by - ay
    sx = np.abs(ax) + np.abs(bx)
    sy = np.abs(ay) + np.abs(by)
    d = dx * dx + dy * dy
    m1 = fma32(sx, np.abs(dx), sy * np.abs(dy))
    m2 = fma32(sx, sx, sy * sy)
    c1, c2, c3 = np.float32(6.1) * U, np.float32(9.1) * U * U, np.float32(4.5) * U
    b = fma32(np.full_like(m1, c1), m1,
              fma32(np.full_like(m2, c2), m2, fma32(np.full_like(d, c3), d, np.full_like(d, np.float32(3.0e-36)))))
    return d, b


@np.errstate(over="ignore", invalid="ignore")
def longest_filter(p):
    """p [n, 3, 2] float64 -> (sure [n], k [n]) of the float32 filter."""
    t, bad = trunc_to_f32(p.reshape(-1))
    t = t.reshape(p.shape)
    bad = bad.reshape(p.shape).any(axis=(1, 2))
    g = [edge32(t[:, i, 0], t[:, i, 1], t[:, (i + 1) % 3, 0], t[:, (i + 1) % 3, 1]) for i in range(3)]
    d = np.stack([x[0] for x in g], 1)
    b = np.stack([x[1] for x in g], 1)
    k = np.where((d[:, 0] >= d[:, 1]) & (d[:, 0] >= d[:, 2]), 0, np.where(d[:, 1] >= d[:, 2], 1, 2))
    n = np.arange(len(p))
    lo = d[n, k] - b[n, k]
    sure = ~bad
    for j in range(1, 3):
        o = (k + j) % 3
        sure &= lo > d[n, o] + b[n, o]
    return sure, k


def longest_f64(p):
    """Binary64 squared lengths of the three edges (every operation rounded
    on its own)."""
    out = []
    for i in range(3):
        dx = p[:, (i + 1) % 3, 0] - p[:, i, 0]
        dy = p[:, (i + 1) % 3, 1] - p[:, i, 1]
        out.append(dx * dx + dy * dy)
    return np.stack(out, 1)


@np.errstate(over="ignore", invalid="ignore")
def turn_filter(a, b, v):
    """Sign (+1, -1; 0 = undecided) from the float32 filter of the turn test
    (an overflow to inf or nan leaves it undecided, as on the GPU)."""
    (ax, bad_a1), (ay, bad_a2) = trunc_to_f32(a[:, 0]), trunc_to_f32(a[:, 1])
    (bx, bad_b1), (by, bad_b2) = trunc_to_f32(b[:, 0]), trunc_to_f32(b[:, 1])
    (vx, bad_v1), (vy, bad_v2) = trunc_to_f32(v[:, 0]), trunc_to_f32(v[:, 1])
    bad = bad_a1 | bad_a2 | bad_b1 | bad_b2 | bad_v1 | bad_v2
    ux, uy, wx, wy = ax - vx, ay - vy, bx - vx, by - vy
    k = np.float32(3.001) * U
    e_ux, e_uy = k * (np.abs(ax) + np.abs(vx)), k * (np.abs(ay) + np.abs(vy))
    e_wx, e_wy = k * (np.abs(bx) + np.abs(vx)), k * (np.abs(by) + np.abs(vy))
    p1, p2 = ux * wy, uy * wx
    c = p1 - p2
    B = e_ux * np.abs(wy) + np.abs(ux) * e_wy + e_ux * e_wy + U * np.abs(p1)
    B = B + (e_uy * np.abs(wx) + np.abs(uy) * e_wx + e_uy * e_wx + U * np.abs(p2))
    B = np.float32(1.01) * (B + U * np.abs(c)) + np.float32(7.5e-37)
    s = np.where(c > B, 1, np.where(c < -B, -1, 0))
    return np.where(bad, 0, s)


def turn_f64(a, b, v):
    ux, uy = a[:, 0] - v[:, 0], a[:, 1] - v[:, 1]
    wx, wy = b[:, 0] - v[:, 0], b[:, 1] - v[:, 1]
    return np.sign(ux * wy - uy * wx)


def _ulps(rng, x, k):
    """x moved by up to k ulps (float64), elementwise."""
    return x + rng.integers(-k, k + 1, size=x.shape) * np.spacing(x)


def _triangle_sets(rng, n):
    sets = {}
    # exact length ties (integer lattice, isosceles and right triangles),
    # scaled and shifted, then moved by a few ulps
    base = rng.integers(-40, 41, size=(n, 3, 2)).astype(np.float64)
    apex = np.stack([np.zeros(n), np.zeros(n)], 1)
    a = rng.integers(1, 30, size=n).astype(np.float64)
    h = rng.integers(1, 30, size=n).astype(np.float64)
    iso = np.stack([np.stack([-a, np.zeros(n)], 1), np.stack([a, np.zeros(n)], 1), np.stack([apex[:, 0], h], 1)], 1)
    for name, tri in (("lattice", base), ("isosceles", iso)):
        for scale, shift in ((1.0, 0.0), (2.0 ** -20, 0.5), (2.0 ** -12, 1000.0), (2.0 ** 10, -3.0e5)):
            q = tri * scale + shift
            sets[f"{name}_{scale:g}_{shift:g}"] = q
            sets[f"{name}_{scale:g}_{shift:g}_ulps"] = _ulps(rng, q, 6)
    # tiny jittered grid cells far from the origin (the perturbed grid's shape)
    cell = 2.0 ** -12
    o = rng.random((n, 1, 2)) * 0.9 + 0.05
    quad = np.array([[0, 0], [1, 0], [1, 1]], np.float64)[None] * cell
    sets["grid_cell"] = o + quad + (rng.random((n, 3, 2)) - 0.5) * 0.6 * cell
    # magnitudes across (and past) the filter's range, zeros included
    e = rng.integers(-140, 70, size=(n, 1, 1)).astype(np.float64)
    sets["magnitudes"] = (rng.random((n, 3, 2)) - 0.5) * 2.0 ** e
    z = rng.random((n, 3, 2))
    z[rng.random((n, 3, 2)) < 0.2] = 0.0
    sets["zeros"] = z
    return sets


def test_longest_edge_filter_never_contradicts_binary64():
    rng = np.random.default_rng(20240321)
    decided = total = 0
    for name, p in _triangle_sets(rng, 200_000).items():
        sure, k = longest_filter(p)
        d = longest_f64(p)
        n = np.arange(len(p))
        dk = d[n, k]
        for j in range(1, 3):
            other = d[n, (k + j) % 3]
            bad = sure & ~(dk > other)
            assert not bad.any(), f"{name}: filter sure but binary64 disagrees at {np.flatnonzero(bad)[:5]}"
        decided += int(sure.sum())
        total += len(p)
    assert decided > 0.5 * total


def test_longest_edge_filter_decides_ordinary_triangles():
    """On jittered grid cells and random triangles the filter answers almost
    always (the binary64 path is the exception)."""
    rng = np.random.default_rng(7)
    sets = _triangle_sets(rng, 100_000)
    for name in ("grid_cell",):
        sure, _ = longest_filter(sets[name])
        assert sure.mean() > 0.99, (name, sure.mean())
    p = rng.random((100_000, 3, 2))
    sure, k = longest_filter(p)
    assert sure.mean() > 0.999


def test_turn_filter_never_contradicts_binary64():
    rng = np.random.default_rng(99)
    n = 300_000
    decided = 0
    cases = {}
    v = rng.random((n, 2)) * 0.9 + 0.05
    d1 = rng.random((n, 2)) - 0.5
    # b on the line through v and a, moved by a few ulps: turns near zero
    t = rng.random((n, 1)) * 4 - 2
    a = v + d1 * 2.0 ** -10
    b = v + t * (a - v)
    cases["collinear"] = (a, _ulps(rng, b, 4), v)
    # exact lattice collinearity and right angles, shifted and scaled
    ia = rng.integers(-20, 21, size=(n, 2)).astype(np.float64)
    m = rng.integers(-3, 4, size=(n, 1)).astype(np.float64)
    for scale, shift in ((1.0, 0.0), (2.0 ** -16, 0.25), (2.0 ** 8, 5.0e4)):
        cases[f"lattice_{scale:g}"] = (ia * scale + shift, m * ia * scale + shift, np.full((n, 2), shift))
        cases[f"lattice_{scale:g}_ulps"] = (_ulps(rng, ia * scale + shift, 3), _ulps(rng, m * ia * scale + shift, 3),
                                            _ulps(rng, np.full((n, 2), shift), 3))
    cases["random"] = (rng.random((n, 2)), rng.random((n, 2)), rng.random((n, 2)))
    e = rng.integers(-140, 70, size=(n, 1)).astype(np.float64)
    cases["magnitudes"] = ((rng.random((n, 2)) - 0.5) * 2.0 ** e, (rng.random((n, 2)) - 0.5) * 2.0 ** e,
                           (rng.random((n, 2)) - 0.5) * 2.0 ** e)
    for name, (a, b, v) in cases.items():
        s = turn_filter(a, b, v)
        ref = turn_f64(a, b, v)
        wrong = (s != 0) & (s != ref)
        assert not wrong.any(), f"{name}: filter sign against binary64 at {np.flatnonzero(wrong)[:5]}"
        decided += int((s != 0).sum())
    assert decided > 0
    s = turn_filter(cases["random"][0], cases["random"][1], cases["random"][2])
    assert (s != 0).mean() > 0.999


def test_truncation_model():
    """The truncation keeps the top 23 significand bits: |x - x^| <= 2^-23
    |x^|, |x^| <= |x|, exact on float32 values, bad outside [2^-126, 2^61)."""
    rng = np.random.default_rng(3)
    sign = np.where(rng.random(100_000) < 0.5, -1.0, 1.0)
    x = sign * (1.0 + rng.random(100_000)) * 2.0 ** rng.integers(-126, 61, size=100_000)
    t, bad = trunc_to_f32(x)
    assert not bad.any()
    t64 = t.astype(np.float64)
    assert np.all(np.abs(t64) <= np.abs(x))
    assert np.all(np.abs(x - t64) <= 2.0 ** -23 * np.abs(t64))
    f = (rng.random(1000) + 0.5).astype(np.float32).astype(np.float64)
    assert np.array_equal(trunc_to_f32(f)[0].astype(np.float64), f)
    edge = np.array([0.0, -0.0, 2.0 ** -127, 2.0 ** 61, -2.0 ** 62, 2.0 ** -126, 2.0 ** 61 - 2.0 ** 9, -2.0 ** 60])
    assert trunc_to_f32(edge)[1].tolist() == [True, True, True, True, True, False, False, False]
