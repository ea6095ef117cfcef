// Convexification of the Polylla mesh (post-processing).  Section 4.2 keeps
// every half-edge of the triangulation, relinking instead of deleting, so
// that a later step can turn non-convex polygons into convex ones; the
// paper gives no method.  This one splits every reflex corner with the
// fewest edges of the triangulation itself:
//   - the corner of a polygon at a frontier half-edge e is (e, x = next[e])
//     at v = target(e); directions leave v, dir(h) = target(h) - v, and the
//     corner's first side is twin(e), dir = origin(e) - v;
//   - cross(a, b) = a.x b.y - a.y b.x, every operation in binary64 rounded
//     to nearest on its own (no FMA); b lies within a half turn clockwise of
//     a iff cross(a, b) <= 0; the corner is reflex iff cross(dir twin e,
//     dir x) > 0;
//   - the corner's interior half-edges, clockwise: y1 = the triangle's next
//     of e, then y = CW(y) = next(twin y), up to x (the relink's rotation);
//     from cur = twin(e) the last of them within a half turn of cur becomes
//     a chord and the new cur, until x is within a half turn of cur.
// Both halves of every chord join the frontier; the links around the chord
// ends are redone exactly as the repair's, and the output stage lists the
// new polygons.  Every turn test first tries a certified float32 filter
// (cross_sign) and computes the binary64 expression only when the filter
// cannot decide, so the decisions are those of binary64 throughout.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ double cross_rn(double ax, double ay, double bx, double by) {
    return __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
}

// A vertex: its id and the float32 truncations of its coordinates (the
// binary64 path reloads the coordinates themselves).
struct Pt {
    float x, y;
    uint32_t bad;  // a coordinate the filter cannot take
    int32_t v;
};

__device__ __forceinline__ Pt load_pt(const double2 *__restrict__ xy, int32_t v) {
    Pt r;
    const double2 p = __ldg(xy + v);
    r.bad = 0;
    r.x = trunc_to_f32(p.x, r.bad);
    r.y = trunc_to_f32(p.y, r.bad);
    r.v = v;
    return r;
}

// Sign (+1, 0, -1) of the binary64 expression cross(a - v, b - v) =
// fl(fl(ux wy) - fl(uy wx)), ux = fl(a.x - v.x), ... (every operation
// rounded to nearest, no FMA): the turn test of the convexification.
//
// Float32 filter (u = 2^-24).  Truncated coordinates satisfy |x - x^| <=
// 2u|x^|, so a float32 difference d^ = fl32(a^ - v^) is within
// e = 3uS of the exact a - v, S = |a^| + |v^|.  For the products,
// |ux wy - ux^ wy^| <= e_ux|wy^| + |ux^|e_wy + e_ux e_wy, plus u|p^| for the
// rounding of p^ = fl32(ux^ wy^); the final difference adds u|c^|.  So the
// exact cross c lies within
//   B = sum over both products (e1|f2| + |f1|e2 + e1 e2 + u|p|) + u|c^|
// of c^.  The binary64 value is within 2^-50 (|p1| + |p2|) of c, far below
// the 1 % margin added to B (with an absolute 2^-120 for float32 underflow);
// so |c^| > B gives the binary64 sign, and a nonzero one.  Otherwise, or
// for coordinates the truncation cannot take, the binary64 expression
// decides, computed exactly as the oracle does.
__device__ int cross_sign(const double2 *__restrict__ xy, const Pt &a, const Pt &b, const Pt &v) {
    if (!(a.bad | b.bad | v.bad)) {
        const float u = 5.9604644775390625e-08f;  // 2^-24
        const float ux = __fsub_rn(a.x, v.x), uy = __fsub_rn(a.y, v.y);
        const float wx = __fsub_rn(b.x, v.x), wy = __fsub_rn(b.y, v.y);
        const float e_ux = 3.001f * u * (fabsf(a.x) + fabsf(v.x)), e_uy = 3.001f * u * (fabsf(a.y) + fabsf(v.y));
        const float e_wx = 3.001f * u * (fabsf(b.x) + fabsf(v.x)), e_wy = 3.001f * u * (fabsf(b.y) + fabsf(v.y));
        const float p1 = __fmul_rn(ux, wy), p2 = __fmul_rn(uy, wx);
        const float c = __fsub_rn(p1, p2);
        float B = e_ux * fabsf(wy) + fabsf(ux) * e_wy + e_ux * e_wy + u * fabsf(p1);
        B += e_uy * fabsf(wx) + fabsf(uy) * e_wx + e_uy * e_wx + u * fabsf(p2);
        B = 1.01f * (B + u * fabsf(c)) + 7.5e-37f;
        if (c > B) return 1;
        if (c < -B) return -1;
    }
    const double2 pa = __ldg(xy + a.v), pb = __ldg(xy + b.v), pv = __ldg(xy + v.v);
    const double c = cross_rn(__dsub_rn(pa.x, pv.x), __dsub_rn(pa.y, pv.y), __dsub_rn(pb.x, pv.x),
                              __dsub_rn(pb.y, pv.y));
    return c > 0.0 ? 1 : (c < 0.0 ? -1 : 0);
}

// A slot at the end of a list shared by the whole grid: the lanes of a warp
// that reach this call together take consecutive slots with one atomic, so
// the list's counter sees one atomic per warp and call instead of one per
// entry (a million same-address atomics serialise in L2).  List order is
// free: every consumer of these lists treats them as sets.
__device__ __forceinline__ int32_t append_slot(int32_t *count) {
    const uint32_t mask = __activemask();
    const int lane = (int)(threadIdx.x & 31u);
    const int leader = __ffs(mask) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// ===========================================================================
// The corners: for a frontier half-edge e = 3t + k, v = target(e) is the
// triangle's vertex k + 1, origin(e) its vertex k, and the corner's other
// side is x = next[e].  k_convex_reflex tests every corner (one thread per
// triangle, its three vertices loaded once, the corners' chains issued
// together); corner_chords chooses a reflex corner's chords (appended to the
// list; the frontier bits are set by the next kernel, so every thread reads
// the frontier of the Polylla mesh).
// ===========================================================================
__device__ void corner_chords(const MeshView &m, const Work &w, int32_t e, int32_t x, const Pt &pv, Pt cur,
                              const Pt &pw, int32_t *list, int32_t *count, int32_t cap) {
    int32_t y = nx_of(e);
    int32_t steps = 0;
    while (cross_sign(m.xy, cur, pw, pv) > 0) {
        int32_t best = -1;
        Pt bp = cur;
        while (y != x) {
            const Pt pd = load_pt(m.xy, __ldg(m.origin + nx_of(y)));  // target(y)
            if (cross_sign(m.xy, cur, pd, pv) > 0) break;             // beyond a half turn
            best = y;
            bp = pd;
            y = nx_of(__ldg(m.twin + y));                             // CW(y)
            if (++steps > w.max_rot) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                break;
            }
        }
        if (best < 0 || steps > w.max_rot) return;                    // candidates ran out: left reflex
        const int32_t slot = append_slot(count);
        if (slot < cap) list[slot] = best;
        else atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        cur = bp;
    }
}

// k_convex_reflex: one thread per triangle; the reflex corners of its
// frontier half-edges go to a list, so that the chord search (a chain of
// dependent loads) runs one reflex corner per thread in k_convex_chords
// instead of holding up a warp of mostly convex corners.
__global__ void __launch_bounds__(256, 4) k_convex_reflex(MeshView m, Work w, int32_t *reflex, int32_t *n_reflex,
                                                          int32_t cap) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m.T; t += gridDim.x * blockDim.x) {
        const uint32_t f = w.flags[t] & 7u;
        if (!f) continue;
        const int32_t e0 = 3 * t;
        // a corner whose successor is the next half-edge of its own triangle
        // is a triangle's angle, less than a half turn: only corners whose
        // link crossed an edge can be reflex
        int32_t x[3];
        uint32_t test = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (!((f >> k) & 1u)) continue;
            x[k] = m.next[e0 + k];
            if (x[k] != e0 + (k == 2 ? 0 : k + 1)) test |= 1u << k;
        }
        if (!test) continue;
        Pt p[3];
#pragma unroll
        for (int k = 0; k < 3; k++) p[k] = load_pt(m.xy, __ldg(m.origin + e0 + k));
        Pt pw[3];
#pragma unroll
        for (int k = 0; k < 3; k++)
            if ((test >> k) & 1u) pw[k] = load_pt(m.xy, __ldg(m.origin + nx_of(x[k])));  // target(x)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (!((test >> k) & 1u)) continue;
            if (cross_sign(m.xy, p[k], pw[k], p[k == 2 ? 0 : k + 1]) > 0) {  // v = target(e): vertex k + 1
                const int32_t slot = append_slot(n_reflex);
                if (slot < cap) reflex[slot] = e0 + k;
                else atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            }
        }
    }
}

// k_convex_chords: one thread per reflex corner e: its chords
__global__ void __launch_bounds__(256) k_convex_chords(MeshView m, Work w, const int32_t *reflex,
                                                       const int32_t *n_reflex, int32_t cap_reflex, int32_t *list,
                                                       int32_t *count, int32_t cap) {
    int32_t n = *n_reflex;
    if (n > cap_reflex) n = cap_reflex;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t e = reflex[i];
        const int32_t x = m.next[e];
        const Pt pv = load_pt(m.xy, __ldg(m.origin + nx_of(e)));   // target(e)
        const Pt pa = load_pt(m.xy, __ldg(m.origin + e));          // origin(e)
        const Pt pw = load_pt(m.xy, __ldg(m.origin + nx_of(x)));   // target(x)
        corner_chords(m, w, e, x, pv, pa, pw, list, count, cap);
    }
}

// both halves of every listed chord join the frontier (F bits of flags)
__global__ void __launch_bounds__(256) k_convex_mark(MeshView m, Work w, const int32_t *list, const int32_t *count,
                                                     int32_t cap) {
    int32_t n = *count;
    if (n > cap) n = cap;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += gridDim.x * blockDim.x) {
        const int32_t c0 = list[i >> 1];
        const int32_t c = (i & 1) ? __ldg(m.twin + c0) : c0;
        const int32_t t = tri_of(c);
        unsigned int *word = reinterpret_cast<unsigned int *>(w.flags) + (t >> 2);
        atomicOr(word, 1u << (8 * (t & 3) + loc_of(c)));
    }
}

void launch_convex_chords(const MeshView &m, const Work &w, int32_t *reflex, int32_t *n_reflex, int32_t *list,
                          int32_t *count, int32_t cap, cudaStream_t s) {
    const int64_t want = ((int64_t)m.T + 255) / 256;
    const int blocks = (int)(want < 16 * (int64_t)w.persistent_blocks ? want : 16 * (int64_t)w.persistent_blocks);
    k_convex_reflex<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(m, w, reflex, n_reflex, cap);
    k_convex_chords<<<8 * w.persistent_blocks, 256, 0, s>>>(m, w, reflex, n_reflex, cap, list, count, cap);
}

void launch_convex_mark(const MeshView &m, const Work &w, const int32_t *list, const int32_t *count, int32_t cap,
                        cudaStream_t s) {
    k_convex_mark<<<w.persistent_blocks, 256, 0, s>>>(m, w, list, count, cap);
}

}  // namespace polylla
