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
// new polygons.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ double cross_rn(double ax, double ay, double bx, double by) {
    return __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
}

// ===========================================================================
// k_convex_chords: one thread per interior half-edge; frontier ones test
// their corner and, when it is reflex, choose its chords (appended to the
// list; the frontier bits are set by the next kernel, so every thread here
// reads the frontier of the Polylla mesh).
// ===========================================================================
__global__ void __launch_bounds__(256) k_convex_chords(MeshView m, Work w, int32_t *list, int32_t *count,
                                                       int32_t cap) {
    const int32_t HI = 3 * m.T;
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < HI; e += gridDim.x * blockDim.x) {
        if (!((w.flags[tri_of(e)] >> loc_of(e)) & 1u)) continue;
        const int32_t x = m.next[e];
        const int32_t v = __ldg(m.origin + x);                 // origin(x) = target(e)
        const double2 pv = __ldg(m.xy + v);
        const double2 pa = __ldg(m.xy + __ldg(m.origin + e));  // origin(e)
        const double2 pw = __ldg(m.xy + __ldg(m.origin + nx_of(x)));  // target(x)
        double ux = __dsub_rn(pa.x, pv.x), uy = __dsub_rn(pa.y, pv.y);
        const double wx = __dsub_rn(pw.x, pv.x), wy = __dsub_rn(pw.y, pv.y);
        if (!(cross_rn(ux, uy, wx, wy) > 0.0)) continue;
        int32_t y = nx_of(e);
        int32_t steps = 0;
        while (cross_rn(ux, uy, wx, wy) > 0.0) {
            int32_t best = -1;
            double bx = 0.0, by = 0.0;
            while (y != x) {
                const double2 pd = __ldg(m.xy + __ldg(m.origin + nx_of(y)));  // target(y)
                const double dx = __dsub_rn(pd.x, pv.x), dy = __dsub_rn(pd.y, pv.y);
                if (!(cross_rn(ux, uy, dx, dy) <= 0.0)) break;
                best = y;
                bx = dx;
                by = dy;
                y = nx_of(__ldg(m.twin + y));                   // CW(y)
                if (++steps > w.max_rot) {
                    atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                    break;
                }
            }
            if (best < 0 || steps > w.max_rot) break;           // candidates ran out: left reflex
            const int32_t slot = atomicAdd(count, 1);
            if (slot < cap) list[slot] = best;
            else atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            ux = bx;
            uy = by;
        }
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

void launch_convex_chords(const MeshView &m, const Work &w, int32_t *list, int32_t *count, int32_t cap,
                          cudaStream_t s) {
    const int64_t want = (3 * (int64_t)m.T + 255) / 256;
    const int blocks = (int)(want < 16 * (int64_t)w.persistent_blocks ? want : 16 * (int64_t)w.persistent_blocks);
    k_convex_chords<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(m, w, list, count, cap);
}

void launch_convex_mark(const MeshView &m, const Work &w, const int32_t *list, const int32_t *count, int32_t cap,
                        cudaStream_t s) {
    k_convex_mark<<<w.persistent_blocks, 256, 0, s>>>(m, w, list, count, cap);
}

}  // namespace polylla
