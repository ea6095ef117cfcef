// Repair-phase kernels (stage 5a): chords from barrier tips and the relink
// around their endpoints.  Both run over the (short) tip list with a
// persistent grid-stride loop, so a mesh without tips costs two tiny
// launches.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ bool f1_of(const uint8_t *__restrict__ flags, int32_t e, int32_t HI) {
    if (e >= HI) return true;  // border half-edges are always frontier
    return (flags[tri_of(e)] >> loc_of(e)) & 1u;
}

__device__ __forceinline__ void set_flag_bit(uint8_t *flags, int32_t e, int shift) {
    const int32_t t = tri_of(e);
    unsigned int *word = reinterpret_cast<unsigned int *>(flags) + (t >> 2);
    atomicOr(word, 1u << (8 * (t & 3) + shift + loc_of(e)));
}
// F1 bit (bits 0-2) and walk-start mark (bits 3-5) of half-edge e
__device__ __forceinline__ void set_f1(uint8_t *flags, int32_t e) { set_flag_bit(flags, e, 0); }
__device__ __forceinline__ void set_start(uint8_t *flags, int32_t e) { set_flag_bit(flags, e, 3); }

// ===========================================================================
// Chords (Algorithm 6 first part / Algorithm 11).  For the tip b left by
// the unique stage-2 frontier half-edge f: count the degree d by rotating
// clockwise (CW(y) = next(twin y)) until f comes back, then the chord is
// m = CW^r(f) with r = floor((d-1)/2) + 1 (the inclusive loop "for 0 to
// (degree-1)/2").  Both halves of m join the frontier (F1).  Tips come only
// from the stage-2 labels, so the result does not depend on the order in
// which tips are processed.
// ===========================================================================
__global__ void __launch_bounds__(256) k_chords(MeshView m, Work w) {
    const int32_t HI = 3 * m.T;
    int32_t n = w.ctrl->n_tips;
    if (n > w.tip_cap) n = w.tip_cap;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t f = w.tips[i];
        int32_t y = f, d = 0;
        bool ok = true;
        do {
            const int32_t ty = __ldg(m.twin + y);
            if (ty >= HI || ++d > w.max_rot) { ok = false; break; }
            y = nx_of(ty);
        } while (y != f);
        if (!ok) {
            atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
            w.chords[i] = -1;
            continue;
        }
        const int32_t r = (d - 1) / 2 + 1;
        y = f;
        for (int32_t s = 0; s < r; s++) y = nx_of(__ldg(m.twin + y));
        w.chords[i] = y;
        set_f1(w.flags, y);
        set_f1(w.flags, __ldg(m.twin + y));
    }
}

void launch_chords(const MeshView &m, const Work &w, cudaStream_t s) {
    k_chords<<<w.persistent_blocks, 256, 0, s>>>(m, w);
}

// ===========================================================================
// Links around chord endpoints.  Around a vertex the relink pairs each
// frontier half-edge o leaving it with the next frontier half-edge leaving
// it in clockwise order: next[twin o] = that half-edge.  A chord half-edge c
// inserts itself into that order, so only the two links touching c change:
//   after c : y = first F1 half-edge clockwise from c  -> next[twin c] = y
//   before c: z = first F1 half-edge counter-clockwise from c (CCW(z) =
//             twin(prev z)) -> next[twin z] = c
// Every other link keeps its stage-4 value.  Two chords at one vertex write
// the link between them with the same value, so no ordering is needed.
// Every half-edge whose next or prev changes gets the walk-start mark (the
// polygon kernel needs the marks to be a superset of the polygon minima).
// ===========================================================================
// in a batch, a union link a -> b (both interior, one mesh) in the mesh's own
// next/prev as well
struct LocalLinks {
    int32_t sh, ho;  // 3 t_off and h_off of the mesh; ho < 0: a single mesh
    __device__ void link(const Work &w, int32_t a, int32_t b) const {
        if (ho < 0) return;
        w.loc_next[ho + (a - sh)] = b - sh;
        w.loc_prev[ho + (b - sh)] = a - sh;
    }
};

__device__ __forceinline__ void relink_around(const MeshView &m, const Work &w, int32_t c, int32_t HI) {
    LocalLinks loc{0, -1};
    if (w.loc_n > 0) {
        const int32_t mj = mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, tri_of(c));
        loc.sh = 3 * __ldg(w.loc_t_off + mj);
        loc.ho = __ldg(w.loc_h_off + mj);
    }
    // clockwise neighbour
    int32_t tc = __ldg(m.twin + c);
    int32_t y = nx_of(tc);
    int32_t steps = 0;
    while (!f1_of(w.flags, y, HI)) {
        y = nx_of(__ldg(m.twin + y));
        if (++steps > w.max_rot) { atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING); return; }
    }
    m.next[tc] = y;
    if (loc.ho < 0) m.prev[y] = tc;  // a batch's union prev is never read
    loc.link(w, tc, y);
    set_start(w.flags, tc);
    set_start(w.flags, y);
    // counter-clockwise neighbour; reaching a border half-edge z means the
    // interior half-edge before it, pv, is twin(z)
    int32_t pv = pv_of(c);
    int32_t z = __ldg(m.twin + pv);
    steps = 0;
    while (!f1_of(w.flags, z, HI)) {
        pv = pv_of(z);
        z = __ldg(m.twin + pv);
        if (++steps > w.max_rot) { atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING); return; }
    }
    // twin(z) == pv
    m.next[pv] = c;
    if (loc.ho < 0) m.prev[c] = pv;
    loc.link(w, pv, c);
    set_start(w.flags, pv);
    set_start(w.flags, c);
}

// over a list of chords (*count of them, at most cap; negative entries are
// skipped): the repair's chords, or the convexification's
__global__ void __launch_bounds__(256) k_chord_links(MeshView m, Work w, const int32_t *list, const int32_t *count,
                                                     int32_t cap) {
    const int32_t HI = 3 * m.T;
    int32_t n = *count;
    if (n > cap) n = cap;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += gridDim.x * blockDim.x) {
        const int32_t c0 = list[i >> 1];
        if (c0 < 0) continue;
        const int32_t c = (i & 1) ? __ldg(m.twin + c0) : c0;
        relink_around(m, w, c, HI);
    }
}

void launch_chord_links(const MeshView &m, const Work &w, cudaStream_t s) {
    k_chord_links<<<w.persistent_blocks, 256, 0, s>>>(m, w, w.chords, &w.ctrl->n_tips, w.tip_cap);
}

void launch_chord_links_list(const MeshView &m, const Work &w, const int32_t *list, const int32_t *count,
                             int32_t cap, cudaStream_t s) {
    k_chord_links<<<w.persistent_blocks, 256, 0, s>>>(m, w, list, count, cap);
}

}  // namespace polylla
