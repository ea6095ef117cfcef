// Internal declarations of the GB300 Polylla kernels (sm_103a).
//
// Layout of the work arrays in HBM (all sized at create, reused by every
// generate; nothing is allocated on the hot path):
//   le      [T]   uint8  local index of each triangle's longest half-edge
//   flags   [T]   uint8  bits 0-2 F1 (frontier after repair) of 3t+k,
//                        bits 3-5 walk-start marks (next and prev larger),
//                        bit 6 the triangle's longest half-edge is a seed
//   tips    [V]   int32  F0 half-edge leaving each barrier tip
//   chords  [V]   int32  chord half-edge leaving each barrier tip
//   tile_state, tile_pre [T/1024] u64  (polygons, length) total of each output
//                        tile, and their exclusive scan within groups of
//                        1024 tiles; group_tot, group_pre [T/2^20 + 1] u64 the
//                        groups' totals and their exclusive scan
//   poly_rec [T/2+2049] u64  per output thread: its (polygons, length)
//                        offset in its warp's range and the mask of its minima
//   poly_wtot [T/128+34] u64  per output warp: its (polygons, length) total
//   seeds [T], offsets [T+1], he_list [3T], v_list [3T]   CSR output
//   ctrl          DevCtrl       counters and the device error word
// A batch context adds the union origin/twin/next/prev [H] (origin and the
// border entries of twin are only filled by the layout check at create; every
// generate writes the interior twin entries from the meshes' own arrays), the
// per-mesh prefix sums and polygon ranges, and the input-check word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace polylla {

// device error bits (ORed into DevCtrl::error)
enum : int32_t {
    DEV_ERR_NONTERMINATING = 1,
    DEV_ERR_CAPACITY = 2,
    DEV_ERR_TIMEOUT = 4,
    DEV_ERR_INPUT = 8,           // a batch mesh held an index outside its own range
};

struct DevCtrl {
    int32_t error;        // OR of DEV_ERR_* bits of this generate
    int32_t n_tips;       // barrier tips found by the relink
    int32_t n_polygons;   // P
    int32_t n_frontier;   // N_F
    int32_t scan_done;    // tile-scan blocks finished
    int32_t pad[3];
};

struct MeshView {
    int32_t V, T, H;
    const double2 *xy;
    const int32_t *origin;
    const int32_t *twin;
    int32_t *next;
    int32_t *prev;
};

struct Work {
    uint8_t *le;
    uint8_t *flags;
    int32_t *tips;
    int32_t *chords;
    int32_t tip_cap;
    unsigned long long *tile_state; // (polygons, length) total per output tile [n_tile_max]
    unsigned long long *tile_pre;   // their exclusive scan within groups of SCAN_THREADS tiles
    unsigned long long *group_tot;  // each group's total [n_tile_max / SCAN_THREADS + 1]
    unsigned long long *group_pre;  // their exclusive scan [n_tile_max / SCAN_THREADS + 1]
    unsigned long long *poly_rec;   // per output thread: its place in its warp and its minima [n_rec_max]
    unsigned long long *poly_wtot;  // per output warp: (polygons, length) of its range
    int32_t n_tile_max;             // ceil(T / OUT_TILE_MIN)
    int32_t out_tile;               // output tile: triangles
    int32_t out_items;              // output kernel: triangles per thread
    int32_t rl_tile;                // relink: triangles per CTA
    int32_t rl_items;               // relink: triangles per thread
    int32_t *seeds;
    int32_t *offsets;
    int32_t *he_list;
    int32_t *v_list;
    DevCtrl *ctrl;
    int32_t max_rot;
    int32_t persistent_blocks;   // grid of the sparse (tip) kernels
    int32_t le_blocks;           // grid of the persistent longest-edge kernel
    int32_t le_items;            // longest edge: triangles per lane (2 or 4)
    int32_t le_batch_blocks;     // grid of the persistent longest-edge kernel on batches
    // batches: the emitted he_list / v_list are made mesh-local when set
    const int32_t *loc_t_off;    // [loc_n+1] triangle offset of each mesh
    const int32_t *loc_v_off;    // [loc_n+1] vertex offset of each mesh
    const int32_t *loc_h_off;    // [loc_n+1] half-edge offset of each mesh in the local arrays
    int32_t *loc_next;           // the meshes' own next/prev (local indices), written
    int32_t *loc_prev;           //   by the relink and repair kernels
    int32_t *loc_poly_off;       // [loc_n+1] first polygon of each mesh, P at the end
    int32_t loc_n;               // number of meshes (0: a single mesh)
    const int32_t *loc_seg;      // [T/256 + 1] mesh of triangle 256 g (SEG_SPAN)
    int32_t loc_aligned;         // loc_origin and loc_twin start on 16-byte boundaries (bulk copies allowed)
    const int32_t *loc_origin;   // the meshes' own origin and twin arrays (local indices),
    const int32_t *loc_twin;     //   read by the longest-edge and listing kernels
    int32_t *u_twin;             // union twin of interior half-edges, written by the longest-edge kernel
    int32_t *input_err;          // batches: set on an index outside its mesh, folded into
                                 //   the error word and cleared by the tile scan
};

// A batch of independent meshes, each in the single-mesh layout with its own
// (local) indices, concatenated; prefix sums locate mesh i.  The kernels run
// on the batch's union: one mesh whose interior half-edges are those of all
// meshes in order ([3 t_off[i], 3 t_off[i+1]) for mesh i), followed by all
// border half-edges ([3 T_tot + b_off[i], ...)), with global vertex ids.
struct BatchView {
    int32_t n;                   // meshes
    int32_t T_tot, H_tot;
    const int32_t *v_off;        // [n+1] device prefix sums of V_i
    const int32_t *t_off;        // [n+1] of T_i
    const int32_t *h_off;        // [n+1] of H_i
    const int32_t *b_off;        // [n+1] of H_i - 3 T_i (border half-edges)
    const int32_t *origin;       // local arrays [sum H_i]
    const int32_t *twin;
    int32_t *next;
    int32_t *prev;
};

// output kernel: tiles of out_tile triangles (1024, 2048 or 4096), out_items
// per thread; single-block scans (Lepp paths) with SCAN_THREADS threads
constexpr int OUT_TILE_MIN = 1024;
constexpr int OUT_TILE_MAX = 4096;
constexpr int OUT_ITEMS_MIN = 2;
constexpr int OUT_TILE_DEFAULT = 2048;
constexpr int OUT_ITEMS_DEFAULT = 4;
// per-thread records of the output stage for T triangles, any configuration
__host__ __device__ constexpr int64_t out_rec_count(int64_t T) { return (T + OUT_TILE_MAX) / OUT_ITEMS_MIN + 1; }
__host__ __device__ constexpr int64_t out_warp_count(int64_t T) { return out_rec_count(T) / 32 + 2; }
constexpr int SCAN_THREADS = 1024;

// longest-edge kernel: persistent warps, each with a two-stage ring of
// tiles of 32 x (2 or 4) triangles of origin bulk-copied (TMA) into shared
// memory
constexpr int LE_THREADS = 256;
constexpr int LE_ITEMS_DEFAULT = 2;

// relink kernel: rl_tile triangles per CTA, rl_items per thread
constexpr int RL_TILE_DEFAULT = 128;
constexpr int RL_ITEMS_DEFAULT = 1;

// bounded waits: iterations of an mbarrier try_wait loop before giving up
constexpr int MBAR_WAIT_LIMIT = 1 << 22;

// ---- bulk copies (TMA engine) and mbarriers, inline PTX --------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity; false after MBAR_WAIT_LIMIT tries
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < MBAR_WAIT_LIMIT; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// batches: the mesh table holds the mesh of every SEG_SPAN-th triangle
constexpr int SEG_SPAN = 256;
__host__ __device__ constexpr int64_t seg_count(int64_t T) { return T / SEG_SPAN + 1; }

// largest i in [0, n) with off[i] <= x, for ascending prefix sums off[0..n]
// with off[0] <= x < off[n]
__device__ __forceinline__ int32_t seg_of(const int32_t *off, int32_t n, int32_t x) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the mesh of union triangle t of a batch: from the mesh table's entry at
// or before t, stepping over the meshes that end by t
__device__ __forceinline__ int32_t mesh_of(const int32_t *seg, const int32_t *t_off, int32_t n, int32_t t) {
    int32_t j = __ldg(seg + t / SEG_SPAN);
    while (j + 1 < n && __ldg(t_off + j + 1) <= t) j++;
    return j;
}

// ---- float32 filters of float64 decisions -----------------------------------
// v truncated to float32: the top 23 significand bits, so |v^ - v| <= 2^-23
// |v^| and |v^| <= |v|, by bit manipulation (no float64 instruction).  A
// magnitude outside [2^-126, 2^61) (zero included) sets bad: the caller then
// takes its exact float64 path.
__device__ __forceinline__ float trunc_to_f32(double v, uint32_t &bad) {
    uint32_t hi = (uint32_t)__double2hiint(v);
    uint32_t lo = (uint32_t)__double2loint(v);
    uint32_t mag = hi & 0x7FFFFFFFu;
    // biased float64 exponent must lie in [897, 1083]: |v| in [2^-126, 2^61)
    bad |= (uint32_t)((mag - (897u << 20)) >= ((1084u - 897u) << 20));
    // (hi:lo) << 3 puts the low 9 exponent bits at 31..23 and the top 23
    // significand bits at 22..0; subtracting 384 from that 9-bit field
    // rebiases 1023 -> 127 for exponents in range
    uint32_t bits = __funnelshift_l(lo, hi, 3) - (384u << 23);
    bits |= hi & 0x80000000u;
    return __uint_as_float(bits);
}

// ---- implicit triangle layout (paper Section 4.2) -------------------------
__device__ __forceinline__ int32_t tri_of(int32_t e) { return e / 3; }
__device__ __forceinline__ int32_t loc_of(int32_t e) { return e - 3 * (e / 3); }
__device__ __forceinline__ int32_t nx_of(int32_t e) {
    int32_t b = 3 * (e / 3);
    int32_t k = e - b;
    return b + (k == 2 ? 0 : k + 1);
}
__device__ __forceinline__ int32_t pv_of(int32_t e) {
    int32_t b = 3 * (e / 3);
    int32_t k = e - b;
    return b + (k == 0 ? 2 : k - 1);
}

// launchers (each enqueues one kernel on stream)
void launch_validate(const MeshView &m, int32_t *bad, cudaStream_t s);
void launch_longest_edge(const MeshView &m, const Work &w, cudaStream_t s);
int longest_edge_blocks_per_sm(int32_t items);
int longest_edge_batch_blocks_per_sm();
void launch_label_relink(const MeshView &m, const Work &w, cudaStream_t s);
// allows the relink kernels their shared memory on the current device (once
// per device before the first launch); 0 on success
int relink_configure();
bool relink_config_valid(int32_t tile, int32_t items);
void launch_chords(const MeshView &m, const Work &w, cudaStream_t s);
void launch_chord_links(const MeshView &m, const Work &w, cudaStream_t s);
void launch_chord_links_list(const MeshView &m, const Work &w, const int32_t *list, const int32_t *count,
                             int32_t cap, cudaStream_t s);
// convexification (kernels_convex.cu)
// two kernels: the reflex corners into reflex (count n_reflex), then their
// chords into list (count count); both lists hold at most cap entries
void launch_convex_chords(const MeshView &m, const Work &w, int32_t *reflex, int32_t *n_reflex, int32_t *list,
                          int32_t *count, int32_t cap, cudaStream_t s);
void launch_convex_mark(const MeshView &m, const Work &w, const int32_t *list, const int32_t *count, int32_t cap,
                        cudaStream_t s);
void launch_poly_count(const MeshView &m, const Work &w, cudaStream_t s);
void launch_tile_scan(const MeshView &m, const Work &w, cudaStream_t s);
void launch_poly_list(const MeshView &m, const Work &w, cudaStream_t s);
// allows the output kernels their shared memory on the current device (once
// per device before the first launch); 0 on success
int polygons_configure();
bool polygons_config_valid(int32_t tile, int32_t items);
int polygons_blocks_per_sm(int32_t tile, int32_t items);
// exclusive scan of n u64 values by one block; *grand gets the sum
void launch_scan_u64(const unsigned long long *in, unsigned long long *out, int32_t n, unsigned long long *grand,
                     cudaStream_t s);
// Lepp (kernels_lepp.cu)
void launch_lepp_terminal(const MeshView &m, const Work &w, int32_t *terminal, int32_t *length, int32_t *err,
                          cudaStream_t s);
void launch_lepp_paths(const MeshView &m, const Work &w, const int32_t *tri, int32_t n, int32_t *offsets,
                       int32_t *paths, int64_t capacity, unsigned long long *blk, unsigned long long *blk_pre,
                       unsigned long long *total, int32_t *err, cudaStream_t s);
// batches (kernels_batch.cu)
void launch_batch_pack(const BatchView &b, int32_t *u_origin, int32_t *u_twin, int32_t *u_next, int32_t *u_prev,
                       int32_t *bad, int32_t *input_err, cudaStream_t s);
void launch_batch_seg(const int32_t *t_off, int32_t n, int32_t T, int32_t *seg, cudaStream_t s);
void launch_batch_meta(const BatchView &b, const Work &w, const int32_t *poly_off, int32_t *local_offsets,
                       int32_t *meta, cudaStream_t s);

}  // namespace polylla
