// Output kernel (stages 5b-5d): find every polygon, key it by its smallest
// half-edge, and write the scan-compacted CSR in ascending seed order, in
// one launch.
//
// A frontier half-edge e is its polygon's minimum iff walking next from e
// comes back to e without meeting a smaller half-edge.  A minimum is smaller
// than both its neighbours along the polygon, so only half-edges carrying
// the relink's walk-start mark (next and prev both larger, a superset kept
// by the repair) walk.  This finds every cycle of the relink exactly once,
// keyed by the canonical seed the paper's Algorithm 14 keeps, without a seed
// list; listing each minimum's cycle from the minimum, minima in ascending
// order, is the canonical CSR (Section 6.8's scan-and-compact output).
//
// The stage works on tiles of consecutive triangles.  Meshes come in a
// spatially coherent order, so about nine polygons in ten lie inside the
// tile that holds their minimum, and two kernels stream the tiles through
// shared memory (bulk copies by the TMA engine, one mbarrier per CTA):
//   k_poly_count  walks the starts of its tile (leaving the tile only for
//                 the polygons that cross it) and totals the minima's
//                 (count, length) pairs per warp and per tile;
//   k_tile_scan   scans the tile totals per group of 1024 tiles;
//   k_poly_list   lists every warp's polygons through a staging buffer
//                 that goes out with coalesced stores.
// No warp waits for another warp.  Two designs that did were slower: a
// single kernel whose tiles looked back for the totals of tiles still being
// walked (every CTA in flight waited for the slowest walk before it), and a
// listing kernel whose tiles looked back for the prefixes of tiles still
// being listed (each look-back summed back over the tiles started during
// its own round trip to L2).
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// exclusive block scan of one value per thread (blockDim.x a multiple of
// 32, at most 1024); returns the exclusive prefix, *total gets the block
// total.  s_warp holds 32 + 1 entries.
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long *s_warp,
                                              unsigned long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned long long inc = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        // one warp scans the warp totals: s_warp[q] becomes the exclusive
        // prefix of warp q, s_warp[32] the block total
        const unsigned long long x = lane < nw ? s_warp[lane] : 0ull;
        const unsigned long long xi = warp_incl_scan(x, lane);
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const unsigned long long wb = s_warp[warp];
    *total = s_warp[32];
    __syncthreads();  // s_warp may be reused by the caller
    return wb + inc - v;
}

// ===========================================================================
// k_scan_blocks: one block, exclusive scan of n 64-bit values; *grand
// receives the sum.  Rounds of blockDim.x coalesced entries with a running
// carry.  (Used by the Lepp paths.)
// ===========================================================================
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_blocks(const unsigned long long *in, unsigned long long *out,
                                                              int32_t n, unsigned long long *grand) {
    __shared__ unsigned long long s_warp[33];
    unsigned long long carry = 0;
    for (int32_t b = 0; b < n; b += SCAN_THREADS) {
        const int32_t i = b + threadIdx.x;
        const unsigned long long v = i < n ? in[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_excl_scan(v, s_warp, &total);
        if (i < n) out[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

void launch_scan_u64(const unsigned long long *in, unsigned long long *out, int32_t n, unsigned long long *grand,
                     cudaStream_t s) {
    k_scan_blocks<<<1, SCAN_THREADS, 0, s>>>(in, out, n, grand);
}

// ---- per-thread records of the count pass ------------------------------------
// One 64-bit word per thread: bits 0-30 the length of the warp's minima
// before the thread (< 2^31 since N_F <= 3T < 2^31), bits 31-40 their count
// (< 32 x 3 x 8), bits 41-63 the mask of the thread's own minima (3 bits per
// triangle, at most 7 triangles per thread).
constexpr int REC_CNT_SHIFT = 31;
constexpr int REC_MASK_SHIFT = 41;
constexpr int REC_MASK_BITS = 64 - REC_MASK_SHIFT;
constexpr unsigned long long REC_LEN_MASK = (1ull << REC_CNT_SHIFT) - 1ull;
constexpr unsigned long long REC_CNT_MASK = (1ull << (REC_MASK_SHIFT - REC_CNT_SHIFT)) - 1ull;

// ---- tiles -----------------------------------------------------------------
// A tile is TILE consecutive triangles (3 TILE half-edges); its copies start
// on 16-byte boundaries (TILE is a multiple of 16) and round their length up
// to 16 bytes: at most 3 ints past 3T, inside next/origin because
// H >= 3T + 3, and flags is allocated to a multiple of 16 bytes.
__device__ __forceinline__ uint32_t tile_bytes(int32_t nt, int32_t bytes_per_triangle) {
    return ((uint32_t)(bytes_per_triangle * nt) + 15u) & ~15u;
}

// ===========================================================================
// k_poly_count<TILE, NT>: one CTA per tile, TILE / NT consecutive triangles
// per thread.  Thread 0 bulk-copies the tile's next and flags into shared
// memory; every start of the thread's triangles walks next (shared memory
// inside the tile, global memory outside) until a smaller half-edge or back
// to itself.  A warp scan of the minima's (count, length) pairs gives each
// thread its place in its warp's range; each warp stores its total and adds
// it to the tile's total (zeroed by the first kernel of the generate).  No
// warp waits for another: a slow walk holds up its own warp only.
// ===========================================================================
template <int TILE, int NT>
__global__ void __launch_bounds__(NT) k_poly_count(MeshView m, Work w) {
    constexpr int IPT = TILE / NT;
    constexpr int E = 3 * TILE;
    constexpr int NW = NT / 32;
    static_assert(TILE % NT == 0 && IPT >= 1 && 3 * IPT <= REC_MASK_BITS, "a thread's minima fit its record");
    static_assert(TILE % 16 == 0, "tile copies start on 16-byte boundaries");
    extern __shared__ __align__(128) unsigned char smem[];
    int32_t *s_nx = reinterpret_cast<int32_t *>(smem);         // [E]
    uint8_t *s_fl = reinterpret_cast<uint8_t *>(s_nx + E);     // [TILE]
    __shared__ __align__(8) uint64_t s_bar;
    const int32_t HI = 3 * m.T;
    const int32_t tile = blockIdx.x;
    const int32_t t0 = tile * TILE;
    const int32_t nt = min(TILE, m.T - t0);
    const int32_t eb = 3 * t0;
    const uint32_t ne = (uint32_t)(3 * nt);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t rec = (int64_t)tile * NT + threadIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        const uint32_t be = tile_bytes(nt, 12), bf = tile_bytes(nt, 1);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar, be + bf);
        bulk_load(s_nx, m.next + eb, be, &s_bar);
        bulk_load(s_fl, w.flags + t0, bf, &s_bar);
    }
    __syncthreads();
    const bool loaded = __all_sync(0xffffffffu, mbar_wait(&s_bar, 0));
    uint32_t minmask = 0, cnt = 0, len = 0;
    if (loaded) {
        const int32_t lt0 = (int32_t)threadIdx.x * IPT;
        bool runaway = false;
#pragma unroll
        for (int q = 0; q < IPT; q++) {
            const int32_t lt = lt0 + q;
            if (lt >= nt) break;
            const uint32_t f = s_fl[lt];
            uint32_t st = f & (f >> 3) & 7u;
            while (st) {
                const int k = __ffs(st) - 1;
                st &= st - 1u;
                const int32_t e = eb + 3 * lt + k;
                int32_t x = s_nx[3 * lt + k];
                uint32_t L = 1;
                while (x > e) {
                    const uint32_t d = (uint32_t)(x - eb);
                    x = d < ne ? s_nx[d] : __ldg(m.next + x);
                    if (++L > (uint32_t)HI) {
                        runaway = true;
                        x = -1;
                    }
                }
                if (x == e) {
                    minmask |= 1u << (3 * q + k);
                    cnt++;
                    len += L;
                }
            }
        }
        if (runaway) atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
    } else if (lane == 0) {
        // copies not seen in time: record it; this warp's part of the tile
        // stays empty
        atomicOr(&w.ctrl->error, DEV_ERR_TIMEOUT);
    }
    const unsigned long long v = ((unsigned long long)cnt << 32) | len;
    const unsigned long long inc = warp_incl_scan(v, lane);
    const unsigned long long ex = inc - v;  // (minima, length) of the lanes before, in the warp
    w.poly_rec[rec] = (ex & REC_LEN_MASK) | ((ex >> 32) << REC_CNT_SHIFT) |
                      ((unsigned long long)minmask << REC_MASK_SHIFT);
    if (lane == 31) {
        w.poly_wtot[(int64_t)tile * NW + wid] = inc;
        atomicAdd(w.tile_state + tile, inc);
    }
    // a CTA leaves only after its bulk copies landed (bounded wait)
    if (!loaded && threadIdx.x == 0) mbar_wait(&s_bar, 0);
}

// ===========================================================================
// k_tile_scan: one block per group of SCAN_THREADS tiles: the exclusive scan
// of the tiles' (polygons, length) totals within the group (tile_pre) and
// the group's total (group_tot).  The last block to finish (a counter in
// the control block) scans the group totals into group_pre and ends the
// output: P, N_F and offsets[P].  A tile's place in the output is then
// tile_pre[tile] + group_pre[its group], and no block waits for another.
// ===========================================================================
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(MeshView m, Work w, int32_t n) {
    __shared__ unsigned long long s_warp[33];
    __shared__ int s_last;
    const int32_t i = blockIdx.x * SCAN_THREADS + threadIdx.x;
    const unsigned long long v = i < n ? w.tile_state[i] : 0ull;
    unsigned long long total;
    const unsigned long long ex = block_excl_scan(v, s_warp, &total);
    if (i < n) w.tile_pre[i] = ex;
    if (threadIdx.x == 0) {
        w.group_tot[blockIdx.x] = total;
        __threadfence();  // the total is visible before the count says so
        s_last = atomicAdd(&w.ctrl->scan_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long carry = 0;
    for (int32_t b = 0; b < (int32_t)gridDim.x; b += SCAN_THREADS) {
        const int32_t g = b + threadIdx.x;
        const unsigned long long x = g < (int32_t)gridDim.x ? __ldcg(w.group_tot + g) : 0ull;
        unsigned long long t;
        const unsigned long long e = block_excl_scan(x, s_warp, &t);
        if (g < (int32_t)gridDim.x) w.group_pre[g] = carry + e;
        carry += t;
    }
    if (threadIdx.x != 0) return;
    int64_t P = (int64_t)(carry >> 32);
    const int64_t NF = (int64_t)(carry & 0xffffffffull);
    if (P > (int64_t)m.T || NF > 3 * (int64_t)m.T) {
        atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        P = P > m.T ? m.T : P;
    }
    w.offsets[P] = (int32_t)NF;
    w.ctrl->n_polygons = (int32_t)P;
    w.ctrl->n_frontier = (int32_t)NF;
    // in a batch, P closes the ranges (and starts the meshes without triangles
    // at the end, which no lane holds)
    for (int32_t j = w.loc_n; w.loc_n > 0 && j >= 0 && __ldg(w.loc_t_off + j) >= m.T; j--) w.loc_poly_off[j] = (int32_t)P;
    // a batch mesh with an index outside its range (found by the longest-edge
    // kernel) fails the run; the word is cleared for the next one
    if (w.input_err && *w.input_err) {
        atomicOr(&w.ctrl->error, DEV_ERR_INPUT);
        *w.input_err = 0;
    }
}

// ===========================================================================
// k_poly_list<TILE, NT, BATCH>: one CTA per tile (BATCH: the mesh is a
// batch's union, whose seeds, lists and per-mesh polygon ranges are written
// in each mesh's own indices).  Thread 0 bulk-copies the tile's
// next and origin (BATCH: next only; the block reads origin from the
// meshes' own arrays, which hold local vertex ids, into shared memory).
// Then every warp works on its own: its first polygon and
// entry are the scanned total of the tiles before its tile plus the totals
// of the warps before it in the tile; every minimum of its lanes writes its
// seed and offset and lists its polygon from itself along next (half-edge
// and its origin) into the warp's staging buffer (entries past it go out
// directly), which the warp then stores, one contiguous range of he_list
// and v_list, coalesced.
// ===========================================================================
template <int TILE, int NT, bool BATCH>
__global__ void __launch_bounds__(NT) k_poly_list(MeshView m, Work w) {
    constexpr int IPT = TILE / NT;
    constexpr int E = 3 * TILE;
    constexpr int NW = NT / 32;
    constexpr int WCAP = 64 * IPT;  // CSR entries a warp stages
    extern __shared__ __align__(128) unsigned char smem[];
    int32_t *s_nx = reinterpret_cast<int32_t *>(smem);  // [E]
    int32_t *s_org = s_nx + E;                          // [E + 4]
    int32_t *s_stage = s_org + E + 4;                   // [NW][2][WCAP]
    __shared__ __align__(8) uint64_t s_bar;
    const int32_t HI = 3 * m.T;
    const int32_t tile = blockIdx.x;
    const int32_t t0 = tile * TILE;
    const int32_t nt = min(TILE, m.T - t0);
    const int32_t eb = 3 * t0;
    const uint32_t ne = (uint32_t)(3 * nt);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // batches: the mesh of the tile's first triangle, and where the tile's
    // origins start in s_org (-1: not bulk-copied, loaded below)
    __shared__ int32_t s_j0, s_r;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        const uint32_t be = tile_bytes(nt, 12);
        fence_proxy_async_smem();
        if (!BATCH) {
            mbar_arrive_expect_tx(&s_bar, 2 * be);
            bulk_load(s_nx, m.next + eb, be, &s_bar);
            bulk_load(s_org, m.origin + eb, be, &s_bar);
            s_r = 0;
        } else {
            // a tile inside one mesh has its origins contiguous in the local
            // array, from entry L0: bulk-copy from L0 rounded down to 16 bytes
            // (r entries early) to 16 bytes past the end, which stays inside
            // the mesh's entries since at least 3 border half-edges follow
            // its interior ones
            const int32_t j = mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, t0);
            s_j0 = j;
            const bool one = w.loc_aligned && 3 * __ldg(w.loc_t_off + j + 1) >= eb + (int32_t)ne;
            const int32_t L0 = eb + __ldg(w.loc_h_off + j) - 3 * __ldg(w.loc_t_off + j);
            const int32_t r = L0 & 3;
            const uint32_t bo = ((uint32_t)(r + (int32_t)ne) * 4u + 15u) & ~15u;
            mbar_arrive_expect_tx(&s_bar, one ? be + bo : be);
            bulk_load(s_nx, m.next + eb, be, &s_bar);
            if (one) bulk_load(s_org, w.loc_origin + (L0 - r), bo, &s_bar);
            s_r = one ? r : -1;
        }
    }
    __syncthreads();
    if (BATCH && s_r < 0) {
        // origin from the meshes' own arrays (already local vertex ids): union
        // half-edge x of mesh j is local entry x + h_off[j] - 3 t_off[j].  All
        // of a thread's addresses first, then all its loads, then the stores,
        // so its loads are in flight together.
        constexpr int NK = E / NT;
        static_assert(E % NT == 0, "whole rounds of the tile's half-edges");
        int32_t j = s_j0;
        int32_t jn = 3 * __ldg(w.loc_t_off + j + 1);
        int32_t sb = __ldg(w.loc_h_off + j) - 3 * __ldg(w.loc_t_off + j);
        int32_t at[NK];
#pragma unroll
        for (int k = 0; k < NK; k++) {
            const uint32_t d = threadIdx.x + (uint32_t)(k * NT);
            const int32_t x = eb + (int32_t)d;
            at[k] = -1;
            if (d < ne) {
                while (x >= jn && j + 1 < w.loc_n) {
                    j++;
                    jn = 3 * __ldg(w.loc_t_off + j + 1);
                    sb = __ldg(w.loc_h_off + j) - 3 * __ldg(w.loc_t_off + j);
                }
                at[k] = x + sb;
            }
        }
#pragma unroll
        for (int k = 0; k < NK; k++) at[k] = at[k] >= 0 ? __ldg(w.loc_origin + at[k]) : 0;
#pragma unroll
        for (int k = 0; k < NK; k++) {
            const uint32_t d = threadIdx.x + (uint32_t)(k * NT);
            if (d < ne) s_org[d] = at[k];
        }
        __syncthreads();
    }
    const int32_t *so = s_org + (s_r > 0 ? s_r : 0);  // the tile's origins
    const int64_t rec = (int64_t)tile * NT + threadIdx.x;
    const unsigned long long r = w.poly_rec[rec];
    const unsigned long long ex = ((r >> REC_CNT_SHIFT) & REC_CNT_MASK) << 32 | (r & REC_LEN_MASK);
    uint32_t minmask = (uint32_t)(r >> REC_MASK_SHIFT);
    // the warps before this one in the tile, and this warp's own total
    const unsigned long long wt = lane <= wid ? w.poly_wtot[(int64_t)tile * NW + lane] : 0ull;
    const unsigned long long wbase = warp_sum(lane < wid ? wt : 0ull);
    const unsigned long long wtot = __shfl_sync(0xffffffffu, wt, wid);
    // the tiles before this one: those of the groups before its group, then
    // those before it in its group
    const unsigned long long tbase = w.group_pre[tile / SCAN_THREADS] + w.tile_pre[tile];
    if (!__all_sync(0xffffffffu, mbar_wait(&s_bar, 0))) {
        if (lane == 0) {
            atomicOr(&w.ctrl->error, DEV_ERR_TIMEOUT);
            if (wid == 0) mbar_wait(&s_bar, 0);
        }
        return;
    }
    const unsigned long long base = tbase + wbase;  // this warp's first polygon and entry
    const int64_t P0 = (int64_t)(base >> 32);
    const int64_t NF0 = (int64_t)(base & 0xffffffffull);
    const int64_t wlen = (int64_t)(wtot & 0xffffffffull);
    if (P0 + (int64_t)(wtot >> 32) > (int64_t)m.T || NF0 + wlen > (int64_t)HI) {
        if (lane == 0) atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        return;  // warp-uniform
    }
    int32_t p = (int32_t)(P0 + (int64_t)(ex >> 32));
    int32_t pos = (int32_t)(ex & 0xffffffffull);  // within the warp's range
    int32_t *he_out = w.he_list + NF0;
    int32_t *v_out = w.v_list + NF0;
    int32_t *st_he = s_stage + wid * 2 * WCAP;
    int32_t *st_v = st_he + WCAP;
    const int32_t lt0 = (int32_t)threadIdx.x * IPT;
    // in a batch, the mesh of the warp's first triangle (from the mesh
    // table); each lane steps forward from it to the meshes of its minima
    int32_t mi = 0;
    if (BATCH) {
        const int32_t tw0 = t0 + (int32_t)(threadIdx.x & ~31u) * IPT;
        mi = __shfl_sync(0xffffffffu, lane == 0 ? mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, min(tw0, m.T - 1)) : 0, 0);
    }
    // in a batch, the lane holding a mesh's first triangle writes the mesh's
    // first polygon: its own first polygon plus its minima before the mesh
    if (BATCH && lt0 < nt) {
        const int32_t lf = t0 + lt0, le_ = t0 + min(lt0 + IPT, nt);  // the lane's triangles [lf, le_)
        int32_t j = mi;
        while (j < w.loc_n && __ldg(w.loc_t_off + j) < lf) j++;
        for (; j < w.loc_n; j++) {
            const int32_t tj = __ldg(w.loc_t_off + j);
            if (tj >= le_) break;
            const uint32_t below = (1u << (3 * (tj - lf))) - 1u;  // minima of the lane's earlier triangles
            w.loc_poly_off[j] = p + __popc(minmask & below);
        }
    }
    while (minmask) {
        const int b = __ffs(minmask) - 1;
        minmask &= minmask - 1u;
        const int32_t e = eb + 3 * (lt0 + b / 3) + b % 3;
        // in a batch, seeds and lists are written in the mesh's own indices
        // (sb: from a union half-edge to its entry in the local arrays)
        int32_t she = 0, sb = 0;
        if (BATCH) {
            while (mi + 1 < w.loc_n && __ldg(w.loc_t_off + mi + 1) <= e / 3) mi++;
            she = 3 * __ldg(w.loc_t_off + mi);
            sb = __ldg(w.loc_h_off + mi) - she;
        }
        w.seeds[p] = e - she;
        w.offsets[p] = (int32_t)NF0 + pos;
        p++;
        int32_t x = e;
        int32_t guard = 0;
        do {  // k_poly_count's walk came back to e: this loop ends
            const uint32_t d = (uint32_t)(x - eb);
            const bool in = d < ne;
            const int32_t v = in ? so[d] : BATCH ? __ldg(w.loc_origin + x + sb) : __ldg(m.origin + x);
            if (pos < WCAP) {
                st_he[pos] = x - she;
                st_v[pos] = v;
            } else {
                he_out[pos] = x - she;
                v_out[pos] = v;
            }
            pos++;
            x = in ? s_nx[d] : __ldg(m.next + x);
        } while (x != e && ++guard < HI);
    }
    __syncwarp();
    const int32_t nb = (int32_t)min(wlen, (int64_t)WCAP);
    for (int32_t k = lane; k < nb; k += 32) {
        he_out[k] = st_he[k];
        v_out[k] = st_v[k];
    }
}

// ---- launch configurations (tile triangles, threads per CTA) ---------------
template <int TILE>
constexpr size_t count_smem() {
    return (size_t)3 * TILE * sizeof(int32_t) + TILE;
}
template <int TILE>
constexpr size_t list_smem() {
    // next and origin of the tile (origin with 4 entries to spare for an
    // unaligned start), and per warp 2 x 64 x (TILE / NT) staged entries:
    // 4 TILE ints in all
    return (size_t)(2 * 3 * TILE + 4 + 4 * TILE) * sizeof(int32_t);
}

#define POLYGON_CONFIGS(X) \
    X(1024, 256)           \
    X(1024, 512)           \
    X(2048, 512)           \
    X(2048, 1024)          \
    X(4096, 1024)

bool polygons_config_valid(int32_t tile, int32_t items) {
#define X(TL, N) \
    if (tile == TL && items == TL / N) return true;
    POLYGON_CONFIGS(X)
#undef X
    return false;
}

int polygons_configure() {
#define X(TL, N)                                                                                             \
    if (cudaFuncSetAttribute(k_poly_count<TL, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                             (int)count_smem<TL>()) != cudaSuccess ||                                        \
        cudaFuncSetAttribute(k_poly_list<TL, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                             (int)list_smem<TL>()) != cudaSuccess ||                                         \
        cudaFuncSetAttribute(k_poly_list<TL, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                             (int)list_smem<TL>()) != cudaSuccess)                                           \
        return -1;
    POLYGON_CONFIGS(X)
#undef X
    return 0;
}

// resident CTAs per SM of the listing kernel (the larger of the two)
int polygons_blocks_per_sm(int32_t tile, int32_t items) {
    int nb = 0;
#define X(TL, N)                                                                                          \
    if (tile == TL && items == TL / N) {                                                                  \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_poly_list<TL, N, false>, N, list_smem<TL>()) != \
            cudaSuccess)                                                                                  \
            nb = 0;                                                                                       \
    }
    POLYGON_CONFIGS(X)
#undef X
    return nb;
}

// the two kernels of the output stage (an unknown configuration takes the
// default one: the tuning entry points accept only valid ones)
void launch_poly_count(const MeshView &m, const Work &w, cudaStream_t s) {
#define X(TL, N)                                                                            \
    if (w.out_tile == TL && w.out_items == TL / N) {                                        \
        k_poly_count<TL, N><<<(m.T + TL - 1) / TL, N, count_smem<TL>(), s>>>(m, w);         \
        return;                                                                             \
    }
    POLYGON_CONFIGS(X)
#undef X
    k_poly_count<2048, 512><<<(m.T + 2047) / 2048, 512, count_smem<2048>(), s>>>(m, w);
}

void launch_tile_scan(const MeshView &m, const Work &w, cudaStream_t s) {
    const int32_t tile = polygons_config_valid(w.out_tile, w.out_items) ? w.out_tile : 2048;
    const int32_t n = (m.T + tile - 1) / tile;
    k_tile_scan<<<(n + SCAN_THREADS - 1) / SCAN_THREADS, SCAN_THREADS, 0, s>>>(m, w, n);
}

void launch_poly_list(const MeshView &m, const Work &w, cudaStream_t s) {
#define X(TL, N)                                                                            \
    if (w.out_tile == TL && w.out_items == TL / N) {                                        \
        if (w.loc_n > 0) k_poly_list<TL, N, true><<<(m.T + TL - 1) / TL, N, list_smem<TL>(), s>>>(m, w); \
        else k_poly_list<TL, N, false><<<(m.T + TL - 1) / TL, N, list_smem<TL>(), s>>>(m, w);      \
        return;                                                                             \
    }
    POLYGON_CONFIGS(X)
#undef X
    if (w.loc_n > 0) k_poly_list<2048, 512, true><<<(m.T + 2047) / 2048, 512, list_smem<2048>(), s>>>(m, w);
    else k_poly_list<2048, 512, false><<<(m.T + 2047) / 2048, 512, list_smem<2048>(), s>>>(m, w);
}

}  // namespace polylla
