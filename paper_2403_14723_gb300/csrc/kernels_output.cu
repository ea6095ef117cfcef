// Output kernel (stages 5b-5d): find every polygon, key it by its smallest
// half-edge, and write the scan-compacted CSR in ascending seed order, in a
// single pass with a decoupled look-back scan.
#include "polylla_internal.cuh"

namespace polylla {

// look-back word: [63:62] flag, [61:32] polygon count, [31:0] half-edge count
constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_INC = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr int LB_SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of this tile over all earlier tiles, by one warp.  Each
// lane watches one predecessor; the window slides back 32 tiles at a time
// until it meets an inclusive prefix.  Every wait is bounded: on timeout the
// error word gets DEV_ERR_TIMEOUT and the (wrong) partial sum is returned.
__device__ unsigned long long lookback(unsigned long long *status, int32_t tile, DevCtrl *ctrl) {
    const int lane = threadIdx.x & 31;
    unsigned long long acc = 0;
    int32_t hi = tile - 1;  // newest predecessor still to account for
    while (hi >= 0) {
        const int32_t idx = hi - lane;
        unsigned long long v = LB_INC;  // lanes before tile 0 see an empty inclusive
        if (idx >= 0) {
            int spins = 0;
            v = lb_load(status + idx);
            while ((v >> 62) == 0) {
                if (++spins > LB_SPIN_LIMIT) {
                    atomicOr(&ctrl->error, DEV_ERR_TIMEOUT);
                    v = LB_INC;
                    break;
                }
                __nanosleep(64);
                v = lb_load(status + idx);
            }
        }
        const unsigned inc_mask = __ballot_sync(0xffffffffu, (v >> 62) == 2);
        // lanes up to (and including) the first inclusive contribute
        const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
        unsigned long long mine = (lane <= stop) ? (v & LB_VAL) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        acc += mine;
        if (inc_mask) break;
        hi -= 32;
    }
    return acc;
}

// ===========================================================================
// Every frontier half-edge e of the tile walks next until it meets a
// smaller half-edge (e is not its polygon's minimum) or comes back to itself
// (e is the minimum: the polygon's seed, and the walk length is the polygon
// length).  This finds every cycle of the relink exactly once, keyed by its
// smallest half-edge -- the canonical seed the paper's Algorithm 14 keeps --
// without a seed list.  The tile's (seed count, half-edge count) pairs are
// scanned in index order, so seeds come out ascending; each seed then writes
// its polygon from itself along next.
//
// Tile = 2048 consecutive interior half-edges; thread i owns 8 consecutive
// ones and walks its 8 chains interleaved (independent loads in flight).
// Tiles take an atomic ticket so that every tile's predecessors are already
// running when it looks back.
// ===========================================================================
__global__ void __launch_bounds__(POLY_THREADS) k_polygons(MeshView m, Work w) {
    __shared__ int32_t s_tile;
    __shared__ unsigned long long s_warp[POLY_THREADS / 32];
    __shared__ unsigned long long s_prefix;
    const int32_t HI = 3 * m.T;
    if (threadIdx.x == 0) s_tile = atomicAdd(&w.ctrl->ticket, 1);
    __syncthreads();
    const int32_t tile = s_tile;
    const int32_t base = tile * POLY_TILE + threadIdx.x * POLY_ITEMS;

    // ---- frontier test and first step -----------------------------------
    int32_t cur[POLY_ITEMS];
    int32_t len[POLY_ITEMS];
    uint32_t active = 0, is_min = 0;
#pragma unroll
    for (int j = 0; j < POLY_ITEMS; j++) {
        const int32_t e = base + j;
        len[j] = 0;
        cur[j] = 0;
        if (e < HI && ((w.flags[tri_of(e)] >> loc_of(e)) & 1u)) {
            cur[j] = m.next[e];
            len[j] = 1;
            active |= 1u << j;
        }
    }
    // ---- walk until a smaller half-edge or back to the start ------------
    int32_t guard = 0;
    while (active) {
#pragma unroll
        for (int j = 0; j < POLY_ITEMS; j++) {
            if (!((active >> j) & 1u)) continue;
            const int32_t e = base + j;
            const int32_t c = cur[j];
            if (c == e) {
                is_min |= 1u << j;
                active &= ~(1u << j);
            } else if (c < e) {
                active &= ~(1u << j);
            }
        }
        if (!active) break;
#pragma unroll
        for (int j = 0; j < POLY_ITEMS; j++) {
            if ((active >> j) & 1u) {
                cur[j] = m.next[cur[j]];
                len[j]++;
            }
        }
        if (++guard > HI) {
            atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
            is_min = 0;
            break;
        }
    }
    // ---- block scan of (seed count, half-edge count) ---------------------
    unsigned long long mine = 0;
#pragma unroll
    for (int j = 0; j < POLY_ITEMS; j++) {
        if ((is_min >> j) & 1u) mine += (1ull << 32) | (unsigned long long)(uint32_t)len[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long warp_base = 0, tile_total = 0;
#pragma unroll
    for (int q = 0; q < POLY_THREADS / 32; q++) {
        const unsigned long long v = s_warp[q];
        if (q < warp) warp_base += v;
        tile_total += v;
    }
    const unsigned long long excl = warp_base + incl - mine;

    // ---- decoupled look-back ----------------------------------------------
    if (warp == 0) {
        unsigned long long prefix = 0;
        if (tile == 0) {
            if (lane == 0) lb_store(w.tile_status + tile, LB_INC | tile_total);
        } else {
            if (lane == 0) lb_store(w.tile_status + tile, LB_AGG | tile_total);
            prefix = lookback(w.tile_status, tile, w.ctrl);
            if (lane == 0) lb_store(w.tile_status + tile, LB_INC | ((prefix + tile_total) & LB_VAL));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    const unsigned long long start = s_prefix + excl;
    int32_t p = (int32_t)(start >> 32);
    int32_t off = (int32_t)(start & 0xffffffffu);

    // ---- emit every polygon whose seed is in this tile -------------------
    // Capacities: P <= T seeds, N_F <= 3T listed half-edges.  A valid run
    // never reaches them; after a device error (next no longer a
    // permutation) they keep every write in bounds.
#pragma unroll 1
    for (int j = 0; j < POLY_ITEMS; j++) {
        if (!((is_min >> j) & 1u)) continue;
        const int32_t e = base + j;
        if (p >= m.T || off < 0 || (int64_t)off + len[j] > (int64_t)HI) {
            atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            break;
        }
        w.seeds[p] = e;
        w.offsets[p] = off;
        int32_t c = e;
        for (int32_t k = 0; k < len[j]; k++) {
            w.he_list[off + k] = c;
            w.v_list[off + k] = __ldg(m.origin + c);
            c = m.next[c];
        }
        p++;
        off += len[j];
    }
    if (tile == w.n_tiles - 1 && threadIdx.x == 0) {
        const unsigned long long tot = s_prefix + tile_total;
        int32_t P = (int32_t)(tot >> 32);
        const int32_t NF = (int32_t)(tot & 0xffffffffu);
        if (P > m.T || NF > HI) {
            atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            P = P > m.T ? m.T : P;
        }
        w.offsets[P] = NF;
        w.ctrl->n_polygons = P;
        w.ctrl->n_frontier = NF;
    }
}

void launch_polygons(const MeshView &m, const Work &w, cudaStream_t s) {
    k_polygons<<<w.n_tiles, POLY_THREADS, 0, s>>>(m, w);
}

}  // namespace polylla
