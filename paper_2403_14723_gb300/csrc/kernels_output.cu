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
// Polygons, keyed by their smallest half-edge.  A frontier half-edge e is
// its polygon's minimum iff walking next from e comes back to e without
// meeting a smaller half-edge.  A minimum is smaller than both its
// neighbours along the polygon, so only frontier half-edges with
// next[e] > e and prev[e] > e walk (about one per polygon on the workloads
// measured: polygons are listed in an order that rises and then falls).
// This finds every cycle of the relink exactly once, keyed by the canonical
// seed the paper's Algorithm 14 keeps, without a seed list.  The tile's
// (seed count, polygon length) pairs are scanned in index order, so seeds
// come out ascending; each seed then lists its polygon from itself along
// next.
//
// Tile = 2048 consecutive interior half-edges per 256-thread block.
//  1. next of the tile is staged in shared memory and prev streamed through
//     registers (coalesced vector loads) to test the walk-start condition;
//     steps that stay in the tile read shared memory.
//  2. walk starts are compacted into a shared list in index order (warp
//     scan), so each lane walks one chain at a time.
//  3. walk results are scanned block-wide; warp 0 runs the decoupled
//     look-back while every warp writes the tile's polygons into a shared
//     buffer at their tile-local offsets; the buffer then goes out with
//     coalesced stores (entries past its capacity go out directly).
// The footprint is kept small (about 25 KB) so that several blocks share an
// SM: the walks are chains of dependent loads and need many in flight.
// Tiles take an atomic ticket so that every tile's predecessors are already
// running when it looks back.
// ===========================================================================
struct PolySmem {
    int32_t nx[POLY_TILE];
    int32_t he[POLY_BUF];
    int32_t v[POLY_BUF];
    int32_t cand[POLY_TILE];   // tile-local index | tile-local polygon index << 16
    int32_t res[POLY_TILE];    // walk: polygon length or 0; after the scan: local offset or -1
    unsigned long long warp_tot[POLY_THREADS / 32];
    unsigned long long prefix;
    int32_t warp_cnt[2][POLY_THREADS / 32];
    int32_t tile;
};

size_t polygons_smem_bytes() { return sizeof(PolySmem); }

__global__ void __launch_bounds__(POLY_THREADS) k_polygons(MeshView m, Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PolySmem &S = *reinterpret_cast<PolySmem *>(smem_raw);
    const int32_t HI = 3 * m.T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) S.tile = atomicAdd(&w.ctrl->ticket, 1);
    __syncthreads();
    const int32_t tile = S.tile;
    const int32_t tb = tile * POLY_TILE;  // 8192-byte aligned
    const int32_t nE = min(POLY_TILE, HI - tb);

    // ---- stage next, test walk starts: thread owns half-edges 4q..4q+3 of
    //      two 1024-entry halves (q = threadIdx.x) -------------------------
    uint32_t mask[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int32_t i = threadIdx.x + h * POLY_THREADS;  // int4 index in the tile
        const int32_t el0 = 4 * i;
        if (el0 >= nE) continue;
        int32_t nv[4], pv[4];
        if (el0 + 3 < nE) {
            const int4 a = reinterpret_cast<const int4 *>(m.next + tb)[i];
            const int4 b = reinterpret_cast<const int4 *>(m.prev + tb)[i];
            nv[0] = a.x; nv[1] = a.y; nv[2] = a.z; nv[3] = a.w;
            pv[0] = b.x; pv[1] = b.y; pv[2] = b.z; pv[3] = b.w;
            reinterpret_cast<int4 *>(S.nx)[i] = a;
        } else {
            for (int q = 0; q < 4; q++) {
                nv[q] = el0 + q < nE ? m.next[tb + el0 + q] : 0;
                pv[q] = el0 + q < nE ? m.prev[tb + el0 + q] : 0;
                if (el0 + q < nE) S.nx[el0 + q] = nv[q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int32_t e = tb + el0 + q;
            if (el0 + q < nE && nv[q] > e && pv[q] > e) {
                const uint32_t f = w.flags[tri_of(e)];
                if ((f >> loc_of(e)) & 1u) mask[h] |= 1u << q;
            }
        }
    }
    // ---- compact the walk starts in index order --------------------------
    int32_t incl[2], cnt[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        cnt[h] = __popc(mask[h]);
        incl[h] = cnt[h];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl[h], o);
            if (lane >= o) incl[h] += v;
        }
        if (lane == 31) S.warp_cnt[h][warp] = incl[h];
    }
    __syncthreads();
    int32_t base0 = 0, tot0 = 0, base1 = 0, tot1 = 0;
#pragma unroll
    for (int q = 0; q < POLY_THREADS / 32; q++) {
        if (q < warp) { base0 += S.warp_cnt[0][q]; base1 += S.warp_cnt[1][q]; }
        tot0 += S.warp_cnt[0][q];
        tot1 += S.warp_cnt[1][q];
    }
    const int32_t NC = tot0 + tot1;
    {
        int32_t pos = base0 + incl[0] - cnt[0];
        for (uint32_t mm = mask[0]; mm; mm &= mm - 1) S.cand[pos++] = 4 * threadIdx.x + __ffs(mm) - 1;
        pos = tot0 + base1 + incl[1] - cnt[1];
        for (uint32_t mm = mask[1]; mm; mm &= mm - 1)
            S.cand[pos++] = 4 * (threadIdx.x + POLY_THREADS) + __ffs(mm) - 1;
    }
    __syncthreads();
    auto next_of = [&](int32_t x) -> int32_t {
        const uint32_t d = (uint32_t)(x - tb);
        return d < (uint32_t)nE ? S.nx[d] : m.next[x];
    };
    // ---- walk from each start --------------------------------------------
    for (int32_t ci = threadIdx.x; ci < NC; ci += POLY_THREADS) {
        const int32_t el = S.cand[ci];
        const int32_t e = tb + el;
        int32_t x = S.nx[el];
        int32_t L = 1;
        while (x > e) {
            x = next_of(x);
            if (++L > HI) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                break;
            }
        }
        S.res[ci] = (x == e) ? L : 0;
    }
    __syncthreads();
    // ---- scan of (polygon count, length) over the starts, in order -------
    // thread i owns starts [8i, 8i+8)
    unsigned long long mine = 0;
    const int32_t cb = threadIdx.x * POLY_ITEMS;
#pragma unroll
    for (int j = 0; j < POLY_ITEMS; j++) {
        const int32_t ci = cb + j;
        if (ci < NC) {
            const int32_t L = S.res[ci];
            if (L > 0) mine += (1ull << 32) | (unsigned long long)(uint32_t)L;
        }
    }
    unsigned long long sincl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, sincl, o);
        if (lane >= o) sincl += v;
    }
    if (lane == 31) S.warp_tot[warp] = sincl;
    __syncthreads();
    unsigned long long warp_base = 0, tile_total = 0;
#pragma unroll
    for (int q = 0; q < POLY_THREADS / 32; q++) {
        const unsigned long long v = S.warp_tot[q];
        if (q < warp) warp_base += v;
        tile_total += v;
    }
    {
        unsigned long long run = warp_base + sincl - mine;
#pragma unroll
        for (int j = 0; j < POLY_ITEMS; j++) {
            const int32_t ci = cb + j;
            if (ci < NC) {
                const int32_t L = S.res[ci];
                S.cand[ci] = (S.cand[ci] & 0xffff) | ((int32_t)(run >> 32) << 16);
                S.res[ci] = L > 0 ? (int32_t)(run & 0xffffffffu) : -1;
                if (L > 0) run += (1ull << 32) | (unsigned long long)(uint32_t)L;
            }
        }
    }
    // ---- decoupled look-back (warp 0) ------------------------------------
    if (warp == 0) {
        unsigned long long prefix = 0;
        if (tile == 0) {
            if (lane == 0) lb_store(w.tile_status + tile, LB_INC | tile_total);
        } else {
            if (lane == 0) lb_store(w.tile_status + tile, LB_AGG | tile_total);
            prefix = lookback(w.tile_status, tile, w.ctrl);
            if (lane == 0) lb_store(w.tile_status + tile, LB_INC | ((prefix + tile_total) & LB_VAL));
        }
        if (lane == 0) S.prefix = prefix;
    }
    __syncthreads();  // offsets visible to all; warp 0 done
    // ---- the tile's polygons into the shared CSR buffer ------------------
    // a thread visits the same starts here and below (ci = tid + 256*it, at
    // most 8 of them); bit it of `over` marks a polygon that runs past the
    // buffer and still has entries to store directly
    uint32_t over = 0;
    {
        int it = 0;
        for (int32_t ci = threadIdx.x; ci < NC; ci += POLY_THREADS, it++) {
            const int32_t lo = S.res[ci];
            if (lo < 0) continue;
            if (lo >= POLY_BUF) { over |= 1u << it; continue; }
            const int32_t e = tb + (S.cand[ci] & 0xffff);
            int32_t x = e, k = lo;
            do {
                S.he[k] = x;
                S.v[k] = __ldg(m.origin + x);
                k++;
                x = next_of(x);
            } while (x != e && k < POLY_BUF);
            if (x != e) over |= 1u << it;
        }
    }
    __syncthreads();
    const unsigned long long pre = S.prefix;
    const int32_t P0 = (int32_t)(pre >> 32);
    const int32_t O0 = (int32_t)(pre & 0xffffffffu);
    const int32_t tile_cnt = (int32_t)(tile_total >> 32);
    const int32_t tile_len = (int32_t)(tile_total & 0xffffffffu);
    // Capacities: P <= T seeds, N_F <= 3T listed half-edges.  A valid run
    // never reaches them; after a device error (next no longer a
    // permutation) they keep every write in bounds.
    const bool fits = P0 >= 0 && O0 >= 0 && (int64_t)P0 + tile_cnt <= (int64_t)m.T &&
                      (int64_t)O0 + tile_len <= (int64_t)HI;
    if (!fits) {
        if (threadIdx.x == 0) atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
    } else {
        int it = 0;
        for (int32_t ci = threadIdx.x; ci < NC; ci += POLY_THREADS, it++) {
            const int32_t lo = S.res[ci];
            if (lo < 0) continue;
            const int32_t e = tb + (S.cand[ci] & 0xffff);
            const int32_t pi = S.cand[ci] >> 16;
            w.seeds[P0 + pi] = e;
            w.offsets[P0 + pi] = O0 + lo;
            if ((over >> it) & 1u) {
                // entries past the shared buffer go out directly
                int32_t x = e, k = lo, guard = 0;
                do {
                    if (k >= POLY_BUF && k < tile_len) {
                        w.he_list[O0 + k] = x;
                        w.v_list[O0 + k] = __ldg(m.origin + x);
                    }
                    k++;
                    x = next_of(x);
                } while (x != e && ++guard < HI);
            }
        }
        const int32_t nbuf = min(tile_len, POLY_BUF);
        for (int32_t k = threadIdx.x; k < nbuf; k += POLY_THREADS) {
            w.he_list[O0 + k] = S.he[k];
            w.v_list[O0 + k] = S.v[k];
        }
    }
    if (tile == w.n_tiles - 1 && threadIdx.x == 0) {
        const unsigned long long tot = pre + tile_total;
        int32_t P = (int32_t)(tot >> 32);
        const int32_t NF = (int32_t)(tot & 0xffffffffu);
        if (P > m.T || NF > HI || NF < 0) {
            atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            P = P > m.T ? m.T : P;
        }
        w.offsets[P] = NF;
        w.ctrl->n_polygons = P;
        w.ctrl->n_frontier = NF;
    }
}

int polygons_configure() {
    return cudaFuncSetAttribute(k_polygons, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(PolySmem)) == cudaSuccess ? 0 : -1;
}

void launch_polygons(const MeshView &m, const Work &w, cudaStream_t s) {
    k_polygons<<<w.n_tiles, POLY_THREADS, sizeof(PolySmem), s>>>(m, w);
}

}  // namespace polylla
