// Output kernels (stages 5b-5d): find every polygon, key it by its smallest
// half-edge, and write the scan-compacted CSR in ascending seed order.
//
// Reduce, scan, emit -- no block ever waits for another:
//   k_poly_count  per tile of 2048 consecutive half-edges: find the
//                 polygons whose smallest half-edge lies in the tile, their
//                 lengths, and the tile's (polygon count, total length);
//   k_tile_scan   one block: exclusive scan of the tile totals;
//   k_poly_emit   per tile: list the tile's polygons at their final place.
//
// A frontier half-edge e is its polygon's minimum iff walking next from e
// comes back to e without meeting a smaller half-edge.  A minimum is smaller
// than both its neighbours along the polygon, so only half-edges carrying
// the relink's walk-start mark (next and prev both larger, a superset kept
// by the repair) walk; polygons are listed in an order that rises and then
// falls, so that is about one walk per polygon on the workloads measured.
// This finds every cycle of the relink exactly once, keyed by the canonical
// seed the paper's Algorithm 14 keeps, without a seed list.
#include "polylla_internal.cuh"

namespace polylla {

constexpr int GROUP = POLY_TILE / (POLY_THREADS / 32);  // starts scanned by one warp

// (polygon count << 32 | length) of one start, if it is a minimum
__device__ __forceinline__ unsigned long long pair_of(int32_t L) {
    return L > 0 ? ((1ull << 32) | (unsigned long long)(uint32_t)L) : 0ull;
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// ===========================================================================
// k_poly_count.  next of the tile is staged in shared memory (coalesced
// vector loads) for the walk steps that stay in the tile; the marked
// half-edges are compacted into a list in index order so that each lane
// walks one chain at a time, two chains interleaved per thread.  The
// minima go to the scratch list of the tile, in index order, as
// (tile-local index | length << 11), length 0 standing for "2^21 or more".
// ===========================================================================
struct CountSmem {
    int32_t nx[POLY_TILE];
    int32_t cand[POLY_TILE];   // tile-local index of each marked half-edge, in order
    int32_t res[POLY_TILE];    // polygon length if the start is a minimum, else 0
    unsigned long long warp_tot[POLY_THREADS / 32];
    int32_t warp_cnt[2][POLY_THREADS / 32];
};

__global__ void __launch_bounds__(POLY_THREADS) k_poly_count(MeshView m, Work w) {
    __shared__ __align__(16) CountSmem S;
    const int32_t HI = 3 * m.T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t tile = blockIdx.x;
    const int32_t tb = tile * POLY_TILE;  // 8192-byte aligned
    const int32_t nE = min(POLY_TILE, HI - tb);

    // ---- stage next; marks of half-edges 4i..4i+3 of each 1024-half -------
    uint32_t mask[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int32_t i = threadIdx.x + h * POLY_THREADS;  // int4 index in the tile
        const int32_t el0 = 4 * i;
        if (el0 >= nE) continue;
        if (el0 + 3 < nE) {
            reinterpret_cast<int4 *>(S.nx)[i] = reinterpret_cast<const int4 *>(m.next + tb)[i];
        } else {
            for (int q = 0; q < 4; q++)
                if (el0 + q < nE) S.nx[el0 + q] = m.next[tb + el0 + q];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int32_t e = tb + el0 + q;
            if (el0 + q < nE) {
                const uint32_t f = w.flags[tri_of(e)];
                const uint32_t k = (uint32_t)loc_of(e);
                mask[h] |= ((f >> k) & (f >> (3 + k)) & 1u) << q;
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
    // ---- walk from each start, two chains per thread interleaved --------
    for (int32_t c0 = threadIdx.x; c0 < NC; c0 += 2 * POLY_THREADS) {
        const int32_t c1 = c0 + POLY_THREADS;
        const bool has1 = c1 < NC;
        const int32_t e0 = tb + S.cand[c0];
        const int32_t e1 = has1 ? tb + S.cand[c1] : 0;
        int32_t x0 = S.nx[e0 - tb];
        int32_t x1 = has1 ? S.nx[e1 - tb] : -1;  // -1 < e1: chain 1 idle
        int32_t L0 = 1, L1 = 1, guard = 0;
        while (x0 > e0 || x1 > e1) {
            if (x0 > e0) { x0 = next_of(x0); L0++; }
            if (x1 > e1) { x1 = next_of(x1); L1++; }
            if (++guard > HI) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                x0 = -1;
                x1 = -1;
                break;
            }
        }
        S.res[c0] = (x0 == e0) ? L0 : 0;
        if (has1) S.res[c1] = (x1 == e1) ? L1 : 0;
    }
    __syncthreads();
    // ---- minima to the scratch list, in order; tile totals ----------------
    // warp g covers starts [GROUP*g, GROUP*(g+1)) in rounds of 32; the
    // per-warp totals give each warp its place in the tile's list
    unsigned long long carry = 0;
#pragma unroll
    for (int c = 0; c < GROUP / 32; c++) {
        const int32_t ci = GROUP * warp + 32 * c + lane;
        const int32_t L = ci < NC ? S.res[ci] : 0;
        carry += __shfl_sync(0xffffffffu, warp_incl_scan(pair_of(L), lane), 31);
    }
    if (lane == 0) S.warp_tot[warp] = carry;
    __syncthreads();
    unsigned long long wb = 0, total = 0;
#pragma unroll
    for (int q = 0; q < POLY_THREADS / 32; q++) {
        if (q < warp) wb += S.warp_tot[q];
        total += S.warp_tot[q];
    }
    int32_t pos = (int32_t)(wb >> 32);
#pragma unroll
    for (int c = 0; c < GROUP / 32; c++) {
        const int32_t ci = GROUP * warp + 32 * c + lane;
        const int32_t L = ci < NC ? S.res[ci] : 0;
        const unsigned ball = __ballot_sync(0xffffffffu, L > 0);
        if (L > 0) {
            const int32_t at = pos + __popc(ball & ((1u << lane) - 1u));
            const int32_t Lc = L < (1 << 21) ? L : 0;
            w.mins[tb + at] = S.cand[ci] | (Lc << 11);
        }
        pos += __popc(ball);
    }
    if (threadIdx.x == 0) w.tile_status[tile] = total;
}

// ===========================================================================
// k_tile_scan.  One block: exclusive scan of the tile totals (polygon count
// << 32 | length) into tile_pre, and the grand totals P and N_F.
// ===========================================================================
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(MeshView m, Work w) {
    __shared__ unsigned long long s_warp[SCAN_THREADS / 32];
    const int32_t n = w.n_tiles;
    const int32_t per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int32_t b = threadIdx.x * per;
    const int32_t e = min(n, b + per);
    unsigned long long sum = 0;
    for (int32_t i = b; i < e; i++) sum += w.tile_status[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long inc = warp_incl_scan(sum, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned long long wb = 0, total = 0;
    for (int q = 0; q < SCAN_THREADS / 32; q++) {
        if (q < warp) wb += s_warp[q];
        total += s_warp[q];
    }
    unsigned long long run = wb + inc - sum;
    for (int32_t i = b; i < e; i++) {
        const unsigned long long v = w.tile_status[i];
        w.tile_pre[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) {
        int32_t P = (int32_t)(total >> 32);
        const int64_t NF = (int64_t)(total & 0xffffffffu);
        const int32_t HI = 3 * m.T;
        if (P > m.T || NF > HI) {
            atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            P = P > m.T ? m.T : P;
        }
        w.offsets[P] = (int32_t)NF;
        w.ctrl->n_polygons = P;
        w.ctrl->n_frontier = (int32_t)NF;
    }
}

// ===========================================================================
// k_poly_emit.  The tile's minima (in order) and their lengths come from the
// count kernel; a block scan gives each polygon its offset.  Each polygon is
// listed from its minimum along next into a shared buffer (two polygons per
// thread interleaved; next staged for steps inside the tile); seeds,
// offsets and the buffer then go out with coalesced stores.  Entries past
// the buffer's capacity go out directly.
// ===========================================================================
struct EmitSmem {
    int32_t nx[POLY_TILE];
    int32_t he[POLY_BUF];
    int32_t v[POLY_BUF];
    int32_t mn[POLY_TILE];     // minima: tile-local index
    int32_t off[POLY_TILE];    // length of each polygon, then its offset within its warp group
    unsigned long long warp_tot[POLY_THREADS / 32];
};

__global__ void __launch_bounds__(POLY_THREADS) k_poly_emit(MeshView m, Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EmitSmem &S = *reinterpret_cast<EmitSmem *>(smem_raw);
    const int32_t HI = 3 * m.T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t tile = blockIdx.x;
    const int32_t tb = tile * POLY_TILE;
    const int32_t nE = min(POLY_TILE, HI - tb);
    const unsigned long long agg = w.tile_status[tile];
    const unsigned long long pre = w.tile_pre[tile];
    const int32_t cnt = (int32_t)(agg >> 32);
    const int32_t tile_len = (int32_t)(agg & 0xffffffffu);
    const int32_t P0 = (int32_t)(pre >> 32);
    const int32_t O0 = (int32_t)(pre & 0xffffffffu);
    // Capacities: P <= T seeds, N_F <= 3T listed half-edges, at most one
    // minimum per half-edge of the tile.  A valid run never reaches them;
    // after a device error they keep every access in bounds.
    if (cnt < 0 || cnt > nE || P0 < 0 || O0 < 0 || tile_len < 0 || (int64_t)P0 + cnt > (int64_t)m.T ||
        (int64_t)O0 + tile_len > (int64_t)HI) {
        if (threadIdx.x == 0) atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        return;
    }
    for (int i = threadIdx.x; 4 * i < nE; i += POLY_THREADS) {
        if (4 * i + 3 < nE) {
            reinterpret_cast<int4 *>(S.nx)[i] = reinterpret_cast<const int4 *>(m.next + tb)[i];
        } else {
            for (int q = 0; q < 4; q++)
                if (4 * i + q < nE) S.nx[4 * i + q] = m.next[tb + 4 * i + q];
        }
    }
    auto next_of = [&](int32_t x) -> int32_t {
        const uint32_t d = (uint32_t)(x - tb);
        return d < (uint32_t)nE ? S.nx[d] : m.next[x];
    };
    for (int i = threadIdx.x; i < cnt; i += POLY_THREADS) {
        const int32_t r = w.mins[tb + i];
        S.mn[i] = r & 0x7ff;
        S.off[i] = (int32_t)((uint32_t)r >> 11);
    }
    __syncthreads();
    // lengths of 2^21 or more were stored as 0: count them again
    for (int i = threadIdx.x; i < cnt; i += POLY_THREADS) {
        if (S.off[i] == 0) {
            const int32_t e = tb + S.mn[i];
            int32_t x = next_of(e), L = 1;
            while (x != e && L <= HI) { x = next_of(x); L++; }
            S.off[i] = L;
        }
    }
    __syncthreads();
    // ---- offsets: warp g scans minima [GROUP*g, GROUP*(g+1)) -------------
    {
        unsigned long long carry = 0;
#pragma unroll
        for (int c = 0; c < GROUP / 32; c++) {
            const int32_t i = GROUP * warp + 32 * c + lane;
            const int32_t L = i < cnt ? S.off[i] : 0;
            const unsigned long long inc = warp_incl_scan((unsigned long long)(uint32_t)L, lane);
            if (i < cnt) S.off[i] = (int32_t)(carry + inc - (unsigned long long)(uint32_t)L);
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) S.warp_tot[warp] = carry;
    }
    __syncthreads();
    auto group_base = [&](int32_t i) -> int32_t {
        unsigned long long b = 0;
        for (int q = 0; q < i / GROUP; q++) b += S.warp_tot[q];
        return (int32_t)b;
    };
    // ---- list the polygons into the shared buffer, two per thread --------
    // a thread visits the same minima here and below (i = tid + 256*it);
    // bit it of `over` marks a polygon that runs past the buffer
    uint32_t over = 0;
    {
        int it = 0;
        for (int32_t c0 = threadIdx.x; c0 < cnt; c0 += 2 * POLY_THREADS, it += 2) {
            const int32_t c1 = c0 + POLY_THREADS;
            int32_t e0 = -1, e1 = -1;
            int32_t k0 = S.off[c0] + group_base(c0), k1 = 0;
            if (k0 >= POLY_BUF) over |= 1u << it;
            else e0 = tb + S.mn[c0];
            if (c1 < cnt) {
                k1 = S.off[c1] + group_base(c1);
                if (k1 >= POLY_BUF) over |= 2u << it;
                else e1 = tb + S.mn[c1];
            }
            int32_t x0 = e0, x1 = e1;
            bool a0 = e0 >= 0, a1 = e1 >= 0;
            while (a0 || a1) {
                if (a0) {
                    S.he[k0] = x0;
                    S.v[k0] = __ldg(m.origin + x0);
                    k0++;
                    x0 = next_of(x0);
                    a0 = x0 != e0 && k0 < POLY_BUF;
                    if (!a0 && x0 != e0) over |= 1u << it;
                }
                if (a1) {
                    S.he[k1] = x1;
                    S.v[k1] = __ldg(m.origin + x1);
                    k1++;
                    x1 = next_of(x1);
                    a1 = x1 != e1 && k1 < POLY_BUF;
                    if (!a1 && x1 != e1) over |= 2u << it;
                }
            }
        }
    }
    // ---- seeds and offsets (coalesced), overflow entries ------------------
    {
        int it = 0;
        for (int32_t c0 = threadIdx.x; c0 < cnt; c0 += 2 * POLY_THREADS, it += 2) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int32_t i = c0 + h * POLY_THREADS;
                if (i >= cnt) continue;
                const int32_t lo = S.off[i] + group_base(i);
                const int32_t e = tb + S.mn[i];
                w.seeds[P0 + i] = e;
                w.offsets[P0 + i] = O0 + lo;
                if ((over >> (it + h)) & 1u) {
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
        }
    }
    __syncthreads();
    const int32_t nbuf = min(tile_len, POLY_BUF);
    for (int32_t k = threadIdx.x; k < nbuf; k += POLY_THREADS) {
        w.he_list[O0 + k] = S.he[k];
        w.v_list[O0 + k] = S.v[k];
    }
}

int polygons_configure() {
    return cudaFuncSetAttribute(k_poly_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(EmitSmem)) == cudaSuccess ? 0 : -1;
}

void launch_poly_count(const MeshView &m, const Work &w, cudaStream_t s) {
    k_poly_count<<<w.n_tiles, POLY_THREADS, 0, s>>>(m, w);
}

void launch_tile_scan(const MeshView &m, const Work &w, cudaStream_t s) {
    k_tile_scan<<<1, SCAN_THREADS, 0, s>>>(m, w);
}

void launch_poly_emit(const MeshView &m, const Work &w, cudaStream_t s) {
    k_poly_emit<<<w.n_tiles, POLY_THREADS, sizeof(EmitSmem), s>>>(m, w);
}

}  // namespace polylla
