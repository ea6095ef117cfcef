// Output kernels (stages 5b-5d): find every polygon, key it by its smallest
// half-edge, and write the scan-compacted CSR in ascending seed order.
//
// A frontier half-edge e is its polygon's minimum iff walking next from e
// comes back to e without meeting a smaller half-edge.  A minimum is smaller
// than both its neighbours along the polygon, so only half-edges carrying
// the relink's walk-start mark (next and prev both larger, a superset kept
// by the repair) walk; polygons are listed in an order that rises and then
// falls, so that is about one walk per polygon on the workloads measured.
// This finds every cycle of the relink exactly once, keyed by the canonical
// seed the paper's Algorithm 14 keeps, without a seed list.
//
// The walks are chains of dependent loads, so the kernels are organised
// for the largest number of chains in flight and no block ever waits for
// the slowest walk of its tile:
//   k_cand_count  marks per block of 16384 triangles        (flags, int4 loads)
//   k_scan_blocks exclusive scan of those counts            (one block)
//   k_cand_write  the walk starts, in index order           (scan-compaction)
//   k_walk        one chain per lane, grid-stride, two chains interleaved;
//                 (polygon count, length) per 32 starts, and per
//                 2048-start chunk by per-warp atomics
//   k_scan_blocks exclusive scan of the chunk totals -> P, N_F, offsets[P]
//   k_emit        per warp and 64 starts: offsets by warp scan over the
//                 chunk prefix and the group totals before it; every
//                 minimum writes its seed and offset and lists its polygon
//                 (two interleaved per lane) through a per-warp shared
//                 buffer that goes out with coalesced stores.
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

// The walk starts of 16 triangles t0 .. t0+15 as four words: byte q of
// word i holds the start bits of triangle t0 + 4i + q in its low 3 bits
// (a start is frontier and marked: f & (f >> 3) & 7 per flags byte, done
// on four bytes at once; bits shifted in from the next byte are masked).
// flags is allocated to a multiple of 16 bytes: the int4 stays in bounds.
__device__ __forceinline__ void start_words(const MeshView &m, const Work &w, int32_t t0, uint32_t st[4]) {
    st[0] = st[1] = st[2] = st[3] = 0u;
    if (t0 >= m.T) return;
    const int4 v = *reinterpret_cast<const int4 *>(w.flags + t0);
    const uint32_t wd[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
    for (int i = 0; i < 4; i++) st[i] = wd[i] & (wd[i] >> 3) & 0x07070707u;
    const int32_t valid = m.T - t0;  // triangles of the 16 inside [0, T)
    if (valid < 16) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int32_t keep = valid - 4 * i;  // bytes of word i to keep
            if (keep <= 0) st[i] = 0u;
            else if (keep < 4) st[i] &= (1u << (8 * keep)) - 1u;
        }
    }
}

// ===========================================================================
// k_cand_count: walk starts per block of CC_TRI triangles; also zeroes the
// chunk totals the walk kernel accumulates into.
// ===========================================================================
__global__ void __launch_bounds__(CC_THREADS) k_cand_count(MeshView m, Work w) {
    __shared__ unsigned long long s_warp[33];
    const int32_t gtid = blockIdx.x * CC_THREADS + threadIdx.x;
    for (int32_t i = gtid; i < w.n_chunk_max; i += gridDim.x * CC_THREADS) w.blk_b[i] = 0ull;
    const int32_t t0 = blockIdx.x * CC_TRI + threadIdx.x * CC_PER;  // 16 triangles per thread
    uint32_t st[4];
    start_words(m, w, t0, st);
    const uint32_t c = __popc(st[0]) + __popc(st[1]) + __popc(st[2]) + __popc(st[3]);
    unsigned long long total;
    block_excl_scan(c, s_warp, &total);
    if (threadIdx.x == 0) w.blk_a[blockIdx.x] = total;
}

// ===========================================================================
// k_scan_blocks: one block, exclusive scan of n (read from *n_dev when n < 0)
// 64-bit totals; *grand receives the sum.  Rounds of blockDim.x coalesced
// entries with a running carry.  With finish set (the chunk totals), thread
// 0 then turns the grand total into P, N_F and offsets[P].
// ===========================================================================
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_blocks(const unsigned long long *in, unsigned long long *out,
                                                              int32_t n, const int32_t *n_dev, int32_t n_max,
                                                              unsigned long long *grand, MeshView m, Work w,
                                                              int finish) {
    __shared__ unsigned long long s_warp[33];
    if (n < 0) n = min(*n_dev, n_max);
    unsigned long long carry = 0;
    for (int32_t b = 0; b < n; b += SCAN_THREADS) {
        const int32_t i = b + threadIdx.x;
        const unsigned long long v = i < n ? in[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_excl_scan(v, s_warp, &total);
        if (i < n) out[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x != 0) return;
    *grand = carry;
    if (!finish) return;
    int32_t P = (int32_t)(carry >> 32);
    const int64_t NF = (int64_t)(carry & 0xffffffffu);
    if (P > m.T || NF > 3 * (int64_t)m.T) {
        atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        P = P > m.T ? m.T : P;
    }
    w.offsets[P] = (int32_t)NF;
    w.ctrl->n_polygons = P;
    w.ctrl->n_frontier = (int32_t)NF;
    if (w.input_err && *w.input_err) atomicOr(&w.ctrl->error, DEV_ERR_INPUT);
}

// ===========================================================================
// k_cand_write: the walk starts of each block, in index order, at the
// block's scanned offset, staged in shared memory and stored coalesced.  Also stores the start count and the number of
// 2048-start chunks for the kernels that follow.
// ===========================================================================
__global__ void __launch_bounds__(CC_THREADS) k_cand_write(MeshView m, Work w) {
    __shared__ unsigned long long s_warp[33];
    __shared__ __align__(16) int32_t s_out[CW_BUF];
    const int32_t t0 = blockIdx.x * CC_TRI + threadIdx.x * CC_PER;
    uint32_t st[4];
    start_words(m, w, t0, st);
    const uint32_t c = __popc(st[0]) + __popc(st[1]) + __popc(st[2]) + __popc(st[3]);
    unsigned long long total;
    const int32_t ex = (int32_t)block_excl_scan(c, s_warp, &total);
    const int64_t base = (int64_t)w.blk_a_pre[blockIdx.x];
    const int32_t cap = 3 * m.T;
    // the block's starts go to shared memory in order, then out with
    // coalesced stores; any past the buffer (more than CW_BUF starts in one
    // block, not seen on the workloads measured) go out directly
    int32_t k = ex;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint32_t bits = st[i];
        while (bits) {
            const int b = __ffs(bits) - 1;  // byte q = b / 8 (triangle t0 + 4i + q), corner k = b % 8
            bits &= bits - 1u;
            const int32_t e = 3 * (t0 + 4 * i + (b >> 3)) + (b & 7);
            if (k < CW_BUF) s_out[k] = e;
            else if (base + k < cap) w.cand[base + k] = e;
            k++;
        }
    }
    __syncthreads();
    const int32_t nb = min((int32_t)total, CW_BUF);
    for (int32_t i = threadIdx.x; i < nb; i += CC_THREADS)
        if (base + i < cap) w.cand[base + i] = s_out[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t nc = (int64_t)w.ctrl->n_cand64;  // written by the scan of the block counts
        if (nc > cap) {
            atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            nc = cap;
        }
        w.ctrl->n_cand = (int32_t)nc;
        w.ctrl->n_chunks = (int32_t)((nc + CHUNK - 1) / CHUNK);
    }
}

// ===========================================================================
// k_walk: every start walks next until a smaller half-edge (not a minimum)
// or back to itself (a minimum: res = polygon length).  Grid-stride, one
// chain per lane, two chains per thread interleaved, no block barrier.  The
// 32 starts of a warp form one group, whose (minimum count, length) the warp
// stores, and lie in one 2048-start chunk, whose total it adds with one
// atomic.
// ===========================================================================
__global__ void __launch_bounds__(WALK_THREADS) k_walk(MeshView m, Work w) {
    const int32_t HI = 3 * m.T;
    const int32_t nc = w.ctrl->n_cand;
    const int32_t G = gridDim.x * WALK_THREADS;
    const int lane = threadIdx.x & 31;
    // warp-uniform loop bounds: every lane of a warp runs the same rounds
    const int32_t first = blockIdx.x * WALK_THREADS + (threadIdx.x & ~31);
    for (int32_t b0 = first; b0 < nc; b0 += 2 * G) {
        const int32_t i0 = b0 + lane;
        const int32_t i1 = b0 + G + lane;
        const bool h0 = i0 < nc, h1 = i1 < nc;
        const int32_t e0 = h0 ? w.cand[i0] : 0;
        const int32_t e1 = h1 ? w.cand[i1] : 0;
        int32_t x0 = h0 ? m.next[e0] : -1;  // -1 < e: chain idle
        int32_t x1 = h1 ? m.next[e1] : -1;
        int32_t L0 = 1, L1 = 1, guard = 0;
        while (x0 > e0 || x1 > e1) {
            if (x0 > e0) { x0 = m.next[x0]; L0++; }
            if (x1 > e1) { x1 = m.next[x1]; L1++; }
            if (++guard > HI) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                x0 = -1;
                x1 = -1;
                break;
            }
        }
        const int32_t r0 = (h0 && x0 == e0) ? L0 : 0;
        const int32_t r1 = (h1 && x1 == e1) ? L1 : 0;
        if (h0) w.res[i0] = r0;
        if (h1) w.res[i1] = r1;
        const unsigned long long p0 = r0 > 0 ? ((1ull << 32) | (uint32_t)r0) : 0ull;
        const unsigned long long p1 = r1 > 0 ? ((1ull << 32) | (uint32_t)r1) : 0ull;
        const unsigned long long s0 = warp_sum(p0);
        const unsigned long long s1 = warp_sum(p1);
        if (lane == 0) {
            if (b0 < nc) w.grp[b0 / 32] = s0;
            if (b0 + G < nc) w.grp[(b0 + G) / 32] = s1;
            if (s0 && b0 < nc) atomicAdd(&w.blk_b[b0 / CHUNK], s0);
            if (s1 && b0 + G < nc) atomicAdd(&w.blk_b[(b0 + G) / CHUNK], s1);
        }
    }
}

// ===========================================================================
// k_emit: grid-stride over groups of 64 starts, one warp each (two starts
// per lane).  A warp scan of the (count, length) pairs, plus the chunk's
// scanned total and the 32-start group totals of the chunk before this
// group, gives every minimum its polygon index and offset; no block
// barrier, so a long polygon holds up its own warp only.  Each lane lists
// its polygons from the minimum along next, interleaved, into the warp's
// shared buffer (entries past it go out directly); the warp then stores
// the buffer, one contiguous range of he_list and v_list, coalesced.
// ===========================================================================
__global__ void __launch_bounds__(EMIT_THREADS) k_emit(MeshView m, Work w) {
    __shared__ int32_t s_he[EMIT_THREADS / 32][EMIT_BUF];
    __shared__ int32_t s_v[EMIT_THREADS / 32][EMIT_BUF];
    static_assert(CHUNK % 64 == 0, "groups of 64 starts do not straddle chunks");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t HI = 3 * m.T;
    const int32_t nc = w.ctrl->n_cand;
    const int32_t n_sg = (nc + 63) / 64;
    const int32_t nwarps = gridDim.x * (EMIT_THREADS / 32);
    int32_t *bhe = s_he[wid];
    int32_t *bv = s_v[wid];
    for (int32_t sg = blockIdx.x * (EMIT_THREADS / 32) + wid; sg < n_sg; sg += nwarps) {
        const int32_t c0 = sg * 64 + 2 * lane;
        int32_t L0 = 0, L1 = 0;
        if (c0 + 1 < nc) {
            const int2 r = *reinterpret_cast<const int2 *>(w.res + c0);  // c0 is even: 8-byte aligned
            L0 = r.x;
            L1 = r.y;
        } else if (c0 < nc) {
            L0 = w.res[c0];
        }
        const unsigned long long q0 = L0 > 0 ? ((1ull << 32) | (uint32_t)L0) : 0ull;
        const unsigned long long q1 = L1 > 0 ? ((1ull << 32) | (uint32_t)L1) : 0ull;
        const unsigned long long inc = warp_incl_scan(q0 + q1, lane);
        const unsigned long long ex = inc - (q0 + q1);
        const unsigned long long tot = __shfl_sync(0xffffffffu, inc, 31);
        // groups of 32 starts [g0, gs) precede this one in its chunk (< 64)
        const int32_t ch = (sg * 64) / CHUNK;
        const int32_t g0 = ch * (CHUNK / 32), gs = 2 * sg;
        unsigned long long u = 0;
        if (g0 + lane < gs) u += w.grp[g0 + lane];
        if (g0 + 32 + lane < gs) u += w.grp[g0 + 32 + lane];
        const unsigned long long base = w.blk_b_pre[ch] + warp_sum(u);
        const int32_t O0 = (int32_t)(base & 0xffffffffu);
        const int32_t len = (int32_t)(tot & 0xffffffffu);
        if ((int64_t)(base >> 32) + (int64_t)(tot >> 32) > (int64_t)m.T || (int64_t)O0 + len > (int64_t)HI) {
            if (lane == 0) atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
            continue;  // warp-uniform
        }
        int32_t ea = -1, ka = 0, eb = -1, kb = 0;  // offsets within the group's range
        if (L0 > 0) {
            const unsigned long long r = base + ex;
            ea = w.cand[c0];
            ka = (int32_t)(ex & 0xffffffffu);
            w.seeds[(int32_t)(r >> 32)] = ea;
            w.offsets[(int32_t)(r >> 32)] = (int32_t)(r & 0xffffffffu);
        }
        if (L1 > 0) {
            const unsigned long long r = base + ex + q0;
            eb = w.cand[c0 + 1];
            kb = (int32_t)((ex + q0) & 0xffffffffu);
            w.seeds[(int32_t)(r >> 32)] = eb;
            w.offsets[(int32_t)(r >> 32)] = (int32_t)(r & 0xffffffffu);
        }
        // in a batch, lists are written in the mesh's own indices
        int32_t she_a = 0, sv_a = 0, she_b = 0, sv_b = 0;
        if (w.loc_n > 0) {
            if (ea >= 0) {
                const int32_t i = seg_of(w.loc_t_off, w.loc_n, ea / 3);
                she_a = 3 * __ldg(w.loc_t_off + i);
                sv_a = __ldg(w.loc_v_off + i);
            }
            if (eb >= 0) {
                const int32_t i = seg_of(w.loc_t_off, w.loc_n, eb / 3);
                she_b = 3 * __ldg(w.loc_t_off + i);
                sv_b = __ldg(w.loc_v_off + i);
            }
        }
        int32_t xa = ea, xb = eb, guard = 0;
        bool a = ea >= 0, b = eb >= 0;
        while (a || b) {
            if (a) {
                const int32_t va = __ldg(m.origin + xa) - sv_a;
                if (ka < EMIT_BUF) {
                    bhe[ka] = xa - she_a;
                    bv[ka] = va;
                } else {
                    w.he_list[O0 + ka] = xa - she_a;
                    w.v_list[O0 + ka] = va;
                }
                ka++;
                xa = m.next[xa];
                a = xa != ea;
            }
            if (b) {
                const int32_t vb = __ldg(m.origin + xb) - sv_b;
                if (kb < EMIT_BUF) {
                    bhe[kb] = xb - she_b;
                    bv[kb] = vb;
                } else {
                    w.he_list[O0 + kb] = xb - she_b;
                    w.v_list[O0 + kb] = vb;
                }
                kb++;
                xb = m.next[xb];
                b = xb != eb;
            }
            if (++guard > HI) break;
        }
        __syncwarp();
        const int32_t nb = min(len, EMIT_BUF);
        for (int32_t k = lane; k < nb; k += 32) {
            w.he_list[O0 + k] = bhe[k];
            w.v_list[O0 + k] = bv[k];
        }
        __syncwarp();  // the buffer is reused by the warp's next group
    }
}

void launch_scan_u64(const unsigned long long *in, unsigned long long *out, int32_t n, unsigned long long *grand,
                     cudaStream_t s) {
    k_scan_blocks<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, 0, grand, MeshView{}, Work{}, 0);
}

int polygons_configure() { return 0; }

int emit_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_emit, EMIT_THREADS, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

void launch_cand_count(const MeshView &m, const Work &w, cudaStream_t s) {
    k_cand_count<<<w.n_cc_blocks, CC_THREADS, 0, s>>>(m, w);
}

void launch_cand_scan(const MeshView &m, const Work &w, cudaStream_t s) {
    k_scan_blocks<<<1, SCAN_THREADS, 0, s>>>(w.blk_a, w.blk_a_pre, w.n_cc_blocks, nullptr, 0,
                                             &w.ctrl->n_cand64, m, w, 0);
}

void launch_cand_write(const MeshView &m, const Work &w, cudaStream_t s) {
    k_cand_write<<<w.n_cc_blocks, CC_THREADS, 0, s>>>(m, w);
}

void launch_walk(const MeshView &m, const Work &w, cudaStream_t s) {
    k_walk<<<w.walk_blocks, WALK_THREADS, 0, s>>>(m, w);
}

void launch_chunk_scan(const MeshView &m, const Work &w, cudaStream_t s) {
    k_scan_blocks<<<1, SCAN_THREADS, 0, s>>>(w.blk_b, w.blk_b_pre, -1, &w.ctrl->n_chunks, w.n_chunk_max,
                                             &w.ctrl->grand_b, m, w, 1);
}

void launch_emit(const MeshView &m, const Work &w, cudaStream_t s) {
    k_emit<<<w.emit_blocks, EMIT_THREADS, 0, s>>>(m, w);
}

}  // namespace polylla
