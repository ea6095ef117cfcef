// Label-phase kernels: mesh layout check, longest edge per triangle
// (stage 1), and the fused frontier / seed / relink pass (stages 2-4).
#include "polylla_internal.cuh"

namespace polylla {

// ===========================================================================
// Layout check (create only).  One thread per half-edge; any violation sets
// *bad.  Checks the contract the hot path relies on instead of re-reading
// next/prev: the implicit triangle layout of interior half-edges, a twin
// involution without fixed points, consistent border links, indices in
// range, target consistency and finite coordinates.
// ===========================================================================
__global__ void k_validate(MeshView m, int32_t *bad) {
    const int32_t HI = 3 * m.T;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t fail = 0;
    if (i < m.V) {
        double2 p = m.xy[i];
        fail |= !isfinite(p.x) || !isfinite(p.y);
    }
    if (i < m.H) {
        int32_t e = (int32_t)i;
        int32_t t = m.twin[e];
        int32_t o = m.origin[e];
        int32_t n = m.next[e];
        int32_t p = m.prev[e];
        fail |= t < 0 || t >= m.H || t == e;
        fail |= o < 0 || o >= m.V;
        fail |= n < 0 || n >= m.H || p < 0 || p >= m.H;
        if (!fail) {
            fail |= m.twin[t] != e;
            fail |= m.prev[n] != e;
            // target(e) = origin(twin e) = origin(next e)
            fail |= m.origin[n] != m.origin[t];
            if (e < HI) {
                fail |= n != nx_of(e) || p != pv_of(e);
            } else {
                fail |= t >= HI || n < HI || p < HI;
            }
        }
    }
    if (fail) atomicOr(bad, 1);
}

void launch_validate(const MeshView &m, int32_t *bad, cudaStream_t s) {
    int64_t n = m.H > m.V ? m.H : m.V;
    int blocks = (int)((n + 255) / 256);
    k_validate<<<blocks, 256, 0, s>>>(m, bad);
}

// ===========================================================================
// Stage 1: longest edge of each triangle (Algorithm 2 / Algorithm 8).
//
// The reference value is the float64 squared length
//     d = fl(fl(dx*dx) + fl(dy*dy)),  dx = fl(xb - xa),  dy = fl(yb - ya),
// and the longest edge is the largest d, equal d going to the smaller edge id
// min(e, twin e).  GB300 issues float64 at a small fraction of its float32
// rate, so the argmax is first decided by a certified float32 filter and
// only triangles the filter cannot decide take the float64 path.
//
// Filter.  Each coordinate x is truncated to float32 (x^ keeps the top 23
// significand bits, so |x^ - x| <= 2^-23 |x| = 2u|x| with u = 2^-24, and
// |x^| <= |x|) by bit manipulation (no float64 instruction); coordinates
// outside [2^-126, 2^61) in magnitude (zero included) send the triangle to
// the float64 path.  With S = |x^a| + |x^b| the float32 difference
// dx^ = fl32(x^b - x^a) satisfies |dx^ - dx| <= 3.0001 u Sx, hence
//   |D^ - d| <= 6.0003u (Sx|dx^| + Sy|dy^|) + 9.0007u^2 (Sx^2 + Sy^2)
//               + 2.0002u D^ + (float64 rounding of d, < 2^-50 d)
// where D^ = fl32(fl32(dx^ dx^) + fl32(dy^ dy^)).  The bound used,
//   B = 6.1u m1 + 9.1u^2 m2 + 4.5u D^ + 2^-118,
// adds 2.5u D^ for the rounding of the final comparison and an absolute
// term for float32 underflow.  If D^max - Bmax > D^j + Bj for the other two
// edges, the float64 argmax is the same edge and has no tie.
// ===========================================================================

struct EdgeF32 {
    float d;   // D^
    float b;   // error bound B
};

__device__ __forceinline__ EdgeF32 edge_f32(float ax, float ay, float bx, float by) {
    const float u = 5.9604644775390625e-08f;  // 2^-24
    float dx = __fsub_rn(bx, ax);
    float dy = __fsub_rn(by, ay);
    float sx = __fadd_rn(fabsf(ax), fabsf(bx));
    float sy = __fadd_rn(fabsf(ay), fabsf(by));
    EdgeF32 r;
    r.d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    float m1 = fmaf(sx, fabsf(dx), sy * fabsf(dy));
    float m2 = fmaf(sx, sx, sy * sy);
    r.b = fmaf(6.1f * u, m1, fmaf(9.1f * u * u, m2, fmaf(4.5f * u, r.d, 3.0e-36f)));
    return r;
}

__device__ __forceinline__ double sq_len_f64(double2 a, double2 b) {
    double dx = __dsub_rn(b.x, a.x);
    double dy = __dsub_rn(b.y, a.y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// the exact float64 argmax; tw0..tw2 are the twins of e0, e0 + 1, e0 + 2
// (equal lengths go to the smaller edge id min(e, twin e))
__device__ __noinline__ uint32_t longest_exact(double2 p0, double2 p1, double2 p2, int32_t e0, int32_t tw0,
                                               int32_t tw1, int32_t tw2) {
    double d0 = sq_len_f64(p0, p1);
    double d1 = sq_len_f64(p1, p2);
    double d2 = sq_len_f64(p2, p0);
    double d[3] = {d0, d1, d2};
    const int32_t tw[3] = {tw0, tw1, tw2};
    uint32_t best = 0;
#pragma unroll
    for (uint32_t k = 1; k < 3; k++) {
        if (d[k] > d[best]) {
            best = k;
        } else if (d[k] == d[best]) {
            int32_t ek = e0 + (int32_t)k, eb = e0 + (int32_t)best;
            int32_t tk = tw[k], tb = tw[best];
            int32_t ik = ek < tk ? ek : tk;
            int32_t ib = eb < tb ? eb : tb;
            if (ik < ib) best = k;
        }
    }
    return best;
}

// TW: the twins of the triangle's half-edges for the exact path, as
// tw(k) (read only when the filter cannot decide)
template <typename TW>
__device__ __forceinline__ uint32_t longest_of(double2 p0, double2 p1, double2 p2, int32_t e0, TW tw) {
    uint32_t bad = 0;
    const float x0 = trunc_to_f32(p0.x, bad), y0 = trunc_to_f32(p0.y, bad);
    const float x1 = trunc_to_f32(p1.x, bad), y1 = trunc_to_f32(p1.y, bad);
    const float x2 = trunc_to_f32(p2.x, bad), y2 = trunc_to_f32(p2.y, bad);
    const EdgeF32 g0 = edge_f32(x0, y0, x1, y1);
    const EdgeF32 g1 = edge_f32(x1, y1, x2, y2);
    const EdgeF32 g2 = edge_f32(x2, y2, x0, y0);
    uint32_t k;
    float dm, bm, dA, bA, dB, bB;
    if (g0.d >= g1.d && g0.d >= g2.d) {
        k = 0; dm = g0.d; bm = g0.b; dA = g1.d; bA = g1.b; dB = g2.d; bB = g2.b;
    } else if (g1.d >= g2.d) {
        k = 1; dm = g1.d; bm = g1.b; dA = g0.d; bA = g0.b; dB = g2.d; bB = g2.b;
    } else {
        k = 2; dm = g2.d; bm = g2.b; dA = g0.d; bA = g0.b; dB = g1.d; bB = g1.b;
    }
    const float lo = __fsub_rn(dm, bm);
    const bool sure = !bad && lo > __fadd_rn(dA, bA) && lo > __fadd_rn(dB, bB);
    if (!sure) k = longest_exact(p0, p1, p2, e0, tw(0), tw(1), tw(2));
    return k;
}

// Persistent warps walk tiles of 32 PER triangles.  Each warp owns a
// two-stage shared-memory ring: lane 0 bulk-copies (TMA engine,
// cp.async.bulk + mbarrier) the origin triples of the warp's next tile while
// the warp computes the current one, so the HBM stream of origin never waits
// on the coordinate gathers and no warp waits for another (no block
// barrier).  Each lane takes PER triangles (lane, lane + 32, ..., so a
// warp's gathers and byte stores stay contiguous) and issues their 3 PER
// coordinate loads together.
template <int PER>
__global__ void __launch_bounds__(LE_THREADS) k_longest_edge(MeshView m, Work w) {
    constexpr int NW = LE_THREADS / 32;
    constexpr int LE_TILE = 32 * PER;
    __shared__ __align__(128) int32_t s_org[NW][2][3 * LE_TILE];
    __shared__ __align__(8) uint64_t s_bar[NW][2];
    // reset this generate's control block (error word, tip count, totals)
    // and the output tiles' totals
    const int32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gtid < (int32_t)(sizeof(DevCtrl) / sizeof(int32_t))) reinterpret_cast<int32_t *>(w.ctrl)[gtid] = 0;
    for (int32_t i = gtid; i < w.n_tile_max; i += gridDim.x * blockDim.x) w.tile_state[i] = 0ull;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t n_tiles = (m.T + LE_TILE - 1) / LE_TILE;
    uint64_t *bar = s_bar[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    // the copy rounds the tail up to 16 bytes: at most 3 ints past 3T,
    // inside origin because H >= 3T + 3 (checked at create)
    auto issue = [&](int32_t tile, int st) {
        const int32_t t0 = tile * LE_TILE;
        const int32_t nt = min(LE_TILE, m.T - t0);
        const uint32_t bytes = ((uint32_t)(12 * nt) + 15u) & ~15u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[st], bytes);
        bulk_load(s_org[warp][st], m.origin + 3 * (int64_t)t0, bytes, &bar[st]);
    };
    const int32_t nwarps = gridDim.x * NW;
    int32_t tile = blockIdx.x * NW + warp;
    if (lane == 0 && tile < n_tiles) issue(tile, 0);
    uint32_t parity = 0u;  // bit st = parity to wait for on stage st
    for (int it = 0; tile < n_tiles; it++, tile += nwarps) {
        const int st = it & 1;
        const int32_t nxt = tile + nwarps;
        if (lane == 0 && nxt < n_tiles) issue(nxt, st ^ 1);
        const bool ok = mbar_wait(&bar[st], (parity >> st) & 1u);
        if (__any_sync(0xffffffffu, !ok)) {
            // give up: record it, wait (bounded) for this warp's copies in
            // flight so no bulk copy lands after the warp has left, return
            if (lane == 0) atomicOr(&w.ctrl->error, DEV_ERR_TIMEOUT);
            mbar_wait(&bar[st], (parity >> st) & 1u);
            if (nxt < n_tiles) mbar_wait(&bar[st ^ 1], (parity >> (st ^ 1)) & 1u);
            return;
        }
        parity ^= 1u << st;
        const int32_t t0 = tile * LE_TILE;
        const int32_t *so = s_org[warp][st];
        double2 p[PER][3];
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int32_t lt = lane + 32 * q;
            if (t0 + lt < m.T) {
                p[q][0] = __ldg(m.xy + so[3 * lt]);
                p[q][1] = __ldg(m.xy + so[3 * lt + 1]);
                p[q][2] = __ldg(m.xy + so[3 * lt + 2]);
            }
        }
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int32_t lt = lane + 32 * q;
            const int32_t t = t0 + lt;
            const int32_t *__restrict__ twin = m.twin + 3 * t;
            if (t < m.T)
                w.le[t] = (uint8_t)longest_of(p[q][0], p[q][1], p[q][2], 3 * t,
                                              [twin](int k) { return __ldg(twin + k); });
        }
        __syncwarp();  // stage st is refilled next iteration
    }
}

// ===========================================================================
// Stage 1 on a batch, straight from the meshes' own arrays (no packing
// pass).  Persistent warps with a two-stage ring as in k_longest_edge; a
// warp's tile of 32 PER triangles that lies inside one mesh has its origin
// and twin entries contiguous in the mesh's local arrays (local half-edge
// 3 (t - t_off) + k of triangle t of mesh j sits at h_off + 3 (t - t_off)
// + k), so lane 0 bulk-copies both from that start rounded down to 16
// bytes (r entries early) to 16 bytes past the end, which stays inside the
// mesh's entries since at least 3 border half-edges follow its interior
// ones.  A tile across meshes, or arrays that do not start on a 16-byte
// boundary, are read with plain loads.  The mesh comes from the batch's
// mesh table (the mesh of every 256th triangle).  Every origin and twin is
// range-checked against its mesh: an index outside it is replaced by one
// inside it (vertex 0; the mesh's first border half-edge, which stops
// rotations) and the run is flagged, so no later kernel reads outside the
// mesh.  Each lane writes its triangles' union twins (interior: 3 t_off +
// y; border: 3 T + b_off + (y - 3 T_j)), which the later stages walk, and
// the longest edge as on a single mesh, from the coordinates at the mesh's
// vertex offset.
// ===========================================================================
template <int PER>
__global__ void __launch_bounds__(LE_THREADS) k_longest_edge_batch(MeshView m, Work w) {
    constexpr int NW = LE_THREADS / 32;
    constexpr int LE_TILE = 32 * PER;
    constexpr int SPAN = 3 * LE_TILE + 4;  // a stage's entries, 4 to spare for an unaligned start
    static_assert(SPAN % 4 == 0, "stages start on 16-byte boundaries");
    __shared__ __align__(128) int32_t s_org[NW][2][SPAN];
    __shared__ __align__(128) int32_t s_tw[NW][2][SPAN];
    __shared__ __align__(8) uint64_t s_bar[NW][2];
    __shared__ int32_t s_r[NW][2], s_j[NW][2];  // per stage: start offset (-1: plain loads), mesh
    const int32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gtid < (int32_t)(sizeof(DevCtrl) / sizeof(int32_t))) reinterpret_cast<int32_t *>(w.ctrl)[gtid] = 0;
    for (int32_t i = gtid; i < w.n_tile_max; i += gridDim.x * blockDim.x) w.tile_state[i] = 0ull;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t HI = 3 * m.T;
    const int32_t n_tiles = (m.T + LE_TILE - 1) / LE_TILE;
    uint64_t *bar = s_bar[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int32_t tile, int st) {
        const int32_t t0 = tile * LE_TILE;
        const int32_t nt = min(LE_TILE, m.T - t0);
        const int32_t j = mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, t0);
        const int32_t t3 = 3 * __ldg(w.loc_t_off + j);
        const bool one = w.loc_aligned && 3 * __ldg(w.loc_t_off + j + 1) >= 3 * (t0 + nt);
        s_j[warp][st] = j;
        fence_proxy_async_smem();
        if (one) {
            const int32_t L0 = __ldg(w.loc_h_off + j) + (3 * t0 - t3);
            const int32_t r = L0 & 3;
            const uint32_t bytes = ((uint32_t)(r + 3 * nt) * 4u + 15u) & ~15u;
            s_r[warp][st] = r;
            mbar_arrive_expect_tx(&bar[st], 2 * bytes);
            bulk_load(s_org[warp][st], w.loc_origin + (L0 - r), bytes, &bar[st]);
            bulk_load(s_tw[warp][st], w.loc_twin + (L0 - r), bytes, &bar[st]);
        } else {
            s_r[warp][st] = -1;
            mbar_arrive_expect_tx(&bar[st], 0u);  // nothing to copy: the phase completes now
        }
    };
    const int32_t nwarps = gridDim.x * NW;
    int32_t tile = blockIdx.x * NW + warp;
    if (lane == 0 && tile < n_tiles) issue(tile, 0);
    uint32_t parity = 0u;
    bool bad = false;
    for (int it = 0; tile < n_tiles; it++, tile += nwarps) {
        const int st = it & 1;
        const int32_t nxt = tile + nwarps;
        if (lane == 0 && nxt < n_tiles) issue(nxt, st ^ 1);
        const bool ok = mbar_wait(&bar[st], (parity >> st) & 1u);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) atomicOr(&w.ctrl->error, DEV_ERR_TIMEOUT);
            mbar_wait(&bar[st], (parity >> st) & 1u);
            if (nxt < n_tiles) mbar_wait(&bar[st ^ 1], (parity >> (st ^ 1)) & 1u);
            return;
        }
        parity ^= 1u << st;
        const int32_t t0 = tile * LE_TILE;
        const int32_t r = s_r[warp][st];
        const int32_t *so = s_org[warp][st] + (r > 0 ? r : 0);
        const int32_t *stw = s_tw[warp][st] + (r > 0 ? r : 0);
        double2 p[PER][3];
        int32_t tw[PER][3];
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int32_t lt = lane + 32 * q;
            const int32_t t = t0 + lt;
            if (t >= m.T) continue;
            const int32_t j = r >= 0 ? s_j[warp][st] : mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, t);
            const int32_t t3 = 3 * __ldg(w.loc_t_off + j);
            const int32_t ti3 = 3 * __ldg(w.loc_t_off + j + 1) - t3;
            const int32_t h0 = __ldg(w.loc_h_off + j), hi = __ldg(w.loc_h_off + j + 1) - h0;
            const int32_t v0 = __ldg(w.loc_v_off + j), vi = __ldg(w.loc_v_off + j + 1) - v0;
            const int32_t g = h0 + (3 * t - t3);
            const int32_t bo = HI + (h0 - t3) - ti3;
            int32_t o[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                o[k] = r >= 0 ? so[3 * lt + k] : __ldg(w.loc_origin + g + k);
                tw[q][k] = r >= 0 ? stw[3 * lt + k] : __ldg(w.loc_twin + g + k);
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if ((uint32_t)o[k] >= (uint32_t)vi) { o[k] = 0; bad = true; }
                if ((uint32_t)tw[q][k] >= (uint32_t)hi) { tw[q][k] = ti3; bad = true; }
                tw[q][k] = tw[q][k] < ti3 ? t3 + tw[q][k] : bo + tw[q][k];
                w.u_twin[3 * t + k] = tw[q][k];
                p[q][k] = __ldg(m.xy + v0 + o[k]);
            }
        }
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int32_t t = t0 + lane + 32 * q;
            const int32_t *twq = tw[q];
            if (t < m.T)
                w.le[t] = (uint8_t)longest_of(p[q][0], p[q][1], p[q][2], 3 * t, [twq](int k) { return twq[k]; });
        }
        __syncwarp();  // stage st is refilled next iteration
    }
    if (bad) atomicOr(w.input_err, 1);
}

int longest_edge_blocks_per_sm(int32_t items) {
    int n = 0;
    const cudaError_t e = items == 4
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_longest_edge<4>, LE_THREADS, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_longest_edge<2>, LE_THREADS, 0);
    if (e != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

int longest_edge_batch_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_longest_edge_batch<2>, LE_THREADS, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

void launch_longest_edge(const MeshView &m, const Work &w, cudaStream_t s) {
    const int32_t tile = 32 * (w.le_items == 4 && w.loc_n == 0 ? 4 : 2);  // batches: 2 per lane
    const int32_t n_tiles = (m.T + tile - 1) / tile;
    const int32_t want = (n_tiles + LE_THREADS / 32 - 1) / (LE_THREADS / 32);  // one tile per warp
    const int32_t grid = w.loc_n > 0 ? w.le_batch_blocks : w.le_blocks;  // persistent: every CTA resident
    const int blocks = want < grid ? want : grid;
    // the control-block reset needs >= 8 threads: any grid >= 1 works
    if (w.loc_n > 0) k_longest_edge_batch<2><<<blocks, LE_THREADS, 0, s>>>(m, w);
    else if (w.le_items == 4) k_longest_edge<4><<<blocks, LE_THREADS, 0, s>>>(m, w);
    else k_longest_edge<2><<<blocks, LE_THREADS, 0, s>>>(m, w);
}


// ===========================================================================
// Stages 2-4 fused: frontier labels (Algorithm 3 / 9), seeds (Algorithm 4 /
// 10) and the relink of every frontier half-edge (Section 4.2; the per-half-
// edge form of Algorithm 12).  A CTA of NT threads takes NT * IPT
// consecutive triangles, IPT per thread (strided: triangle t0 + q NT + tid);
// with BATCH (a batch's union) it also writes every link in the meshes' own
// indices and arrays.
//
//   F0[e] = border(e) or (not LE[e] and not LE[twin e])
//   seed  = the triangle's longest half-edge e when it is the smaller half of
//           a terminal edge (LE[e] and LE[twin e]) or lies on the border
//   next[e] for frontier e: x = next(e); while not F0[x]: x = CW(x) =
//           next(twin x); then next[e] = x, prev[x] = e.  Non-frontier e get
//           their triangle links.  A rotation that comes back to twin(e)
//           means target(e) has one frontier edge: a barrier tip, recorded
//           with the frontier half-edge twin(e) leaving it.
//
// F0 of a half-edge in another triangle is evaluated on the fly from the
// longest-edge bytes (L2-resident) and that half-edge's twin, which the
// rotation loads anyway, so the twin array is read from HBM once and no
// frontier array is needed.  Twin values are split into (triangle, corner)
// once, so a rotation step costs one twin and one byte load, and the next
// step's twin is fetched together with the current step's byte.
// next and prev of the CTA's triangles are assembled in shared memory and
// stored coalesced; only prev[x] for an x outside them is stored directly.
// In place is race-free: the rotation reads only twin and le; each next[e]
// is written once (by e's thread, or by the lane that ran e's rotation) and
// each prev[x] once, for the unique e with next[e] = x (or by x's own
// thread when x is not frontier).
//
// Rotations are compacted per warp.  Each thread labels its triangles and
// links the frontier half-edges whose successor is the next half-edge of the
// same triangle; the others (the successor lies across a non-frontier edge)
// become tasks that the warp's lanes then take one each, so a warp runs its
// rotations side by side instead of once per local half-edge.  (Staging the
// CTA's twin and longest-edge bytes in shared memory by bulk copies measured
// slower: on row-major grids half of each vertex fan lies in the next row,
// outside any tile narrower than a row.)
// ===========================================================================
__device__ __forceinline__ int32_t div3(int32_t x) { return (int32_t)((uint32_t)x / 3u); }

template <int NT, int IPT, bool BATCH>
__global__ void __launch_bounds__(NT, 2048 / NT / IPT) k_label_relink(MeshView m, Work w) {
    constexpr int TT = NT * IPT;  // triangles per CTA
    static_assert(IPT >= 1 && IPT <= 4, "a thread's flag bytes fit one 32-bit word");
    __shared__ __align__(16) int32_t s_nx[3 * TT];
    __shared__ __align__(16) int32_t s_pv[3 * TT];
    __shared__ int4 s_task[NT / 32][96 * IPT];
    __shared__ int32_t s_m0;  // batches: the mesh of the CTA's first triangle
    const int32_t t0 = blockIdx.x * TT;
    const int32_t nT = min(TT, m.T - t0);
    const int32_t eb = 3 * t0;
    const int32_t nE = 3 * nT;
    const int32_t HI = 3 * m.T;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    if (BATCH && threadIdx.x == 0) s_m0 = mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, t0);
    uint32_t fls = 0;  // byte q: flags of triangle t0 + q NT + tid
    uint32_t total = 0;
#pragma unroll
    for (int q = 0; q < IPT; q++) {
        const int32_t lt = q * NT + (int32_t)threadIdx.x;
        const bool live = lt < nT;
        const int32_t t = t0 + lt;
        const int32_t e0 = 3 * t;
        const int32_t lb = 3 * lt;
        uint32_t pend = 0;
        int32_t tw[3], ttri[3];
        uint32_t tloc[3], lnb[3];
        if (live) {
            tw[0] = __ldg(m.twin + e0);
            tw[1] = __ldg(m.twin + e0 + 1);
            tw[2] = __ldg(m.twin + e0 + 2);
            const uint32_t ltl = w.le[t];
            uint32_t F = 0, twle = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const bool b = tw[k] >= HI;
                ttri[k] = b ? 0 : div3(tw[k]);
                tloc[k] = (uint32_t)(tw[k] - 3 * ttri[k]);
                lnb[k] = b ? 3u : (uint32_t)w.le[ttri[k]];
                const bool tl = !b && lnb[k] == tloc[k];
                F |= (uint32_t)(b || ((uint32_t)k != ltl && !tl)) << k;
                twle |= (uint32_t)tl << k;
            }
            const int32_t twl = ltl == 0u ? tw[0] : (ltl == 1u ? tw[1] : tw[2]);
            const bool seed = (twl >= HI) || (((twle >> ltl) & 1u) && (e0 + (int32_t)ltl) < twl);
            fls |= (F | ((uint32_t)seed << 6)) << (8 * q);
            // own slots: non-frontier half-edges keep their triangle links,
            // frontier ones wait for their predecessor (-1 until then)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int j = k == 2 ? 0 : k + 1;
                const bool f = (F >> k) & 1u;
                s_pv[lb + k] = f ? -1 : e0 + (k == 0 ? 2 : k - 1);
                if (!f || ((F >> j) & 1u)) s_nx[lb + k] = e0 + j;
                else pend |= 1u << k;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int j = k == 2 ? 0 : k + 1;
                if (((F >> k) & 1u) && ((F >> j) & 1u)) s_pv[lb + j] = e0 + k;  // successor in the triangle
            }
        }
        // compact the warp's pending rotations (the order of the tasks does
        // not matter: each writes its own slots)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const bool mine = (pend >> k) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const int j = k == 2 ? 0 : k + 1;
                s_task[wid][total + __popc(bal & below)] =
                    make_int4(e0 + k, tw[k], ttri[j], (int32_t)(tloc[j] | (lnb[j] << 2)));
            }
            total += __popc(bal);
        }
    }
    __syncthreads();  // every slot initialised before the rotations write prev
    for (uint32_t i = lane; i < total; i += 32) {
        const int4 tk = s_task[wid][i];
        const int32_t e = tk.x;
        int32_t ty = tk.z;
        uint32_t ly = (uint32_t)tk.w & 3u;
        uint32_t ley = ((uint32_t)tk.w >> 2) & 3u;
        uint32_t lx = ly == 2u ? 0u : ly + 1u;
        int32_t x = 3 * ty + (int32_t)lx;
        int32_t tx = __ldg(m.twin + x);
        int32_t steps = 0;
        while (true) {
            if (tx >= HI) break;                     // border edge: frontier
            const int32_t ttx = div3(tx);
            const uint32_t ltx = (uint32_t)(tx - 3 * ttx);
            const uint32_t lxn = ltx == 2u ? 0u : ltx + 1u;
            const int32_t xn = 3 * ttx + (int32_t)lxn;
            const uint32_t lex = w.le[ttx];
            const int32_t txn = __ldg(m.twin + xn);
            if (ley != lx && lex != ltx) break;      // neither half longest: frontier
            ley = lex;
            x = xn;
            lx = lxn;
            tx = txn;
            if (++steps > w.max_rot) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                break;
            }
        }
        s_nx[e - eb] = x;
        const uint32_t dx = (uint32_t)(x - eb);
        if (dx < (uint32_t)nE) s_pv[dx] = e;
        else {
            if (!BATCH) m.prev[x] = e;
            else {  // e, x lie in one mesh, at or after the CTA's first
                int32_t mj = s_m0;
                while (mj + 1 < w.loc_n && 3 * __ldg(w.loc_t_off + mj + 1) <= e) mj++;
                const int32_t sh = 3 * __ldg(w.loc_t_off + mj);
                w.loc_prev[__ldg(w.loc_h_off + mj) + (x - sh)] = e - sh;
            }
        }
        if (x == tk.y) {
            const int32_t sl = atomicAdd(&w.ctrl->n_tips, 1);
            if (sl < w.tip_cap) w.tips[sl] = tk.y;
            else atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        }
    }
    __syncthreads();
    // walk-start marks: frontier, next and prev larger (prev unknown: set
    // by another CTA, counted as larger)
#pragma unroll
    for (int q = 0; q < IPT; q++) {
        const int32_t lt = q * NT + (int32_t)threadIdx.x;
        if (lt >= nT) break;
        uint32_t fl = (fls >> (8 * q)) & 0xffu;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int32_t e = eb + 3 * lt + k;
            const int32_t pv = s_pv[3 * lt + k];
            if (((fl >> k) & 1u) && s_nx[3 * lt + k] > e && (pv < 0 || pv > e)) fl |= 8u << k;
        }
        w.flags[t0 + lt] = (uint8_t)fl;
    }
    int4 *dn = reinterpret_cast<int4 *>(m.next + eb);
    for (int i = threadIdx.x; 4 * i < nE; i += NT) {
        if (4 * i + 3 < nE) {
            dn[i] = reinterpret_cast<const int4 *>(s_nx)[i];
        } else {
            for (int c = 0; c < 4; c++)
                if (4 * i + c < nE) m.next[eb + 4 * i + c] = s_nx[4 * i + c];
        }
    }
    // (a batch's union prev is never read: its links go to the meshes' own
    // prev only)
    for (int i = threadIdx.x; i < nE && !BATCH; i += NT) {
        const int32_t v = s_pv[i];
        if (v >= 0) m.prev[eb + i] = v;
    }
    // in a batch, the links in the meshes' own indices and arrays (the CTA's
    // half-edges are consecutive in a mesh's local arrays between mesh
    // boundaries, so these stores stay coalesced)
    if (BATCH) {
        // mesh mj spans union half-edges [sh, nb); its local entry of union
        // x is x + gsh
        int32_t mj = s_m0;
        int32_t sh = 3 * __ldg(w.loc_t_off + mj);
        int32_t nb = 3 * __ldg(w.loc_t_off + mj + 1);
        int32_t gsh = __ldg(w.loc_h_off + mj) - sh;
        for (int i = threadIdx.x; i < nE; i += NT) {
            const int32_t x = eb + i;
            while (x >= nb && mj + 1 < w.loc_n) {
                mj++;
                sh = nb;
                nb = 3 * __ldg(w.loc_t_off + mj + 1);
                gsh = __ldg(w.loc_h_off + mj) - sh;
            }
            const int32_t g = x + gsh;
            w.loc_next[g] = s_nx[i] - sh;
            const int32_t v = s_pv[i];
            if (v >= 0) w.loc_prev[g] = v - sh;
        }
    }
}

// ===========================================================================
// Stages 2-4 fused, one triangle per thread (the same labels, seeds, links,
// tips and marks as k_label_relink).  A triangle's frontier half-edges form
// at most one cyclic run among its three (one run, or none, or all three),
// and only the last half-edge of a run has a successor across a
// non-frontier edge: a triangle has at most one rotation.  With one
// triangle per thread, each thread runs its own rotation: a warp's lanes
// run their rotations side by side without any task list, and every next
// entry of the CTA is set by its own thread.  prev goes through shared
// memory (a rotation sets prev[x] for an x of another thread), which also
// gives the walk-start marks their prev; each warp then stores the next and
// prev of its 32 triangles as contiguous, coalesced runs.
// ===========================================================================
template <int NT, bool BATCH>
__global__ void __launch_bounds__(NT, 2048 / NT) k_label_relink1(MeshView m, Work w) {
    static_assert(NT % 32 == 0, "whole warps");
    __shared__ int32_t s_pv[3 * NT];
    __shared__ int32_t s_nx[3 * NT];
    __shared__ int32_t s_m0;  // batches: the mesh of the CTA's first triangle
    const int32_t t0 = blockIdx.x * NT;
    const int32_t eb = 3 * t0;
    const int32_t nE = 3 * min(NT, m.T - t0);
    const int32_t HI = 3 * m.T;
    const int32_t lb = 3 * (int32_t)threadIdx.x;
    const int32_t t = t0 + (int32_t)threadIdx.x;
    const bool live = t < m.T;
    const int32_t e0 = 3 * t;
    if (BATCH && threadIdx.x == 0) s_m0 = mesh_of(w.loc_seg, w.loc_t_off, w.loc_n, t0);
    uint32_t F = 0, fl = 0;
    uint32_t kt = 3;          // the local index of the rotating half-edge (3: none)
    int32_t twk = 0;          // its twin (the rotation coming back to it finds a tip)
    int32_t ty = 0;           // the rotation: current half-edge 3 ty + lx, ley = le(ty)
    uint32_t lx = 0, ley = 0;
    if (live) {
        int32_t tw[3], ttri[3];
        uint32_t tloc[3], lnb[3];
        tw[0] = __ldg(m.twin + e0);
        tw[1] = __ldg(m.twin + e0 + 1);
        tw[2] = __ldg(m.twin + e0 + 2);
        const uint32_t ltl = w.le[t];
        uint32_t twle = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const bool b = tw[k] >= HI;
            ttri[k] = b ? 0 : div3(tw[k]);
            tloc[k] = (uint32_t)(tw[k] - 3 * ttri[k]);
            lnb[k] = b ? 3u : (uint32_t)w.le[ttri[k]];
            const bool tl = !b && lnb[k] == tloc[k];
            F |= (uint32_t)(b || ((uint32_t)k != ltl && !tl)) << k;
            twle |= (uint32_t)tl << k;
        }
        const int32_t twl = ltl == 0u ? tw[0] : (ltl == 1u ? tw[1] : tw[2]);
        const bool seed = (twl >= HI) || (((twle >> ltl) & 1u) && (e0 + (int32_t)ltl) < twl);
        fl = F | ((uint32_t)seed << 6);
        // prev of slot j: its triangle link when j is not frontier or its
        // predecessor in the triangle is frontier; else set by a rotation
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int k = j == 0 ? 2 : j - 1;
            s_pv[lb + j] = (!((F >> j) & 1u) || ((F >> k) & 1u)) ? e0 + k : -1;
        }
        // the frontier half-edge whose successor in the triangle is not
        // frontier: bit k of rot is F bit k + 1 (mod 3), so pend has one bit
        // at most (1, 2 or 4 -> k = pend >> 1)
        const uint32_t rot = ((F >> 1) | (F << 2)) & 7u;
        const uint32_t pend = F & ~rot;
        if (pend) {
            kt = pend >> 1;
            const uint32_t j = kt == 2u ? 0u : kt + 1u;
            twk = kt == 0u ? tw[0] : (kt == 1u ? tw[1] : tw[2]);
            ty = j == 0u ? ttri[0] : (j == 1u ? ttri[1] : ttri[2]);
            const uint32_t ly = j == 0u ? tloc[0] : (j == 1u ? tloc[1] : tloc[2]);
            ley = j == 0u ? lnb[0] : (j == 1u ? lnb[1] : lnb[2]);
            lx = ly == 2u ? 0u : ly + 1u;
        }
    }
    __syncthreads();  // every prev slot initialised before rotations write them
    int32_t mj = 0, sh = 0;  // batches: the thread's mesh and its first union half-edge
    if (BATCH && live) {
        mj = s_m0;
        while (mj + 1 < w.loc_n && __ldg(w.loc_t_off + mj + 1) <= t) mj++;
        sh = 3 * __ldg(w.loc_t_off + mj);
    }
    int32_t x = 3 * ty + (int32_t)lx;
    if (kt < 3u) {
        // x = CW(next e) = next(twin(next e)); while x is not frontier,
        // x = CW(x).  The next step's twin is fetched with this step's label.
        const int32_t e = e0 + (int32_t)kt;
        int32_t tx = __ldg(m.twin + x);
        int32_t steps = 0;
        while (true) {
            if (tx >= HI) break;                     // border edge: frontier
            const int32_t ttx = div3(tx);
            const uint32_t ltx = (uint32_t)(tx - 3 * ttx);
            const uint32_t lxn = ltx == 2u ? 0u : ltx + 1u;
            const int32_t xn = 3 * ttx + (int32_t)lxn;
            const uint32_t lex = w.le[ttx];
            const int32_t txn = __ldg(m.twin + xn);
            if (ley != lx && lex != ltx) break;      // neither half longest: frontier
            ley = lex;
            x = xn;
            lx = lxn;
            tx = txn;
            if (++steps > w.max_rot) {
                atomicOr(&w.ctrl->error, DEV_ERR_NONTERMINATING);
                break;
            }
        }
        const uint32_t dx = (uint32_t)(x - eb);
        if (dx < (uint32_t)nE) s_pv[dx] = e;
        else if (!BATCH) m.prev[x] = e;
        else w.loc_prev[__ldg(w.loc_h_off + mj) + (x - sh)] = e - sh;  // e, x lie in mesh mj
        if (x == twk) {
            const int32_t sl = atomicAdd(&w.ctrl->n_tips, 1);
            if (sl < w.tip_cap) w.tips[sl] = twk;
            else atomicOr(&w.ctrl->error, DEV_ERR_CAPACITY);
        }
    }
    __syncthreads();  // every prev slot is final
    // walk-start marks: frontier, next and prev larger (prev -1: set by
    // another CTA, counted as larger)
    if (live) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int32_t e = e0 + k;
            const int32_t nk = (uint32_t)k == kt ? x : e0 + (k == 2 ? 0 : k + 1);
            const int32_t pk = s_pv[lb + k];
            if (((F >> k) & 1u) && nk > e && (pk < 0 || pk > e)) fl |= 8u << k;
            s_nx[lb + k] = nk;
        }
        w.flags[t] = (uint8_t)fl;
    }
    __syncwarp();
    // each warp stores the links of its 96 half-edges in place, coalesced
    // (in a batch, also in the meshes' own indices and arrays; a batch's
    // union prev is never read, so it is not written)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t bj = BATCH ? s_m0 : 0;
    for (int i = lane; i < 96; i += 32) {
        const int32_t sl = 96 * wid + i;
        if (sl >= nE) break;
        const int32_t xe = eb + sl;
        const int32_t nv = s_nx[sl];
        const int32_t pv = s_pv[sl];
        m.next[xe] = nv;
        if (!BATCH) {
            if (pv >= 0) m.prev[xe] = pv;
        } else {
            while (bj + 1 < w.loc_n && 3 * __ldg(w.loc_t_off + bj + 1) <= xe) bj++;
            const int32_t shj = 3 * __ldg(w.loc_t_off + bj);
            const int32_t g = __ldg(w.loc_h_off + bj) + (xe - shj);
            w.loc_next[g] = nv - shj;
            if (pv >= 0) w.loc_prev[g] = pv - shj;
        }
    }
}

// launch configurations: (triangles per CTA, triangles per thread); one per
// thread runs k_label_relink1, more run k_label_relink
#define RELINK1_CONFIGS(X) \
    X(64)                  \
    X(128)                 \
    X(256)
#define RELINK_CONFIGS(X) \
    X(128, 2)             \
    X(64, 4)

bool relink_config_valid(int32_t tile, int32_t items) {
#define X(N) \
    if (tile == N && items == 1) return true;
    RELINK1_CONFIGS(X)
#undef X
#define X(N, I) \
    if (tile == N * I && items == I) return true;
    RELINK_CONFIGS(X)
#undef X
    return false;
}

int relink_configure() { return 0; }  // static shared memory only

void launch_label_relink(const MeshView &m, const Work &w, cudaStream_t s) {
#define X(N)                                                                         \
    if (w.rl_tile == N && w.rl_items == 1) {                                         \
        if (w.loc_n > 0) k_label_relink1<N, true><<<(m.T + N - 1) / N, N, 0, s>>>(m, w); \
        else k_label_relink1<N, false><<<(m.T + N - 1) / N, N, 0, s>>>(m, w);       \
        return;                                                                      \
    }
    RELINK1_CONFIGS(X)
#undef X
#define X(N, I)                                                                      \
    if (w.rl_tile == N * I && w.rl_items == I) {                                     \
        if (w.loc_n > 0) k_label_relink<N, I, true><<<(m.T + N * I - 1) / (N * I), N, 0, s>>>(m, w);  \
        else k_label_relink<N, I, false><<<(m.T + N * I - 1) / (N * I), N, 0, s>>>(m, w);        \
        return;                                                                      \
    }
    RELINK_CONFIGS(X)
#undef X
    if (w.loc_n > 0) k_label_relink1<128, true><<<(m.T + 127) / 128, 128, 0, s>>>(m, w);
    else k_label_relink1<128, false><<<(m.T + 127) / 128, 128, 0, s>>>(m, w);
}

}  // namespace polylla
