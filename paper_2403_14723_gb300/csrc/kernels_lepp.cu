// Longest-edge propagation paths (Definition 1, Section 3.1) as a device
// primitive over the longest edges of the last generate.  Section 1 lists a
// data-parallel Lepp among the paper's contributions, as a building block
// for Lepp-based refinement and optimisation.
//
// Lepp(t0) = t0, t1, ...: t_i is the neighbour of t_{i-1} across the longest
// edge of t_{i-1}; the path ends at the terminal edge, the longest edge of
// both of its triangles (both are listed), or at a longest edge on the
// border.  The terminal edge is reported by its seed half-edge: the smaller
// half of an interior terminal edge, the interior half of a border one.
// Every step is a dependent load of twin then of the neighbour's longest-
// edge byte; one thread per path.
#include "polylla_internal.cuh"

namespace polylla {

// one step bound: under the strict (length, edge id) order a path never
// revisits a triangle, so T + 1 steps are never reached on a valid mesh
__device__ __forceinline__ int32_t lepp_chase(const MeshView &m, const uint8_t *le, int32_t t, int32_t max_steps,
                                              int32_t *path, int64_t path_cap, int32_t *terminal, bool *ok) {
    const int32_t HI = 3 * m.T;
    int32_t n = 1;
    if (path && 0 < path_cap) path[0] = t;
    uint32_t l = le[t];
    for (;;) {
        const int32_t e = 3 * t + (int32_t)l;
        const int32_t tw = __ldg(m.twin + e);
        if (tw >= HI) {
            *terminal = e;
            break;
        }
        const int32_t t1 = (int32_t)((uint32_t)tw / 3u);
        const uint32_t l1 = le[t1];
        if (path && n < path_cap) path[n] = t1;
        n++;
        if ((int32_t)l1 == tw - 3 * t1) {
            *terminal = e < tw ? e : tw;
            break;
        }
        t = t1;
        l = l1;
        if (n > max_steps) {
            *ok = false;
            break;
        }
    }
    return n;
}

__global__ void k_lepp_terminal(MeshView m, const uint8_t *le, int32_t max_steps, int32_t *terminal,
                                int32_t *length, int32_t *err) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m.T; t += gridDim.x * blockDim.x) {
        int32_t term = -1;
        bool ok = true;
        const int32_t n = lepp_chase(m, le, t, max_steps, nullptr, 0, &term, &ok);
        if (!ok) atomicOr(err, DEV_ERR_NONTERMINATING);
        terminal[t] = term;
        if (length) length[t] = n;
    }
}

// paths, pass 1: the length of each query's path into offsets[i]
__global__ void k_lepp_len(MeshView m, const uint8_t *le, const int32_t *tri, int32_t n, int32_t max_steps,
                           int32_t *offsets, int32_t *err) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t t = tri[i];
        if (t < 0 || t >= m.T) {
            atomicOr(err, DEV_ERR_INPUT);
            offsets[i] = 0;
            continue;
        }
        int32_t term;
        bool ok = true;
        const int32_t len = lepp_chase(m, le, t, max_steps, nullptr, 0, &term, &ok);
        if (!ok) atomicOr(err, DEV_ERR_NONTERMINATING);
        offsets[i] = len;
    }
}

// paths, pass 2: exclusive scan of the lengths per block of LP_THREADS,
// block totals into blk
constexpr int LP_THREADS = 1024;
__global__ void __launch_bounds__(LP_THREADS) k_lepp_scan_local(int32_t *offsets, int32_t n, unsigned long long *blk) {
    __shared__ int32_t s_w[LP_THREADS / 32];
    const int32_t i = blockIdx.x * LP_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t v = i < n ? offsets[i] : 0;
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int32_t x = s_w[lane];
        int32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        s_w[lane] = xi - x;
        if (lane == 31) blk[blockIdx.x] = (unsigned long long)xi;
    }
    __syncthreads();
    if (i < n) offsets[i] = s_w[wid] + inc - v;
}

// paths, pass 3 (after the block totals are scanned): add the block's
// prefix; offsets[n] = total; paths written where they fit the capacity
__global__ void k_lepp_write(MeshView m, const uint8_t *le, const int32_t *tri, int32_t n, int32_t max_steps,
                             int32_t *offsets, const unsigned long long *blk_pre, const unsigned long long *total,
                             int32_t *paths, int64_t capacity, int32_t *err) {
    const int32_t i = blockIdx.x * LP_THREADS + threadIdx.x;
    if (i == 0) {
        if ((long long)*total > (long long)INT32_MAX) atomicOr(err, DEV_ERR_CAPACITY);
        offsets[n] = (int32_t)min(*total, (unsigned long long)INT32_MAX);
        if ((long long)*total > capacity) atomicOr(err, DEV_ERR_CAPACITY);
    }
    if (i >= n) return;
    const int64_t off = (int64_t)offsets[i] + (int64_t)blk_pre[blockIdx.x];
    offsets[i] = (int32_t)min(off, (int64_t)INT32_MAX);
    const int32_t t = tri[i];
    if (t < 0 || t >= m.T || off >= capacity) return;
    int32_t term;
    bool ok = true;
    lepp_chase(m, le, t, max_steps, paths + off, capacity - off, &term, &ok);
}

void launch_lepp_terminal(const MeshView &m, const Work &w, int32_t *terminal, int32_t *length, int32_t *err,
                          cudaStream_t s) {
    k_lepp_terminal<<<w.persistent_blocks * 4, 256, 0, s>>>(m, w.le, m.T + 1, terminal, length, err);
}

void launch_lepp_paths(const MeshView &m, const Work &w, const int32_t *tri, int32_t n, int32_t *offsets,
                       int32_t *paths, int64_t capacity, unsigned long long *blk, unsigned long long *blk_pre,
                       unsigned long long *total, int32_t *err, cudaStream_t s) {
    const int32_t nb = (n + LP_THREADS - 1) / LP_THREADS;
    k_lepp_len<<<w.persistent_blocks * 4, 256, 0, s>>>(m, w.le, tri, n, m.T + 1, offsets, err);
    k_lepp_scan_local<<<nb, LP_THREADS, 0, s>>>(offsets, n, blk);
    launch_scan_u64(blk, blk_pre, nb, total, s);
    k_lepp_write<<<nb, LP_THREADS, 0, s>>>(m, w.le, tri, n, m.T + 1, offsets, blk_pre, total, paths, capacity, err);
}

}  // namespace polylla
