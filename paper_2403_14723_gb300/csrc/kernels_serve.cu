// Copy kernels of the serving loop (no counterpart in the paper).
//
// The copy engines run the copies of one direction in the order they were
// issued, whatever stream issued them: a 1 MiB copy issued right after
// 4 GiB of copies on another stream completes after them (20 ms measured on
// GB300), while the same 1 MiB moved by a kernel through host-mapped pinned
// memory completes in 0.06 ms beside them.  The serving loop therefore
// moves every small transfer (offsets, per-mesh metadata, the control
// block) and all the data of its low-latency lane with these kernels; large
// batches keep the copy engines, whose full-duplex rate is higher.
//
// Host memory is reached through the device addresses that
// cudaPointerGetAttributes / cudaHostGetDevicePointer give for pinned
// allocations.  Every range a kernel touches is one the request declared
// (its vertex, triangle and half-edge counts) or one the run's metadata
// gives after it is checked against those counts and the outputs' sizes.
#include "polylla_internal.cuh"
#include "polylla_serve.cuh"

namespace polylla {

namespace {

constexpr int SV_THREADS = 256;

// request i's ranges, read once per block from pinned host memory
struct Ranges {
    int32_t v0, nv, t0, nt, h0, nh;
};

__device__ __forceinline__ void load_ranges(const int32_t *off4, int32_t n, int32_t i, Ranges *r) {
    const int32_t *vo = off4, *to = off4 + (n + 1), *ho = off4 + 2 * (n + 1);
    r->v0 = vo[i];
    r->nv = vo[i + 1] - r->v0;
    r->t0 = to[i];
    r->nt = to[i + 1] - r->t0;
    r->h0 = ho[i];
    r->nh = ho[i + 1] - r->h0;
}

__global__ void __launch_bounds__(SV_THREADS) k_serve_offsets(const int32_t *off4, int32_t n, int32_t *v_off,
                                                                int32_t *t_off, int32_t *h_off, int32_t *b_off) {
    const int32_t m = n + 1;
    int32_t *dst[4] = {v_off, t_off, h_off, b_off};
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < 4 * m; q += gridDim.x * blockDim.x)
        dst[q / m][q % m] = off4[q];
}

__global__ void __launch_bounds__(SV_THREADS) k_serve_gather(const ServeTab *tab, const int32_t *off4, int32_t n,
                                                               double *coords, int32_t *origin, int32_t *twin) {
    __shared__ ServeTab st;
    __shared__ Ranges sr;
    const int32_t i = blockIdx.y;
    if (threadIdx.x == 0) {
        st = tab[i];
        load_ranges(off4, n, i, &sr);
    }
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    double *cd = coords + 2 * (int64_t)sr.v0;
    for (int64_t k = g; k < 2 * (int64_t)sr.nv; k += gs) cd[k] = st.coords[k];
    int32_t *od = origin + sr.h0, *td = twin + sr.h0;
    for (int64_t k = g; k < sr.nh; k += gs) {
        od[k] = st.origin[k];
        td[k] = st.twin[k];
    }
}

__device__ __forceinline__ void copy_ctrl(const DevCtrl *ctrl, DevCtrl *ctrl_host) {
    static_assert(sizeof(DevCtrl) % 4 == 0 && sizeof(DevCtrl) / 4 <= SV_THREADS, "control block words");
    if (threadIdx.x < sizeof(DevCtrl) / 4)
        reinterpret_cast<int32_t *>(ctrl_host)[threadIdx.x] = reinterpret_cast<const int32_t *>(ctrl)[threadIdx.x];
}

__global__ void __launch_bounds__(SV_THREADS) k_serve_scatter(const ServeTab *tab, const int32_t *off4, int32_t n,
                                                                ServeOutputs o, const int32_t *next,
                                                                const int32_t *prev, int32_t T_tot,
                                                                int32_t *meta_host, DevCtrl *ctrl_host) {
    __shared__ ServeTab st;
    __shared__ Ranges sr;
    __shared__ int32_t sm[4];
    const int32_t i = blockIdx.y;
    if (threadIdx.x == 0) {
        st = tab[i];
        load_ranges(off4, n, i, &sr);
        const int32_t P = o.meta[4 * i], NF = o.meta[4 * i + 1], p0 = o.meta[4 * i + 2], c0 = o.meta[4 * i + 3];
        // a run that failed leaves no usable metadata: copy nothing then
        const bool ok = P >= 0 && P <= sr.nt && NF >= 0 && (int64_t)NF <= 3 * (int64_t)sr.nt && p0 >= 0 &&
                        (int64_t)p0 + P <= T_tot && c0 >= 0 && (int64_t)c0 + NF <= 3 * (int64_t)T_tot;
        sm[0] = ok ? P : -1;
        sm[1] = NF;
        sm[2] = p0;
        sm[3] = c0;
        if (blockIdx.x == 0) {
            meta_host[4 * i] = sm[0];
            meta_host[4 * i + 1] = NF;
            meta_host[4 * i + 2] = p0;
            meta_host[4 * i + 3] = c0;
        }
    }
    __syncthreads();
    if (i == 0 && blockIdx.x == 0) copy_ctrl(o.ctrl, ctrl_host);
    if (sm[0] >= 0) {
        const int32_t P = sm[0], NF = sm[1], p0 = sm[2], c0 = sm[3];
        const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
        for (int64_t k = g; k < P; k += gs) st.seeds[k] = o.seeds[p0 + k];
        // mesh i's rebased offsets start at its first polygon + i
        for (int64_t k = g; k <= P; k += gs) st.offsets[k] = o.local_offsets[(int64_t)p0 + i + k];
        for (int64_t k = g; k < NF; k += gs) {
            st.he_list[k] = o.he_list[c0 + k];
            st.v_list[k] = o.v_list[c0 + k];
        }
        const int32_t *nx = next + sr.h0, *pv = prev + sr.h0;
        for (int64_t k = g; k < 3 * (int64_t)sr.nt; k += gs) {
            st.next[k] = nx[k];
            st.prev[k] = pv[k];
        }
    }
    __threadfence_system();
}

__global__ void __launch_bounds__(SV_THREADS) k_serve_meta_out(ServeOutputs o, int32_t n, int32_t *meta_host,
                                                                 DevCtrl *ctrl_host) {
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < 4 * n; q += gridDim.x * blockDim.x)
        meta_host[q] = o.meta[q];
    if (blockIdx.x == 0) copy_ctrl(o.ctrl, ctrl_host);
    __threadfence_system();
}

int32_t grid_for(int64_t words) {
    const int64_t b = (words + SV_THREADS * 8 - 1) / (SV_THREADS * 8);
    return (int32_t)(b < 1 ? 1 : b > 1024 ? 1024 : b);
}

}  // namespace

void launch_serve_offsets(const int32_t *off4, int32_t n, int32_t *v_off, int32_t *t_off, int32_t *h_off,
                          int32_t *b_off, cudaStream_t s) {
    k_serve_offsets<<<grid_for(4 * (int64_t)(n + 1)), SV_THREADS, 0, s>>>(off4, n, v_off, t_off, h_off, b_off);
}

void launch_serve_gather(const ServeTab *tab, const int32_t *off4, int32_t n, int32_t blocks_x, double *coords,
                         int32_t *origin, int32_t *twin, cudaStream_t s) {
    k_serve_gather<<<dim3(blocks_x, n), SV_THREADS, 0, s>>>(tab, off4, n, coords, origin, twin);
}

void launch_serve_scatter(const ServeTab *tab, const int32_t *off4, int32_t n, int32_t blocks_x,
                          const ServeOutputs &o, const int32_t *next, const int32_t *prev, int32_t T_tot,
                          int32_t *meta_host, DevCtrl *ctrl_host, cudaStream_t s) {
    k_serve_scatter<<<dim3(blocks_x, n), SV_THREADS, 0, s>>>(tab, off4, n, o, next, prev, T_tot, meta_host,
                                                             ctrl_host);
}

void launch_serve_meta_out(const ServeOutputs &o, int32_t n, int32_t *meta_host, DevCtrl *ctrl_host, cudaStream_t s) {
    k_serve_meta_out<<<grid_for(4 * (int64_t)n), SV_THREADS, 0, s>>>(o, n, meta_host, ctrl_host);
}

}  // namespace polylla
