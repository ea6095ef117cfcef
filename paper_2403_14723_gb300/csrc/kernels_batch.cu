// Batches of independent meshes (no counterpart in the paper, whose method
// takes one mesh): the stage kernels run once over the batch's union, a
// single mesh whose connected components are the batch's meshes.  A
// generate reads the meshes' own arrays: the longest-edge kernel checks
// every interior origin and twin against its mesh and writes the union
// twins, the listing kernel reads local origins; the relink and repair
// kernels write the relinked next/prev in local indices too, and the listing
// kernel writes local seeds and each mesh's first polygon.  Packing all four
// arrays into the union (this file) is done once, at create, for the layout
// check.
//
// The union keeps every order the method depends on within a mesh: interior
// half-edges of mesh i are shifted by 3 t_off[i], its border half-edges go
// after all interior ones (still after its own interior ones, still in
// order), so longest-edge ties (smallest edge id), rotation, canonical seeds
// (smallest half-edge) and the polygon order (by seed) are those of the
// mesh alone, and mesh i's polygons come before mesh i+1's.
#include "polylla_internal.cuh"

namespace polylla {

constexpr int BP_THREADS = 256;
constexpr int BP_ITEMS = 8;
constexpr int BP_SPAN = BP_THREADS * BP_ITEMS;
constexpr int BP_TABLE = 48;  // meshes a block keeps in shared memory

// Per-mesh constants of the meshes a block's range touches, in shared
// memory: for interior blocks the range [base, end) of union half-edges
// starts in mesh m0.  Entry j describes mesh m0 + j: the union index its
// segment starts at (interior: 3 t_off, border: 3T_tot + b_off), the
// offset from union to concatenated local position, the vertex offset, and
// the border shift (union index of local border half-edge y is bo + y).
struct PackTable {
    int32_t m0, n;
    int32_t start[BP_TABLE + 1];
    int32_t to_local[BP_TABLE];   // g = x + to_local
    int32_t t3[BP_TABLE];         // 3 t_off: interior shift
    int32_t ti3[BP_TABLE];        // 3 T_i
    int32_t bo[BP_TABLE];
    int32_t v0[BP_TABLE];
    int32_t hi[BP_TABLE];         // H_i
    int32_t vi[BP_TABLE];         // V_i
};

// fill the table (block-wide); returns false when the range spans more
// meshes than the table holds (then every element looks its mesh up)
__device__ bool pack_table(const BatchView &b, bool border, int32_t base, int32_t end, PackTable &tb) {
    const int32_t HI = 3 * b.T_tot;
    if (threadIdx.x == 0) {
        int32_t m0, m1;
        if (!border) {
            m0 = seg_of(b.t_off, b.n, base / 3);
            m1 = seg_of(b.t_off, b.n, (end - 1) / 3);
        } else {
            m0 = seg_of(b.b_off, b.n, base - HI);
            m1 = seg_of(b.b_off, b.n, end - 1 - HI);
        }
        tb.m0 = m0;
        tb.n = m1 - m0 + 1;
    }
    __syncthreads();
    const int32_t n = tb.n;
    if (n > BP_TABLE) return false;
    for (int j = threadIdx.x; j < n; j += BP_THREADS) {
        const int32_t m = tb.m0 + j;
        const int32_t t0 = b.t_off[m], Ti = b.t_off[m + 1] - t0;
        const int32_t h0 = b.h_off[m], bb = b.b_off[m];
        tb.t3[j] = 3 * t0;
        tb.ti3[j] = 3 * Ti;
        tb.bo[j] = HI + bb - 3 * Ti;
        tb.v0[j] = b.v_off[m];
        tb.hi[j] = b.h_off[m + 1] - h0;
        tb.vi[j] = b.v_off[m + 1] - b.v_off[m];
        if (!border) {
            tb.start[j] = 3 * t0;
            tb.to_local[j] = h0 - 3 * t0;              // g = h0 + (x - 3 t0)
        } else {
            tb.start[j] = HI + bb;
            tb.to_local[j] = h0 + 3 * Ti - HI - bb;    // g = h0 + 3 Ti + (x - HI - bb)
        }
    }
    if (threadIdx.x == 0) tb.start[n] = 0x7fffffff;
    __syncthreads();
    return true;
}

// ===========================================================================
// k_batch_pack (create, for the layout check): union origin/twin (and
// next/prev when given) from the local arrays.  Logical blocks [0, nbI)
// cover interior union half-edges, the rest the border ones (blk0 offsets
// the launch); a block tabulates the meshes its range touches and each
// element finds its mesh there.  Every origin and twin is range-checked:
// one outside its mesh is replaced by an index inside it (vertex 0, the
// mesh's first border half-edge), so the layout check that follows cannot
// leave the mesh, and input_err / bad are set; with bad != nullptr next
// and prev are checked too.
// ===========================================================================
__global__ void __launch_bounds__(BP_THREADS) k_batch_pack(BatchView b, int32_t *u_origin, int32_t *u_twin,
                                                           int32_t *u_next, int32_t *u_prev, int32_t *bad,
                                                           int32_t *input_err, int32_t blk0) {
    __shared__ PackTable tb;
    const int32_t HI = 3 * b.T_tot;
    const int32_t nbI = (HI + BP_SPAN - 1) / BP_SPAN;
    const int32_t blk = (int32_t)blockIdx.x + blk0;
    const bool border = blk >= nbI;
    const int32_t base = border ? HI + (blk - nbI) * BP_SPAN : blk * BP_SPAN;
    const int32_t end = min(base + BP_SPAN, border ? b.H_tot : HI);
    const bool tabled = pack_table(b, border, base, end, tb);
    // all loads of the thread's items first, then all stores: the stores
    // could alias later loads as far as the compiler knows, which would
    // otherwise serialise one memory round trip per item
    int32_t o[BP_ITEMS], tw[BP_ITEMS], nx[BP_ITEMS], pv[BP_ITEMS], jj[BP_ITEMS];
    int32_t j = 0;
#pragma unroll
    for (int k = 0; k < BP_ITEMS; k++) {
        const int32_t x = base + k * BP_THREADS + (int32_t)threadIdx.x;
        jj[k] = -1;
        if (x >= end) continue;
        int32_t g;
        if (tabled) {
            while (tb.start[j + 1] <= x) j++;
            g = x + tb.to_local[j];
            jj[k] = j;
        } else {
            const int32_t m = border ? seg_of(b.b_off, b.n, x - HI) : seg_of(b.t_off, b.n, x / 3);
            const int32_t t0 = b.t_off[m], Ti = b.t_off[m + 1] - t0;
            g = border ? b.h_off[m] + 3 * Ti + (x - HI - b.b_off[m]) : b.h_off[m] + (x - 3 * t0);
            jj[k] = m;
        }
        o[k] = b.origin[g];
        tw[k] = b.twin[g];
        if (u_next) {
            nx[k] = b.next[g];
            pv[k] = b.prev[g];
        }
    }
    int32_t fail = 0;
#pragma unroll
    for (int k = 0; k < BP_ITEMS; k++) {
        if (jj[k] < 0) continue;
        const int32_t x = base + k * BP_THREADS + (int32_t)threadIdx.x;
        int32_t t3, ti3, bo, v0, hi, vi;
        if (tabled) {
            const int32_t q = jj[k];
            t3 = tb.t3[q];
            ti3 = tb.ti3[q];
            bo = tb.bo[q];
            v0 = tb.v0[q];
            hi = tb.hi[q];
            vi = tb.vi[q];
        } else {
            const int32_t m = jj[k];
            const int32_t t0 = b.t_off[m], Ti = b.t_off[m + 1] - t0;
            t3 = 3 * t0;
            ti3 = 3 * Ti;
            bo = HI + b.b_off[m] - 3 * Ti;
            v0 = b.v_off[m];
            hi = b.h_off[m + 1] - b.h_off[m];
            vi = b.v_off[m + 1] - v0;
        }
        const bool out = o[k] < 0 || o[k] >= vi || tw[k] < 0 || tw[k] >= hi;
        fail |= out;
        if (out) {
            // keep every later access inside the mesh: vertex 0, and the
            // mesh's first border half-edge (a twin that stops rotations)
            if (o[k] < 0 || o[k] >= vi) o[k] = 0;
            if (tw[k] < 0 || tw[k] >= hi) tw[k] = ti3;
        }
        u_origin[x] = o[k] + v0;
        u_twin[x] = tw[k] < ti3 ? t3 + tw[k] : bo + tw[k];
        if (u_next) {
            if (bad) fail |= nx[k] < 0 || nx[k] >= hi || pv[k] < 0 || pv[k] >= hi;
            u_next[x] = nx[k] < ti3 ? t3 + nx[k] : bo + nx[k];
            u_prev[x] = pv[k] < ti3 ? t3 + pv[k] : bo + pv[k];
        }
    }
    if (fail) {
        if (bad) atomicOr(bad, 1);
        if (input_err) atomicOr(input_err, 1);
    }
}

// ===========================================================================
// k_batch_meta (serving): per mesh i, meta[4i..4i+3] = {P_i, N_F,i, first
// polygon, first CSR entry}, and each mesh's offsets rebased to start at 0
// in local_offsets[poly_off[i] + i .. poly_off[i+1] + i] (P_i + 1 entries),
// so that every mesh's CSR is four contiguous slices.  Grid-stride over all
// P + n rebased entries (entry q belongs to the last mesh i with
// poly_off[i] + i <= q), so one large mesh is spread over the whole grid.
// ===========================================================================
__global__ void k_batch_meta(BatchView b, const int32_t *offsets, const int32_t *poly_off, int32_t *local_offsets,
                             int32_t *meta) {
    const int32_t n = b.n;
    const int32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (int32_t i = gt; i < n; i += gs) {
        const int32_t p0 = poly_off[i], p1 = poly_off[i + 1];
        const int32_t c0 = offsets[p0];
        meta[4 * i] = p1 - p0;
        meta[4 * i + 1] = offsets[p1] - c0;
        meta[4 * i + 2] = p0;
        meta[4 * i + 3] = c0;
    }
    const int32_t total = poly_off[n] + n;
    for (int32_t q = gt; q < total; q += gs) {
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (__ldg(poly_off + mid) + mid <= q) lo = mid;
            else hi = mid - 1;
        }
        const int32_t p0 = __ldg(poly_off + lo);
        local_offsets[q] = offsets[p0 + (q - p0 - lo)] - offsets[p0];
    }
}

// ===========================================================================
// k_batch_seg (serving, per batch): the mesh table, seg[g] = the mesh of
// union triangle min(g SEG_SPAN, T - 1), by binary search over the triangle
// prefix sums.
// ===========================================================================
__global__ void k_batch_seg(const int32_t *t_off, int32_t n, int32_t T, int32_t *seg) {
    const int32_t ns = (int32_t)seg_count(T);
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ns; g += gridDim.x * blockDim.x)
        seg[g] = seg_of(t_off, n, min(g * SEG_SPAN, T - 1));
}

void launch_batch_seg(const int32_t *t_off, int32_t n, int32_t T, int32_t *seg, cudaStream_t s) {
    const int32_t ns = (int32_t)seg_count(T);
    const int32_t blocks = (ns + 255) / 256;
    k_batch_seg<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(t_off, n, T, seg);
}

void launch_batch_meta(const BatchView &b, const Work &w, const int32_t *poly_off, int32_t *local_offsets,
                       int32_t *meta, cudaStream_t s) {
    k_batch_meta<<<w.persistent_blocks, 256, 0, s>>>(b, w.offsets, poly_off, local_offsets, meta);
}

void launch_batch_pack(const BatchView &b, int32_t *u_origin, int32_t *u_twin, int32_t *u_next, int32_t *u_prev,
                       int32_t *bad, int32_t *input_err, cudaStream_t s) {
    const int32_t HI = 3 * b.T_tot, HB = b.H_tot - HI;
    const int32_t blocks = (HI + BP_SPAN - 1) / BP_SPAN + (HB + BP_SPAN - 1) / BP_SPAN;
    k_batch_pack<<<blocks, BP_THREADS, 0, s>>>(b, u_origin, u_twin, u_next, u_prev, bad, input_err, 0);
}

}  // namespace polylla
