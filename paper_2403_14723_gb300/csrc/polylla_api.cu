// Host side of the C ABI declared in include/polylla.h: context lifetime,
// argument checks, the kernel sequence of polylla_generate, and readback.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/polylla.h"
#include "polylla_internal.cuh"
#include "polylla_serve.cuh"

using namespace polylla;

namespace {

constexpr int kCore = 7;     // the method's kernels, on one mesh or a batch's union
constexpr int kStages = 8;   // + the serving loop's per-mesh metadata
constexpr int kMeta = 7;
const char *kStageNames[kStages] = {
    "longest_edge", "label_relink", "chords", "chord_links", "poly_count", "tile_scan", "poly_list",
    "batch_meta",
};
constexpr int kKernels = 7;        // one kernel per stage

}  // namespace

struct polylla_ctx {
    int device = 0;
    MeshView mesh{};
    bool owns_mesh = false;
    Work w{};
    int32_t *d_bad = nullptr;       // create-time layout check result
    DevCtrl *h_ctrl = nullptr;      // pinned readback of the control block
    cudaError_t last_cuda = cudaSuccess;
    bool timing = false;
    cudaEvent_t ev_begin[kStages]{}, ev_end[kStages]{};
    bool stage_ran[kStages]{};
    bool timed_last = false;
    int launches = 0;
    cudaStream_t last_stream = nullptr;
    // batch: c->mesh is the union, bv the caller's local arrays
    bool is_batch = false;
    BatchView bv{};
    int32_t *poly_off = nullptr;    // [n+1] first polygon of each mesh
    int32_t *u_origin = nullptr, *u_twin = nullptr;  // union arrays, owned
    // Lepp paths: per-1024-query totals, their scan, the grand total
    unsigned long long *lepp_blk = nullptr, *lepp_blk_pre = nullptr, *lepp_total = nullptr;
    // serving: per-mesh metadata and rebased offsets after each run
    bool serve = false;
    int32_t *meta = nullptr;           // [4 n_cap]
    int32_t *local_offsets = nullptr;  // [T_cap + n_cap + 1]
    size_t bytes = 0;                  // device bytes allocated
    // host-buffer path: a side stream for copies that overlap the kernels,
    // and the events that order them against the stages
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_twin = nullptr, ev_links = nullptr;
    cudaEvent_t wait_before_relink = nullptr;  // enqueue: stage 1 waits for it
    cudaEvent_t record_after_links = nullptr;  // enqueue: recorded after stage 3
    // convexification: its chord list (allocated by the first call) and count
    int32_t *cv_list = nullptr;
    int32_t *cv_count = nullptr;   // [2]: chords, reflex corners
    int32_t *cv_reflex = nullptr;
    int32_t cv_cap = 0;
    // captured generate (polylla_capture_graph)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_launches = 0;
    // device allocations (for destroy)
    void *allocs[64]{};
    int n_allocs = 0;
};

static int cuda_fail(polylla_ctx *c, cudaError_t e) {
    if (c) c->last_cuda = e;
    return e == cudaErrorMemoryAllocation ? POLYLLA_ERR_OUT_OF_MEMORY : POLYLLA_ERR_CUDA;
}

#define CK(call)                                      \
    do {                                              \
        cudaError_t _e = (call);                      \
        if (_e != cudaSuccess) return cuda_fail(c, _e); \
    } while (0)

static int dev_alloc(polylla_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->n_allocs >= (int)(sizeof(c->allocs) / sizeof(c->allocs[0]))) return POLYLLA_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->allocs[c->n_allocs++] = *p;
    c->bytes += bytes;
    return POLYLLA_OK;
}

static void drop_graph(polylla_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_launches = 0;
}

static void free_all(polylla_ctx *c) {
    drop_graph(c);
    if (c->aux) cudaStreamSynchronize(c->aux);
    if (c->ev_twin) cudaEventDestroy(c->ev_twin);
    if (c->ev_links) cudaEventDestroy(c->ev_links);
    if (c->aux) cudaStreamDestroy(c->aux);
    c->aux = nullptr;
    c->ev_twin = c->ev_links = nullptr;
    for (int i = 0; i < c->n_allocs; i++) cudaFree(c->allocs[i]);
    c->n_allocs = 0;
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    c->h_ctrl = nullptr;
    for (int i = 0; i < kStages; i++) {
        if (c->ev_begin[i]) cudaEventDestroy(c->ev_begin[i]);
        if (c->ev_end[i]) cudaEventDestroy(c->ev_end[i]);
        c->ev_begin[i] = c->ev_end[i] = nullptr;
    }
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_sizes(int32_t V, int32_t T, int32_t H) {
    if (V < 3 || T < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    if ((int64_t)T * 3 >= (int64_t)INT32_MAX) return POLYLLA_ERR_INVALID_ARGUMENT;
    if ((int64_t)H < 3 * (int64_t)T + 3) return POLYLLA_ERR_INVALID_ARGUMENT;
    return POLYLLA_OK;
}

// ---- launch tuning ----------------------------------------------------------
// Launch settings that do not change results: the relink block size and the
// grids of the persistent longest-edge, walk and emit kernels.  A process-
// wide table keeps the settings polylla_autotune found per device and size
// bucket (floor(log2 T)); contexts created later for a mesh or batch in a
// tuned bucket start from them.
namespace {
constexpr int kTuneDevices = 16;
constexpr int kTuneBuckets = 32;
struct TuneEntry {
    bool set;
    polylla_tuning t;
};
TuneEntry g_tune[kTuneDevices][kTuneBuckets];
std::mutex g_tune_lock;

int size_bucket(int32_t T) {
    int b = 0;
    while (T > 1 && b < kTuneBuckets - 1) {
        T >>= 1;
        b++;
    }
    return b;
}
}  // namespace

static int sm_count(polylla_ctx *c) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1) sms = 1;
    return sms;
}

static bool tuning_valid(polylla_ctx *c, const polylla_tuning &t) {
    const int cap = 64 * sm_count(c);
    return relink_config_valid(t.relink_tile, t.relink_items) &&
           t.longest_edge_blocks >= 1 && t.longest_edge_blocks <= cap &&
           (t.longest_edge_items == 2 || t.longest_edge_items == 4) &&
           polygons_config_valid(t.output_tile, t.output_items);
}

static void apply_tuning(polylla_ctx *c, const polylla_tuning &t) {
    c->w.rl_tile = t.relink_tile;
    c->w.rl_items = t.relink_items;
    c->w.le_blocks = t.longest_edge_blocks;
    c->w.le_items = t.longest_edge_items;
    c->w.out_tile = t.output_tile;
    c->w.out_items = t.output_items;
}

static polylla_tuning current_tuning(const polylla_ctx *c) {
    polylla_tuning t;
    t.relink_tile = c->w.rl_tile;
    t.relink_items = c->w.rl_items;
    t.longest_edge_blocks = c->w.le_blocks;
    t.longest_edge_items = c->w.le_items;
    t.output_tile = c->w.out_tile;
    t.output_items = c->w.out_items;
    return t;
}

static void apply_cached_tuning(polylla_ctx *c) {
    if (c->device < 0 || c->device >= kTuneDevices) return;
    std::lock_guard<std::mutex> g(g_tune_lock);
    const TuneEntry &e = g_tune[c->device][size_bucket(c->mesh.T)];
    if (e.set && tuning_valid(c, e.t)) apply_tuning(c, e.t);
}

// allocate scratch and outputs for the sizes in c->mesh
static int alloc_work(polylla_ctx *c, const polylla_options *opt) {
    const int32_t V = c->mesh.V, T = c->mesh.T;
    const int64_t Tpad = ((int64_t)T + 15) / 16 * 16;
    const int64_t HI = 3 * (int64_t)T;
    int rc;
    void *p;
    if ((rc = dev_alloc(c, &p, Tpad))) return rc;
    c->w.le = (uint8_t *)p;
    if ((rc = dev_alloc(c, &p, Tpad))) return rc;
    c->w.flags = (uint8_t *)p;
    c->w.tip_cap = V;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)V))) return rc;
    c->w.tips = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)V))) return rc;
    c->w.chords = (int32_t *)p;
    c->w.n_tile_max = (int32_t)(((int64_t)T + OUT_TILE_MIN - 1) / OUT_TILE_MIN);
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_tile_max))) return rc;
    c->w.tile_state = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_tile_max))) return rc;
    c->w.tile_pre = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)(c->w.n_tile_max / SCAN_THREADS + 1)))) return rc;
    c->w.group_tot = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)(c->w.n_tile_max / SCAN_THREADS + 1)))) return rc;
    c->w.group_pre = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)out_rec_count(T)))) return rc;
    c->w.poly_rec = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)out_warp_count(T)))) return rc;
    c->w.poly_wtot = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)T))) return rc;
    c->w.seeds = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)(T + 1)))) return rc;
    c->w.offsets = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)HI))) return rc;
    c->w.he_list = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)HI))) return rc;
    c->w.v_list = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(DevCtrl)))) return rc;
    c->w.ctrl = (DevCtrl *)p;
    const size_t n_lepp_blk = ((size_t)T + 1023) / 1024 + 1;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * n_lepp_blk))) return rc;
    c->lepp_blk = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * n_lepp_blk))) return rc;
    c->lepp_blk_pre = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long)))) return rc;
    c->lepp_total = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t)))) return rc;
    c->d_bad = (int32_t *)p;
    cudaError_t e = cudaMallocHost((void **)&c->h_ctrl, sizeof(DevCtrl));
    if (e != cudaSuccess) return cuda_fail(c, e);
    memset(c->h_ctrl, 0, sizeof(DevCtrl));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->w.persistent_blocks = 4 * (sms > 0 ? sms : 1);
    c->w.le_items = LE_ITEMS_DEFAULT;
    c->w.le_blocks = longest_edge_blocks_per_sm(LE_ITEMS_DEFAULT) * (sms > 0 ? sms : 1);
    c->w.le_batch_blocks = longest_edge_batch_blocks_per_sm() * (sms > 0 ? sms : 1);
    c->w.out_tile = OUT_TILE_DEFAULT;
    c->w.out_items = OUT_ITEMS_DEFAULT;
    c->w.rl_tile = RL_TILE_DEFAULT;
    c->w.rl_items = RL_ITEMS_DEFAULT;
    if (polygons_configure() != 0 || relink_configure() != 0) return cuda_fail(c, cudaGetLastError());
    c->w.max_rot = (opt && opt->max_rotation > 0) ? opt->max_rotation : 4096;
    apply_cached_tuning(c);
    for (int i = 0; i < kStages; i++) {
        e = cudaEventCreate(&c->ev_begin[i]);
        if (e == cudaSuccess) e = cudaEventCreate(&c->ev_end[i]);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return POLYLLA_OK;
}

// Union arrays, offset arrays and polygon ranges of a batch context for n
// meshes of V, T, H in total; c->mesh becomes the union view (sizes V, T, H)
// over the caller's coords.  The offset arrays are left to the caller.
static int batch_alloc(polylla_ctx *c, int32_t n, int32_t V, int32_t T, int32_t H, const double *coords,
                       const int32_t *origin, const int32_t *twin, int32_t *next, int32_t *prev) {
    c->is_batch = true;
    c->mesh.V = V;
    c->mesh.T = T;
    c->mesh.H = H;
    c->mesh.xy = reinterpret_cast<const double2 *>(coords);
    BatchView &bv = c->bv;
    bv.n = n;
    bv.T_tot = T;
    bv.H_tot = H;
    bv.origin = origin;
    bv.twin = twin;
    bv.next = next;
    bv.prev = prev;
    int rc = POLYLLA_OK;
    void *p = nullptr;
    int32_t *d_off[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4 && !rc; k++)
        if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)(n + 1))) == 0) d_off[k] = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)(n + 1))) == 0) c->poly_off = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * (size_t)H)) == 0) c->u_origin = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * (size_t)H)) == 0) c->u_twin = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * (size_t)H)) == 0) c->mesh.next = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * (size_t)H)) == 0) c->mesh.prev = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)seg_count(T))) == 0) c->w.loc_seg = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, sizeof(int32_t))) == 0) c->w.input_err = (int32_t *)p;
    if (!rc && cudaMemset(c->w.input_err, 0, sizeof(int32_t)) != cudaSuccess) rc = POLYLLA_ERR_CUDA;
    // the union origin is filled by the layout check at create only; every
    // generate writes the interior union twins from the local arrays
    c->mesh.origin = c->u_origin;
    c->mesh.twin = c->u_twin;
    c->w.loc_origin = origin;
    c->w.loc_aligned = ((uintptr_t)origin & 15u) == 0 && ((uintptr_t)twin & 15u) == 0;
    c->w.loc_twin = twin;
    c->w.u_twin = c->u_twin;
    bv.v_off = d_off[0];
    bv.t_off = d_off[1];
    bv.h_off = d_off[2];
    bv.b_off = d_off[3];
    return rc;
}

static int run_validate(polylla_ctx *c, cudaStream_t s) {
    CK(cudaMemsetAsync(c->d_bad, 0, sizeof(int32_t), s));
    launch_validate(c->mesh, c->d_bad, s);
    CK(cudaGetLastError());
    int32_t bad = 0;
    CK(cudaMemcpyAsync(&bad, c->d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return bad ? POLYLLA_ERR_INVALID_MESH : POLYLLA_OK;
}

extern "C" {

const char *polylla_status_string(int status) {
    switch (status) {
        case POLYLLA_OK: return "ok";
        case POLYLLA_ERR_INVALID_ARGUMENT: return "invalid argument";
        case POLYLLA_ERR_INVALID_MESH: return "invalid mesh layout";
        case POLYLLA_ERR_OUT_OF_MEMORY: return "out of device memory";
        case POLYLLA_ERR_CUDA: return "CUDA error";
        case POLYLLA_ERR_NONTERMINATING: return "rotation or cycle walk did not terminate";
        case POLYLLA_ERR_CAPACITY: return "internal list capacity exceeded";
        case POLYLLA_ERR_TIMEOUT: return "device wait timed out";
        case POLYLLA_ERR_TOO_LARGE: return "mesh larger than the available capacity (no-allocation scratch or server slot)";
        default: return "unknown status";
    }
}

int polylla_create(polylla_ctx **out, const polylla_mesh *mesh, const polylla_options *opt,
                   polylla_stream stream) {
    if (!out) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!mesh) return POLYLLA_ERR_INVALID_ARGUMENT;
    int rc = check_sizes(mesh->n_vertices, mesh->n_triangles, mesh->n_halfedges);
    if (rc) return rc;
    if (!mesh->coords || !mesh->origin || !mesh->twin || !mesh->next || !mesh->prev)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!aligned(mesh->coords, 16) || !aligned(mesh->origin, 16) || !aligned(mesh->twin, 16) ||
        !aligned(mesh->next, 16) || !aligned(mesh->prev, 16))
        return POLYLLA_ERR_INVALID_ARGUMENT;
    polylla_ctx *c = new (std::nothrow) polylla_ctx();
    if (!c) return POLYLLA_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { delete c; return POLYLLA_ERR_CUDA; }
    c->mesh.V = mesh->n_vertices;
    c->mesh.T = mesh->n_triangles;
    c->mesh.H = mesh->n_halfedges;
    c->mesh.xy = reinterpret_cast<const double2 *>(mesh->coords);
    c->mesh.origin = mesh->origin;
    c->mesh.twin = mesh->twin;
    c->mesh.next = mesh->next;
    c->mesh.prev = mesh->prev;
    rc = alloc_work(c, opt);
    if (!rc && (!opt || opt->validate)) rc = run_validate(c, (cudaStream_t)stream);
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return POLYLLA_OK;
}

int polylla_create_host(polylla_ctx **out, int32_t n_vertices, int32_t n_triangles, int32_t n_halfedges,
                        const polylla_options *opt) {
    if (!out) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    int rc = check_sizes(n_vertices, n_triangles, n_halfedges);
    if (rc) return rc;
    polylla_ctx *c = new (std::nothrow) polylla_ctx();
    if (!c) return POLYLLA_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return POLYLLA_ERR_CUDA; }
    c->owns_mesh = true;
    c->mesh.V = n_vertices;
    c->mesh.T = n_triangles;
    c->mesh.H = n_halfedges;
    void *p;
    const size_t H = (size_t)n_halfedges;
    if ((rc = dev_alloc(c, &p, 16 * (size_t)n_vertices)) == 0) c->mesh.xy = (const double2 *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * H)) == 0) c->mesh.origin = (const int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * H)) == 0) c->mesh.twin = (const int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * H)) == 0) c->mesh.next = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, 4 * H)) == 0) c->mesh.prev = (int32_t *)p;
    if (!rc) rc = alloc_work(c, opt);
    if (!rc) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_twin, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_links, cudaEventDisableTiming);
        if (e != cudaSuccess) rc = cuda_fail(c, e);
    }
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return POLYLLA_OK;
}

}  // extern "C"

// Enqueue one whole run on s: the method's stages (on a batch, on its union:
// the longest-edge kernel reads the meshes' own arrays and writes the union
// twins, the later kernels also write each mesh's own next/prev, seeds and
// polygon ranges), then, when serving, the per-mesh metadata; with timing,
// an event pair around every stage.
static int enqueue(polylla_ctx *c, cudaStream_t s, bool timing) {
    for (int i = 0; i < kStages; i++) c->stage_ran[i] = false;
    auto begin = [&](int i) -> cudaError_t {
        c->stage_ran[i] = true;
        return timing ? cudaEventRecord(c->ev_begin[i], s) : cudaSuccess;
    };
    auto end = [&](int i) -> cudaError_t { return timing ? cudaEventRecord(c->ev_end[i], s) : cudaSuccess; };
    void (*stages[kCore])(const MeshView &, const Work &, cudaStream_t) = {
        launch_longest_edge, launch_label_relink, launch_chords, launch_chord_links, launch_poly_count,
        launch_tile_scan, launch_poly_list,
    };
    for (int i = 0; i < kCore; i++) {
        if (i == 1 && c->wait_before_relink) CK(cudaStreamWaitEvent(s, c->wait_before_relink, 0));
        CK(begin(i));
        stages[i](c->mesh, c->w, s);
        CK(end(i));
        if (i == 3 && c->record_after_links) CK(cudaEventRecord(c->record_after_links, s));
    }
    if (c->is_batch) {
        CK(begin(kMeta));
        // the relink and repair kernels wrote the meshes' own next/prev and
        // the listing kernel their seeds and polygon ranges
        if (c->serve) launch_batch_meta(c->bv, c->w, c->poly_off, c->local_offsets, c->meta, s);
        CK(end(kMeta));
    }
    c->launches = kKernels + (c->serve ? 1 : 0);
    CK(cudaGetLastError());
    return POLYLLA_OK;
}

extern "C" {

int polylla_generate(polylla_ctx *c, polylla_stream stream) {
    if (!c) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    if (c->graph_exec) {
        c->timed_last = false;
        CK(cudaGraphLaunch(c->graph_exec, s));
        c->launches = c->graph_launches;
        return POLYLLA_OK;
    }
    c->timed_last = c->timing;
    return enqueue(c, s, c->timing);
}

int polylla_capture_graph(polylla_ctx *c, polylla_stream stream) {
    if (!c || !stream) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    drop_graph(c);
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue(c, s, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_fail(c, e);
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        c->graph_exec = nullptr;
        return cuda_fail(c, ei);
    }
    c->graph = g;
    c->graph_launches = c->launches;
    return POLYLLA_OK;
}

int polylla_release_graph(polylla_ctx *c) {
    if (!c) return POLYLLA_ERR_INVALID_ARGUMENT;
    drop_graph(c);
    return POLYLLA_OK;
}

static int device_status(const DevCtrl &h) {
    if (h.error & DEV_ERR_INPUT) return POLYLLA_ERR_INVALID_MESH;
    if (h.error & DEV_ERR_NONTERMINATING) return POLYLLA_ERR_NONTERMINATING;
    if (h.error & DEV_ERR_CAPACITY) return POLYLLA_ERR_CAPACITY;
    if (h.error & DEV_ERR_TIMEOUT) return POLYLLA_ERR_TIMEOUT;
    return POLYLLA_OK;
}

static int read_ctrl(polylla_ctx *c, cudaStream_t s) {
    CK(cudaMemcpyAsync(c->h_ctrl, c->w.ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return POLYLLA_OK;
}

int polylla_get_polygons(polylla_ctx *c, polylla_polygons *out, polylla_stream stream) {
    if (!c || !out) return POLYLLA_ERR_INVALID_ARGUMENT;
    int rc = read_ctrl(c, (cudaStream_t)stream);
    if (rc) return rc;
    out->n_polygons = c->h_ctrl->n_polygons;
    out->n_frontier = c->h_ctrl->n_frontier;
    out->seeds = c->w.seeds;
    out->offsets = c->w.offsets;
    out->he_list = c->w.he_list;
    out->v_list = c->w.v_list;
    return device_status(*c->h_ctrl);
}

int polylla_last_error(polylla_ctx *c) {
    if (!c) return POLYLLA_ERR_INVALID_ARGUMENT;
    int rc = read_ctrl(c, c->last_stream);
    if (rc) return rc;
    return device_status(*c->h_ctrl);
}

int polylla_cuda_error(polylla_ctx *c) { return c ? (int)c->last_cuda : 0; }

int polylla_get_labels(polylla_ctx *c, polylla_labels *out, polylla_stream stream) {
    if (!c || !out) return POLYLLA_ERR_INVALID_ARGUMENT;
    int rc = read_ctrl(c, (cudaStream_t)stream);
    if (rc) return rc;
    out->longest_local = c->w.le;
    out->flags = c->w.flags;
    out->tips = c->w.tips;
    out->chords = c->w.chords;
    int32_t n = c->h_ctrl->n_tips;
    out->n_tips = n < c->w.tip_cap ? n : c->w.tip_cap;
    return device_status(*c->h_ctrl);
}

int polylla_generate_host(polylla_ctx *c, const polylla_host_mesh *in, polylla_host_result *out,
                          int32_t validate, polylla_stream stream) {
    if (!c || !in || !out || !c->owns_mesh || c->graph_exec) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!in->coords || !in->origin || !in->twin || !in->next || !in->prev) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!out->seeds || !out->offsets || !out->he_list || !out->v_list || !out->next || !out->prev)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t H = (size_t)c->mesh.H, V = (size_t)c->mesh.V, HI = 3 * (size_t)c->mesh.T;
    // In: the longest-edge stage needs only coords and origin; twin comes
    // in on the side stream meanwhile and the relink waits for it.  The
    // method never reads next/prev, so they go in only for the layout check.
    CK(cudaMemcpyAsync((void *)c->mesh.xy, in->coords, 16 * V, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)c->mesh.origin, in->origin, 4 * H, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)c->mesh.twin, in->twin, 4 * H, cudaMemcpyHostToDevice, c->aux));
    CK(cudaEventRecord(c->ev_twin, c->aux));
    if (validate) {
        CK(cudaMemcpyAsync(c->mesh.next, in->next, 4 * H, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->mesh.prev, in->prev, 4 * H, cudaMemcpyHostToDevice, s));
        CK(cudaStreamWaitEvent(s, c->ev_twin, 0));
        int rc = run_validate(c, s);
        if (rc) return rc;
    }
    // the stages; next/prev are final after stage 3 and go out on the side
    // stream while the polygon output stages run
    c->wait_before_relink = c->ev_twin;
    c->record_after_links = c->ev_links;
    const bool timing = c->timing;
    c->last_stream = s;
    c->timed_last = timing;
    int rc = enqueue(c, s, timing);
    c->wait_before_relink = nullptr;
    c->record_after_links = nullptr;
    if (rc) return rc;
    CK(cudaStreamWaitEvent(c->aux, c->ev_links, 0));
    CK(cudaMemcpyAsync(out->next, c->mesh.next, 4 * HI, cudaMemcpyDeviceToHost, c->aux));
    CK(cudaMemcpyAsync(out->prev, c->mesh.prev, 4 * HI, cudaMemcpyDeviceToHost, c->aux));
    // border half-edges are never written: their links are the input's
    if (H > HI) {
        memcpy(out->next + HI, in->next + HI, 4 * (H - HI));
        memcpy(out->prev + HI, in->prev + HI, 4 * (H - HI));
    }
    rc = read_ctrl(c, s);
    if (rc == POLYLLA_OK) rc = device_status(*c->h_ctrl);
    if (rc) {
        cudaStreamSynchronize(c->aux);
        return rc;
    }
    const int32_t P = c->h_ctrl->n_polygons, NF = c->h_ctrl->n_frontier;
    CK(cudaMemcpyAsync(out->seeds, c->w.seeds, 4 * (size_t)P, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->offsets, c->w.offsets, 4 * (size_t)(P + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->he_list, c->w.he_list, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->v_list, c->w.v_list, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamSynchronize(c->aux));
    out->n_polygons = P;
    out->n_frontier = NF;
    return POLYLLA_OK;
}

int polylla_set_timing(polylla_ctx *c, int32_t enable) {
    if (!c) return POLYLLA_ERR_INVALID_ARGUMENT;
    c->timing = enable != 0;
    return POLYLLA_OK;
}

int polylla_get_stage_times(polylla_ctx *c, float *ms, int32_t n) {
    if (!c || !ms || n < 0) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!c->timed_last) return 0;
    int last = -1;
    for (int i = 0; i < kStages; i++)
        if (c->stage_ran[i]) last = i;
    if (last < 0) return 0;
    CK(cudaEventSynchronize(c->ev_end[c->is_batch ? kMeta : kCore - 1]));
    const int k = n < kStages ? n : kStages;
    for (int i = 0; i < k; i++) {
        float t = 0.f;
        if (c->stage_ran[i]) CK(cudaEventElapsedTime(&t, c->ev_begin[i], c->ev_end[i]));
        ms[i] = t;
    }
    return k;
}

int polylla_stage_count(void) { return kStages; }

const char *polylla_stage_name(int32_t i) { return (i >= 0 && i < kStages) ? kStageNames[i] : ""; }

int polylla_launch_count(polylla_ctx *c) { return c ? c->launches : 0; }

void polylla_destroy(polylla_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

// ---- batches ------------------------------------------------------------------

int polylla_batch_create(polylla_ctx **out, const polylla_batch *b, const polylla_options *opt,
                         polylla_stream stream) {
    if (!out) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (!b || b->n_meshes < 1 || !b->vertex_offset || !b->triangle_offset || !b->halfedge_offset)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!b->coords || !b->origin || !b->twin || !b->next || !b->prev) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!aligned(b->coords, 16) || !aligned(b->origin, 4) || !aligned(b->twin, 4) || !aligned(b->next, 4) ||
        !aligned(b->prev, 4))
        return POLYLLA_ERR_INVALID_ARGUMENT;
    const int32_t n = b->n_meshes;
    const int32_t *vo = b->vertex_offset, *to = b->triangle_offset, *ho = b->halfedge_offset;
    if (vo[0] != 0 || to[0] != 0 || ho[0] != 0) return POLYLLA_ERR_INVALID_ARGUMENT;
    for (int32_t i = 0; i < n; i++) {
        const int64_t Vi = (int64_t)vo[i + 1] - vo[i], Ti = (int64_t)to[i + 1] - to[i], Hi = (int64_t)ho[i + 1] - ho[i];
        if (Vi < 3 || Ti < 1 || Hi < 3 * Ti + 3) return POLYLLA_ERR_INVALID_ARGUMENT;
    }
    int rc = check_sizes(vo[n], to[n], ho[n]);
    if (rc) return rc;
    polylla_ctx *c = new (std::nothrow) polylla_ctx();
    if (!c) return POLYLLA_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return POLYLLA_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = batch_alloc(c, n, vo[n], to[n], ho[n], b->coords, b->origin, b->twin, b->next, b->prev);
    BatchView &bv = c->bv;
    int32_t *d_off[4] = {const_cast<int32_t *>(bv.v_off), const_cast<int32_t *>(bv.t_off),
                         const_cast<int32_t *>(bv.h_off), const_cast<int32_t *>(bv.b_off)};
    if (!rc) {
        // border prefix sums b_off[i] = h_off[i] - 3 t_off[i]
        int32_t *h_b = new (std::nothrow) int32_t[(size_t)n + 1];
        if (!h_b) rc = POLYLLA_ERR_OUT_OF_MEMORY;
        else {
            for (int32_t i = 0; i <= n; i++) h_b[i] = ho[i] - 3 * to[i];
            const int32_t *src[4] = {vo, to, ho, h_b};
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < 4 && e == cudaSuccess; k++)
                e = cudaMemcpy(d_off[k], src[k], sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice);
            delete[] h_b;
            // the mesh table: the mesh of every SEG_SPAN-th triangle
            const int64_t ns = seg_count(to[n]);
            int32_t *h_seg = e == cudaSuccess ? new (std::nothrow) int32_t[(size_t)ns] : nullptr;
            if (e == cudaSuccess && !h_seg) rc = POLYLLA_ERR_OUT_OF_MEMORY;
            if (h_seg) {
                int32_t i = 0;
                for (int64_t g = 0; g < ns; g++) {
                    const int64_t t = std::min<int64_t>(g * SEG_SPAN, (int64_t)to[n] - 1);
                    while (i + 1 < n && to[i + 1] <= t) i++;
                    h_seg[g] = i;
                }
                e = cudaMemcpy(const_cast<int32_t *>(c->w.loc_seg), h_seg, sizeof(int32_t) * (size_t)ns,
                               cudaMemcpyHostToDevice);
                delete[] h_seg;
            }
            if (e != cudaSuccess) rc = cuda_fail(c, e);
        }
    }
    if (!rc) rc = alloc_work(c, opt);
    if (!rc) {
        c->w.loc_t_off = bv.t_off;
        c->w.loc_v_off = bv.v_off;
        c->w.loc_h_off = bv.h_off;
        c->w.loc_next = bv.next;
        c->w.loc_prev = bv.prev;
        c->w.loc_poly_off = c->poly_off;
        c->w.loc_n = n;
        if (!opt || opt->validate) {
            // range checks of every local index while packing all four
            // arrays, then the single-mesh layout check on the union
            cudaError_t e = cudaMemsetAsync(c->d_bad, 0, sizeof(int32_t), s);
            if (e == cudaSuccess) {
                launch_batch_pack(bv, c->u_origin, c->u_twin, c->mesh.next, c->mesh.prev, c->d_bad, nullptr, s);
                e = cudaGetLastError();
            }
            int32_t bad = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(c, e);
            else if (bad) rc = POLYLLA_ERR_INVALID_MESH;
            else rc = run_validate(c, s);
        }
    }
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return POLYLLA_OK;
}

int polylla_batch_polygon_offsets(polylla_ctx *c, const int32_t **poly_offset) {
    if (!c || !poly_offset || !c->is_batch) return POLYLLA_ERR_INVALID_ARGUMENT;
    *poly_offset = c->poly_off;
    return POLYLLA_OK;
}

// ---- tuning -------------------------------------------------------------------

int polylla_get_tuning(polylla_ctx *c, polylla_tuning *out) {
    if (!c || !out) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = current_tuning(c);
    return POLYLLA_OK;
}

int polylla_set_tuning(polylla_ctx *c, const polylla_tuning *t) {
    if (!c || !t || !tuning_valid(c, *t)) return POLYLLA_ERR_INVALID_ARGUMENT;
    drop_graph(c);
    apply_tuning(c, *t);
    return POLYLLA_OK;
}

int polylla_autotune(polylla_ctx *c, int32_t reps, polylla_tuning *out, polylla_stream stream) {
    if (!c || reps < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    drop_graph(c);
    const bool timing = c->timing;
    c->timing = true;
    const int sms = sm_count(c);
    // median time of stages [stage, last] over reps whole runs
    auto stage_ms = [&](int stage, int last, float *med) -> int {
        float v[64];
        const int r = reps < 64 ? reps : 64;
        for (int i = 0; i < r; i++) {
            int rc = polylla_generate(c, stream);
            if (rc) return rc;
            float ms[kStages];
            if (polylla_get_stage_times(c, ms, kStages) != kStages) return POLYLLA_ERR_CUDA;
            v[i] = 0.f;
            for (int k = stage; k <= last; k++) v[i] += ms[k];
        }
        for (int i = 1; i < r; i++)  // insertion sort, r is small
            for (int j = i; j > 0 && v[j] < v[j - 1]; j--) {
                float t = v[j];
                v[j] = v[j - 1];
                v[j - 1] = t;
            }
        *med = v[r / 2];
        return POLYLLA_OK;
    };
    // one knob per stage, tried in stage order: its candidates are whole
    // tunings that differ from the current one in that knob's fields only
    int rc = POLYLLA_OK;
    for (int q = 0; q < 3 && !rc; q++) {
        // relink, longest edge, the output kernels (count, scan, list)
        const int stage = q == 0 ? 1 : (q == 1 ? 0 : 4), last = q == 2 ? 6 : stage;
        polylla_tuning cand[16];
        int n = 0;
        const polylla_tuning cur = current_tuning(c);
        if (q == 0) {
            // relink tile and triangles per thread
            const int32_t pairs[][2] = {{64, 1}, {128, 1}, {256, 1}, {256, 2}, {256, 4}};
            for (const auto &pr : pairs)
                if (relink_config_valid(pr[0], pr[1])) {
                    cand[n] = cur;
                    cand[n].relink_tile = pr[0];
                    cand[n++].relink_items = pr[1];
                }
        } else if (q == 1) {
            // triangles per lane and persistent grid
            for (int32_t items : {2, 4}) {
                const int occ = longest_edge_blocks_per_sm(items);
                for (int k = 1; k <= occ && n < 16; k++) {
                    cand[n] = cur;
                    cand[n].longest_edge_items = items;
                    cand[n++].longest_edge_blocks = k * sms;
                }
            }
        } else {
            // output tile and triangles per thread (the launch configurations
            // the library is built with)
            const int32_t pairs[][2] = {{1024, 2}, {1024, 4}, {2048, 2}, {2048, 4}, {4096, 4}};
            for (const auto &pr : pairs)
                if (polygons_config_valid(pr[0], pr[1]) && polygons_blocks_per_sm(pr[0], pr[1]) > 0) {
                    cand[n] = cur;
                    cand[n].output_tile = pr[0];
                    cand[n++].output_items = pr[1];
                }
        }
        polylla_tuning best = cur;
        float best_ms = 0.f;
        rc = stage_ms(stage, last, &best_ms);
        for (int i = 0; i < n && !rc; i++) {
            if (memcmp(&cand[i], &best, sizeof(best)) == 0) continue;
            apply_tuning(c, cand[i]);
            float t = 0.f;
            rc = stage_ms(stage, last, &t);
            if (!rc && t < best_ms) {
                best_ms = t;
                best = cand[i];
            }
        }
        apply_tuning(c, best);
    }
    c->timing = timing;
    if (rc) return rc;
    const polylla_tuning t = current_tuning(c);
    if (c->device >= 0 && c->device < kTuneDevices) {
        std::lock_guard<std::mutex> g(g_tune_lock);
        g_tune[c->device][size_bucket(c->mesh.T)] = TuneEntry{true, t};
    }
    if (out) *out = t;
    return POLYLLA_OK;
}

int polylla_tuning_cache_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    for (int d = 0; d < kTuneDevices; d++)
        for (int b = 0; b < kTuneBuckets; b++) g_tune[d][b].set = false;
    return POLYLLA_OK;
}

// ---- Lepp ------------------------------------------------------------------------

int polylla_convexify(polylla_ctx *c, polylla_stream stream) {
    if (!c || c->is_batch) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->cv_list) {
        // every chord is a distinct non-frontier interior half-edge and
        // every reflex corner a frontier one: 3T bounds
        void *p = nullptr;
        int rc = dev_alloc(c, &p, sizeof(int32_t) * 3 * (size_t)c->mesh.T);
        if (rc) return rc;
        c->cv_list = (int32_t *)p;
        if ((rc = dev_alloc(c, &p, sizeof(int32_t) * 3 * (size_t)c->mesh.T))) return rc;
        c->cv_reflex = (int32_t *)p;
        if ((rc = dev_alloc(c, &p, 2 * sizeof(int32_t)))) return rc;
        c->cv_count = (int32_t *)p;
        c->cv_cap = 3 * c->mesh.T;
    }
    c->last_stream = s;
    const int32_t tile = polygons_config_valid(c->w.out_tile, c->w.out_items) ? c->w.out_tile : OUT_TILE_DEFAULT;
    const size_t n_tiles = ((size_t)c->mesh.T + tile - 1) / tile;
    CK(cudaMemsetAsync(c->cv_count, 0, 2 * sizeof(int32_t), s));
    CK(cudaMemsetAsync(c->w.tile_state, 0, sizeof(unsigned long long) * n_tiles, s));
    CK(cudaMemsetAsync(&c->w.ctrl->scan_done, 0, sizeof(int32_t), s));
    launch_convex_chords(c->mesh, c->w, c->cv_reflex, c->cv_count + 1, c->cv_list, c->cv_count, c->cv_cap, s);
    launch_convex_mark(c->mesh, c->w, c->cv_list, c->cv_count, c->cv_cap, s);
    launch_chord_links_list(c->mesh, c->w, c->cv_list, c->cv_count, c->cv_cap, s);
    launch_poly_count(c->mesh, c->w, s);
    launch_tile_scan(c->mesh, c->w, s);
    launch_poly_list(c->mesh, c->w, s);
    CK(cudaGetLastError());
    return POLYLLA_OK;
}

int polylla_convex_chords(polylla_ctx *c, const int32_t **chords, int32_t *n, polylla_stream stream) {
    if (!c || !chords || !n || c->is_batch) return POLYLLA_ERR_INVALID_ARGUMENT;
    *chords = c->cv_list;
    *n = 0;
    if (!c->cv_list) return POLYLLA_OK;
    int32_t h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(&h, c->cv_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n = h < c->cv_cap ? h : c->cv_cap;
    return POLYLLA_OK;
}

int polylla_lepp_terminal(polylla_ctx *c, int32_t *terminal, int32_t *length, polylla_stream stream) {
    if (!c || !terminal || c->is_batch || c->serve) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    launch_lepp_terminal(c->mesh, c->w, terminal, length, &c->w.ctrl->error, s);
    CK(cudaGetLastError());
    return POLYLLA_OK;
}

int polylla_lepp_paths(polylla_ctx *c, const int32_t *tri, int32_t n, int32_t *offsets, int32_t *paths,
                       int64_t capacity, polylla_stream stream) {
    if (!c || !tri || !offsets || (!paths && capacity > 0) || capacity < 0 || c->is_batch || c->serve)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    if (n < 1 || n > c->mesh.T) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    launch_lepp_paths(c->mesh, c->w, tri, n, offsets, paths, capacity, c->lepp_blk, c->lepp_blk_pre, c->lepp_total,
                      &c->w.ctrl->error, s);
    CK(cudaGetLastError());
    return POLYLLA_OK;
}

}  // extern "C"

// ---- serving slots (see polylla_serve.cuh) --------------------------------------

namespace polylla {

int serve_reserve(polylla_ctx **out, int32_t n_cap, int32_t V_cap, int32_t T_cap, int32_t H_cap,
                  const double *coords, const int32_t *origin, const int32_t *twin, int32_t *next, int32_t *prev,
                  int32_t max_rotation) {
    if (!out || n_cap < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    int rc = check_sizes(V_cap, T_cap, H_cap);
    if (rc) return rc;
    polylla_ctx *c = new (std::nothrow) polylla_ctx();
    if (!c) return POLYLLA_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return POLYLLA_ERR_CUDA;
    }
    c->serve = true;
    rc = batch_alloc(c, n_cap, V_cap, T_cap, H_cap, coords, origin, twin, next, prev);
    void *p = nullptr;
    if (!rc && (rc = dev_alloc(c, &p, sizeof(int32_t) * 4 * (size_t)n_cap)) == 0) c->meta = (int32_t *)p;
    if (!rc && (rc = dev_alloc(c, &p, sizeof(int32_t) * ((size_t)T_cap + n_cap + 1))) == 0)
        c->local_offsets = (int32_t *)p;
    polylla_options opt{0, max_rotation};
    if (!rc) rc = alloc_work(c, &opt);
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    c->w.loc_t_off = c->bv.t_off;
    c->w.loc_v_off = c->bv.v_off;
    c->w.loc_h_off = c->bv.h_off;
    c->w.loc_next = c->bv.next;
    c->w.loc_prev = c->bv.prev;
    c->w.loc_poly_off = c->poly_off;
    *out = c;
    return POLYLLA_OK;
}

size_t serve_bytes(const polylla_ctx *c) { return c ? c->bytes : 0; }

int serve_run(polylla_ctx *c, int32_t n, int32_t V, int32_t T, int32_t H, const int32_t *off4, cudaStream_t s) {
    if (!c || !c->serve || n < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    c->mesh.V = V;
    c->mesh.T = T;
    c->mesh.H = H;
    c->bv.n = n;
    c->bv.T_tot = T;
    c->bv.H_tot = H;
    c->w.loc_n = n;
    c->w.n_tile_max = (int32_t)(((int64_t)T + OUT_TILE_MIN - 1) / OUT_TILE_MIN);
    launch_serve_offsets(off4, n, const_cast<int32_t *>(c->bv.v_off), const_cast<int32_t *>(c->bv.t_off),
                         const_cast<int32_t *>(c->bv.h_off), const_cast<int32_t *>(c->bv.b_off), s);
    launch_batch_seg(c->bv.t_off, n, T, const_cast<int32_t *>(c->w.loc_seg), s);
    c->last_stream = s;
    c->timed_last = false;
    return enqueue(c, s, false);
}

void serve_outputs(const polylla_ctx *c, ServeOutputs *o) {
    o->seeds = c->w.seeds;
    o->local_offsets = c->local_offsets;
    o->he_list = c->w.he_list;
    o->v_list = c->w.v_list;
    o->meta = c->meta;
    o->ctrl = c->w.ctrl;
}

int serve_status(const DevCtrl &h) { return device_status(h); }

}  // namespace polylla
