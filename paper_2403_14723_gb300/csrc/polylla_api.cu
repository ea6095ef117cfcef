// Host side of the C ABI declared in include/polylla.h: context lifetime,
// argument checks, the kernel sequence of polylla_generate, and readback.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/polylla.h"
#include "polylla_internal.cuh"

using namespace polylla;

namespace {

constexpr int kStages = 10;
const char *kStageNames[kStages] = {
    "longest_edge", "label_relink", "chords", "chord_links", "cand_count",
    "cand_scan", "cand_write", "walk", "chunk_scan", "emit",
};
constexpr int kKernels = 11;  // chunk_scan launches two kernels

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
    cudaEvent_t ev[kStages + 1]{};
    bool timed_last = false;
    int launches = 0;
    cudaStream_t last_stream = nullptr;
    // device allocations (for destroy)
    void *allocs[32]{};
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
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->allocs[c->n_allocs++] = *p;
    return POLYLLA_OK;
}

static void free_all(polylla_ctx *c) {
    for (int i = 0; i < c->n_allocs; i++) cudaFree(c->allocs[i]);
    c->n_allocs = 0;
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    c->h_ctrl = nullptr;
    for (int i = 0; i <= kStages; i++) {
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
        c->ev[i] = nullptr;
    }
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_sizes(int32_t V, int32_t T, int32_t H) {
    if (V < 3 || T < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    if ((int64_t)T * 3 >= (int64_t)INT32_MAX) return POLYLLA_ERR_INVALID_ARGUMENT;
    if ((int64_t)H < 3 * (int64_t)T + 3) return POLYLLA_ERR_INVALID_ARGUMENT;
    return POLYLLA_OK;
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
    c->w.n_cc_blocks = (int32_t)(((int64_t)T + CC_TRI - 1) / CC_TRI);
    c->w.n_chunk_max = (int32_t)((HI + CHUNK - 1) / CHUNK);
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_cc_blocks))) return rc;
    c->w.blk_a = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_cc_blocks))) return rc;
    c->w.blk_a_pre = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_chunk_max))) return rc;
    c->w.blk_b = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)c->w.n_chunk_max))) return rc;
    c->w.blk_b_pre = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(unsigned long long) * (size_t)((HI + 31) / 32)))) return rc;
    c->w.grp = (unsigned long long *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)HI))) return rc;
    c->w.cand = (int32_t *)p;
    if ((rc = dev_alloc(c, &p, sizeof(int32_t) * (size_t)HI))) return rc;
    c->w.res = (int32_t *)p;
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
    if ((rc = dev_alloc(c, &p, sizeof(int32_t)))) return rc;
    c->d_bad = (int32_t *)p;
    cudaError_t e = cudaMallocHost((void **)&c->h_ctrl, sizeof(DevCtrl));
    if (e != cudaSuccess) return cuda_fail(c, e);
    memset(c->h_ctrl, 0, sizeof(DevCtrl));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->w.persistent_blocks = 4 * (sms > 0 ? sms : 1);
    c->w.le_blocks = longest_edge_blocks_per_sm() * (sms > 0 ? sms : 1);
    c->w.walk_blocks = 8 * (sms > 0 ? sms : 1);
    c->w.emit_blocks = emit_blocks_per_sm() * (sms > 0 ? sms : 1);
    if (polygons_configure() != 0) return cuda_fail(c, cudaGetLastError());
    c->w.max_rot = (opt && opt->max_rotation > 0) ? opt->max_rotation : 4096;
    for (int i = 0; i <= kStages; i++) {
        e = cudaEventCreate(&c->ev[i]);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    return POLYLLA_OK;
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
        case POLYLLA_ERR_TOO_LARGE: return "mesh larger than the no-allocation scratch";
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
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return POLYLLA_OK;
}

int polylla_generate(polylla_ctx *c, polylla_stream stream) {
    if (!c) return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    c->timed_last = c->timing;
    c->launches = 0;
    if (c->timing) CK(cudaEventRecord(c->ev[0], s));
    void (*stages[kStages])(const MeshView &, const Work &, cudaStream_t) = {
        launch_longest_edge, launch_label_relink, launch_chords, launch_chord_links,
        launch_cand_count, launch_cand_scan, launch_cand_write, launch_walk,
        launch_chunk_scan, launch_emit,
    };
    for (int i = 0; i < kStages; i++) {
        stages[i](c->mesh, c->w, s);
        if (c->timing) CK(cudaEventRecord(c->ev[i + 1], s));
    }
    c->launches = kKernels;
    CK(cudaGetLastError());
    return POLYLLA_OK;
}

static int device_status(const DevCtrl &h) {
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
    if (!c || !in || !out || !c->owns_mesh) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!in->coords || !in->origin || !in->twin || !in->next || !in->prev) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!out->seeds || !out->offsets || !out->he_list || !out->v_list || !out->next || !out->prev)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t H = (size_t)c->mesh.H, V = (size_t)c->mesh.V;
    CK(cudaMemcpyAsync((void *)c->mesh.xy, in->coords, 16 * V, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)c->mesh.origin, in->origin, 4 * H, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void *)c->mesh.twin, in->twin, 4 * H, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->mesh.next, in->next, 4 * H, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->mesh.prev, in->prev, 4 * H, cudaMemcpyHostToDevice, s));
    if (validate) {
        int rc = run_validate(c, s);
        if (rc) return rc;
    }
    int rc = polylla_generate(c, stream);
    if (rc) return rc;
    rc = read_ctrl(c, s);
    if (rc) return rc;
    rc = device_status(*c->h_ctrl);
    if (rc) return rc;
    const int32_t P = c->h_ctrl->n_polygons, NF = c->h_ctrl->n_frontier;
    CK(cudaMemcpyAsync(out->seeds, c->w.seeds, 4 * (size_t)P, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->offsets, c->w.offsets, 4 * (size_t)(P + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->he_list, c->w.he_list, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->v_list, c->w.v_list, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->next, c->mesh.next, 4 * H, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->prev, c->mesh.prev, 4 * H, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
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
    CK(cudaEventSynchronize(c->ev[kStages]));
    int k = n < kStages ? n : kStages;
    for (int i = 0; i < k; i++) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
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

}  // extern "C"
