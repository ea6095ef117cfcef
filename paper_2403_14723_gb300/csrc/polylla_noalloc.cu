// polylla_generate_noalloc: the whole method without any allocation.
//
// Some callers of this library cannot call cudaMalloc: a serving loop that
// must not allocate once it is running (an allocation can stall on the
// device or fail under a full memory budget), or a process whose device
// memory is entirely owned by another allocator, which a stray cudaMalloc
// would bypass or fragment.  This entry point runs the same kernels as
// polylla_generate, with every scratch buffer carved from one file-scope
// __device__ array of fixed size; the caller passes the mesh and the output
// buffers.  It allocates nothing and frees nothing, on the device or on the
// host.
#include <cstring>
#include <mutex>

#include "polylla.h"
#include "polylla_internal.cuh"

using namespace polylla;

namespace {

constexpr int32_t NA_MAX_T = POLYLLA_NOALLOC_MAX_TRIANGLES;
// a triangulated disk has V = (T + B + 2) / 2 with B <= T + 2 boundary edges
constexpr int32_t NA_MAX_V = NA_MAX_T + 2;
constexpr int64_t NA_MAX_TILES = ((int64_t)NA_MAX_T + OUT_TILE_MIN - 1) / OUT_TILE_MIN;

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
// layout of the scratch array (byte offsets, each 256-aligned)
constexpr size_t OFF_LE = 0;
constexpr size_t OFF_FLAGS = OFF_LE + up256(NA_MAX_T);
constexpr size_t OFF_TIPS = OFF_FLAGS + up256(NA_MAX_T);
constexpr size_t OFF_CHORDS = OFF_TIPS + up256(4 * (size_t)NA_MAX_V);
constexpr size_t OFF_TILES = OFF_CHORDS + up256(4 * (size_t)NA_MAX_V);
constexpr size_t OFF_TILE_PRE = OFF_TILES + up256(8 * (size_t)NA_MAX_TILES);
constexpr size_t OFF_GROUPS = OFF_TILE_PRE + up256(8 * (size_t)NA_MAX_TILES);
constexpr size_t OFF_GROUP_PRE = OFF_GROUPS + up256(8 * (size_t)(NA_MAX_TILES / SCAN_THREADS + 1));
constexpr size_t OFF_REC = OFF_GROUP_PRE + up256(8 * (size_t)(NA_MAX_TILES / SCAN_THREADS + 1));
constexpr size_t OFF_WTOT = OFF_REC + up256(8 * (size_t)out_rec_count(NA_MAX_T));
constexpr size_t OFF_CTRL = OFF_WTOT + up256(8 * (size_t)out_warp_count(NA_MAX_T));
constexpr size_t NA_BYTES = OFF_CTRL + up256(sizeof(DevCtrl));

constexpr int kMaxDevices = 64;

}  // namespace

// The scratch.  Every GPU that loads the library holds it (NA_BYTES, about
// 1.7 MB) until the process exits.  In host code its name is only a host-side
// stand-in: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

static std::mutex g_setup_lock;
static unsigned char *g_scratch_addr[kMaxDevices];  // device address per device, set once
static int g_sms[kMaxDevices];

// Set-up, once per device, on the current device (the first call there):
// look up the scratch array's device address, allow the relink and output
// kernels their shared memory, read the SM count.
static int device_setup(unsigned char **out, int *sms) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return POLYLLA_ERR_CUDA;
    if (d < 0 || d >= kMaxDevices) return POLYLLA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> guard(g_setup_lock);
    if (!g_scratch_addr[d]) {
        void *p = nullptr;
        int n = 0;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return POLYLLA_ERR_CUDA;
        if (polygons_configure() != 0 || relink_configure() != 0) return POLYLLA_ERR_CUDA;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) return POLYLLA_ERR_CUDA;
        g_sms[d] = n > 0 ? n : 1;
        g_scratch_addr[d] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[d];
    *sms = g_sms[d];
    return POLYLLA_OK;
}

extern "C" int polylla_generate_noalloc(const polylla_mesh *mesh, int32_t *seeds, int32_t *offsets,
                                        int32_t *he_list, int32_t *v_list, int32_t *status3,
                                        polylla_stream stream) {
    if (!mesh || !seeds || !offsets || !he_list || !v_list || !status3) return POLYLLA_ERR_INVALID_ARGUMENT;
    const int32_t V = mesh->n_vertices, T = mesh->n_triangles, H = mesh->n_halfedges;
    if (V < 3 || T < 1 || (int64_t)H < 3 * (int64_t)T + 3) return POLYLLA_ERR_INVALID_ARGUMENT;
    if (T > NA_MAX_T || V > NA_MAX_V) return POLYLLA_ERR_TOO_LARGE;
    if (!mesh->coords || !mesh->origin || !mesh->twin || !mesh->next || !mesh->prev)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    auto aligned16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (!aligned16(mesh->coords) || !aligned16(mesh->origin) || !aligned16(mesh->twin) ||
        !aligned16(mesh->next) || !aligned16(mesh->prev))
        return POLYLLA_ERR_INVALID_ARGUMENT;
    // an error the caller left pending would be taken for one of ours by
    // the launch check below: report it, leave it pending, launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return POLYLLA_ERR_CUDA;
    unsigned char *base = nullptr;
    int sms = 1;
    int rc = device_setup(&base, &sms);
    if (rc) return rc;

    MeshView m{};
    m.V = V;
    m.T = T;
    m.H = H;
    m.xy = reinterpret_cast<const double2 *>(mesh->coords);
    m.origin = mesh->origin;
    m.twin = mesh->twin;
    m.next = mesh->next;
    m.prev = mesh->prev;
    Work w{};
    w.le = base + OFF_LE;
    w.flags = base + OFF_FLAGS;
    w.tips = reinterpret_cast<int32_t *>(base + OFF_TIPS);
    w.chords = reinterpret_cast<int32_t *>(base + OFF_CHORDS);
    w.tip_cap = V;
    w.tile_state = reinterpret_cast<unsigned long long *>(base + OFF_TILES);
    w.tile_pre = reinterpret_cast<unsigned long long *>(base + OFF_TILE_PRE);
    w.group_tot = reinterpret_cast<unsigned long long *>(base + OFF_GROUPS);
    w.group_pre = reinterpret_cast<unsigned long long *>(base + OFF_GROUP_PRE);
    w.poly_rec = reinterpret_cast<unsigned long long *>(base + OFF_REC);
    w.poly_wtot = reinterpret_cast<unsigned long long *>(base + OFF_WTOT);
    w.n_tile_max = (int32_t)(((int64_t)T + OUT_TILE_MIN - 1) / OUT_TILE_MIN);
    w.seeds = seeds;
    w.offsets = offsets;
    w.he_list = he_list;
    w.v_list = v_list;
    w.ctrl = reinterpret_cast<DevCtrl *>(base + OFF_CTRL);
    w.max_rot = 4096;
    w.persistent_blocks = 4 * sms;
    w.le_items = LE_ITEMS_DEFAULT;
    w.le_blocks = longest_edge_blocks_per_sm(LE_ITEMS_DEFAULT) * sms;
    w.out_tile = OUT_TILE_DEFAULT;
    w.out_items = OUT_ITEMS_DEFAULT;
    w.rl_tile = RL_TILE_DEFAULT;
    w.rl_items = RL_ITEMS_DEFAULT;

    // The first kernel zeroes the control block (counters) and the output
    // tiles' totals; every other scratch word is written
    // before it is read, so the previous call's contents never leak into
    // this one.
    cudaStream_t s = (cudaStream_t)stream;
    launch_longest_edge(m, w, s);
    launch_label_relink(m, w, s);
    launch_chords(m, w, s);
    launch_chord_links(m, w, s);
    launch_poly_count(m, w, s);
    launch_tile_scan(m, w, s);
    launch_poly_list(m, w, s);
    // status3 = {P, N_F, device error bits}, copied device to device
    if (cudaMemcpyAsync(status3, &w.ctrl->n_polygons, 2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(status3 + 2, &w.ctrl->error, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return POLYLLA_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return POLYLLA_ERR_CUDA;
    return POLYLLA_OK;
}
