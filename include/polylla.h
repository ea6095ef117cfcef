/*
 * polylla.h -- C ABI of the GB300 Polylla library (libpolylla).
 *
 * Turns a triangulation stored as device-resident half-edge arrays into the
 * Polylla polygonal mesh of "GPolylla: Fully GPU-accelerated polygonal mesh
 * generator" (arXiv 2403.14723): terminal-edge regions (Definitions 1-3,
 * Section 3.1), joined by relinking next/prev of the frontier half-edges
 * (Section 4.2, Fig. 3), with non-simple regions split at barrier tips
 * (Section 5.3, Algorithm 6; Section 6.4, Algorithm 11).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - All array pointers in polylla_mesh and polylla_polygons are DEVICE
 *   pointers of the current CUDA device; coords are float64, topology int32.
 * - Mesh layout (the paper's implicit face indexing, Section 4.2): interior
 *   half-edges are [0, 3T); triangle t owns 3t, 3t+1, 3t+2, counter-
 *   clockwise, so next(e) = 3*(e/3) + (e+1)%3 and prev(e) = 3*(e/3) + (e+2)%3
 *   for e < 3T.  Border half-edges are [3T, H): each is the twin of an
 *   interior half-edge on the domain boundary and their next/prev walk the
 *   exterior face.  coords is [V][2] interleaved (x, y), 16-byte aligned.
 * - A "stream" is a cudaStream_t (NULL = the legacy default stream).  Unless
 *   stated otherwise a call only enqueues work on that stream and returns.
 * - Every int-returning call returns POLYLLA_OK (0) or a negative status.
 *   Status strings come from polylla_status_string().  A context is not
 *   thread-safe; distinct contexts are independent.
 * - The library never falls back to the CPU: without a usable CUDA device
 *   polylla_create fails with POLYLLA_ERR_CUDA.
 */
#ifndef POLYLLA_H
#define POLYLLA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct polylla_ctx polylla_ctx;
typedef struct CUstream_st *polylla_stream; /* same type as cudaStream_t */

enum polylla_status {
    POLYLLA_OK = 0,
    POLYLLA_ERR_INVALID_ARGUMENT = -1, /* NULL pointer, bad size, misaligned coords  */
    POLYLLA_ERR_INVALID_MESH = -2,     /* layout check failed at create             */
    POLYLLA_ERR_OUT_OF_MEMORY = -3,    /* cudaMalloc failed                          */
    POLYLLA_ERR_CUDA = -4,             /* any other CUDA error (see polylla_cuda_error) */
    POLYLLA_ERR_NONTERMINATING = -5,   /* a rotation or cycle walk hit its cap       */
    POLYLLA_ERR_CAPACITY = -6,         /* an internal list overflowed its capacity   */
    POLYLLA_ERR_TIMEOUT = -7,          /* a device wait gave up                      */
    POLYLLA_ERR_TOO_LARGE = -8,        /* mesh larger than the capacity available:    */
                                       /* the no-allocation scratch, or a server slot */
};

/* Input mesh (device arrays owned by the caller). */
typedef struct {
    int32_t n_vertices;   /* V >= 3                                     */
    int32_t n_triangles;  /* T >= 1, 3T < 2^31                          */
    int32_t n_halfedges;  /* H = 3T + number of border half-edges (>= 3) */
    const double *coords; /* [V][2] float64, 16-byte aligned            */
    const int32_t *origin; /* [H] vertex each half-edge leaves           */
    const int32_t *twin;   /* [H] opposite half-edge                      */
    int32_t *next;         /* [H] read by create's layout check; generate  */
    int32_t *prev;         /* [H] rewrites entries [0, 3T) (see below)     */
} polylla_mesh;

typedef struct {
    int32_t validate;      /* nonzero: check the mesh layout at create (default on);
                              with 0 the caller guarantees the layout: the
                              kernels index with the input values unchecked */
    int32_t max_rotation;  /* cap on one vertex rotation (0: 4096)               */
} polylla_options;

/* Output polygons (device arrays owned by the context). */
typedef struct {
    int32_t n_polygons;       /* P                                           */
    int32_t n_frontier;       /* N_F = total polygon length                  */
    const int32_t *seeds;     /* [P]   smallest half-edge of each polygon, ascending */
    const int32_t *offsets;   /* [P+1] polygon p is he_list[offsets[p] .. offsets[p+1]) */
    const int32_t *he_list;   /* [N_F] half-edges of each polygon from its seed along next */
    const int32_t *v_list;    /* [N_F] origin of each listed half-edge        */
} polylla_polygons;

/*
 * polylla_create -- validate a mesh and allocate every buffer generate needs.
 *   out    receives the new context (NULL on failure).
 *   mesh   device arrays, not copied: they must stay valid and keep their
 *          layout until polylla_destroy.  coords/origin/twin are only read.
 *   opt    NULL for defaults.
 *   stream used for the layout check; create synchronizes this stream.
 * Allocates scratch and output buffers sized from V, T and H (about
 * 8 bytes per triangle of scratch plus 4*(T + T+1 + 3T + 3T) bytes of
 * output); polylla_generate then allocates and frees nothing (the paper's
 * point in Section 4.2: the method runs in the input's own memory).
 * Errors: INVALID_ARGUMENT, INVALID_MESH (twin not an involution without
 * fixed points, interior next/prev not the implicit triangle layout,
 * origin(next e) != origin(twin e), border links inconsistent, an index
 * out of range, a non-finite coordinate), OUT_OF_MEMORY, CUDA.
 */
int polylla_create(polylla_ctx **out, const polylla_mesh *mesh,
                   const polylla_options *opt, polylla_stream stream);

/*
 * polylla_generate -- run the whole method on the context's mesh.
 * Enqueues, on stream, the five stages of the hot path:
 *   (1) longest edge of each triangle (Algorithm 2 / 8): squared float64
 *       lengths dx*dx + dy*dy, each operation rounded to nearest, no FMA;
 *       equal lengths go to the smaller edge id min(e, twin e);
 *   (2) frontier labels (Algorithm 3 / 9): e is frontier iff e or twin(e)
 *       is a border half-edge, or neither is a longest edge;
 *   (3) terminal and border-terminal seeds (Algorithm 4 / 10);
 *   (4) relinking (Section 4.2, Algorithm 5 / 12): for every frontier
 *       interior half-edge e, next(e) = the first frontier half-edge met
 *       rotating clockwise about target(e) from the triangle's next, and
 *       prev of that half-edge = e;
 *   (5) repair (Algorithm 6 / 11): a vertex with one frontier edge f is a
 *       barrier tip of degree d; its chord is CW^r(f), r = floor((d-1)/2)+1,
 *       found with the stage-2 labels; chords join the frontier and the
 *       links around their endpoints are redone; then every polygon (each
 *       cycle of next) is found, keyed by its smallest half-edge and written
 *       as a scan-compacted CSR list (Section 6.8).
 * On completion next/prev of every interior half-edge [0, 3T) hold the
 * polygon mesh: polygon links for frontier half-edges, the triangle links
 * for the rest (the values create validated).  Border half-edges are not
 * written.  The input next/prev of interior half-edges are never read, so
 * generate may be called again on the same mesh and gives the same result.
 * Asynchronous; no allocation, no host synchronization.  Device-side
 * failures (NONTERMINATING, CAPACITY, TIMEOUT) are recorded in the context
 * and reported by polylla_get_polygons / polylla_last_error.
 */
int polylla_generate(polylla_ctx *ctx, polylla_stream stream);

/*
 * polylla_get_polygons -- read the polygon count and hand out the CSR.
 * Copies 32 bytes device->host on stream and synchronizes it.  The device
 * arrays stay owned by the context and valid until the next generate or
 * destroy.  Returns the recorded device status if the last generate failed.
 */
int polylla_get_polygons(polylla_ctx *ctx, polylla_polygons *out, polylla_stream stream);

/* Status of the last generate (synchronizes the context's last stream). */
int polylla_last_error(polylla_ctx *ctx);

/* CUDA error code behind the last POLYLLA_ERR_CUDA (cudaError_t as int). */
int polylla_cuda_error(polylla_ctx *ctx);

/* Free every buffer of the context (synchronizes the device first). */
void polylla_destroy(polylla_ctx *ctx);

/* Static string for a status code. */
const char *polylla_status_string(int status);

/*
 * Intermediate labels, for stage-by-stage checks (not needed to use the
 * output).  Device arrays owned by the context, valid after a generate
 * completes and until the next generate or destroy:
 *   longest_local [T] uint8: local index k (0..2) of triangle t's longest
 *                 half-edge 3t+k (stage 1);
 *   flags [T] uint8: bits 0-2 frontier after repair (F1) of 3t+k (the
 *                 stage-2 frontier F0 is F1 without the chord half-edges),
 *                 bits 3-5 walk-start marks: set on every frontier
 *                 half-edge that may be the smallest of its polygon (a
 *                 superset of the seeds), bit 6 set when the triangle's
 *                 longest half-edge is the seed of its terminal-edge region
 *                 (stage 3);
 *   tips [n_tips] int32: for each barrier tip, the stage-2 frontier
 *                 half-edge leaving it (order unspecified);
 *   chords [n_tips] int32: the chord half-edge leaving the same tip.
 * n_tips is copied to the host (synchronizes stream).
 */
typedef struct {
    const uint8_t *longest_local;
    const uint8_t *flags;
    const int32_t *tips;
    const int32_t *chords;
    int32_t n_tips;
} polylla_labels;
int polylla_get_labels(polylla_ctx *ctx, polylla_labels *out, polylla_stream stream);

/*
 * Host-buffer path (end-to-end use): a context that owns device copies of
 * the mesh.  polylla_create_host allocates device arrays for a mesh of the
 * given sizes (no data yet); polylla_generate_host copies the host mesh in,
 * generates, and copies the polygons and the rewritten next/prev back.
 * Copies overlap the kernels where the method allows: twin is copied while
 * the longest-edge stage runs on coords and origin, and next/prev (final
 * after the repair) are copied back while the polygon output runs; the
 * input next/prev are only copied (and the layout checked) when validate is
 * nonzero, since the method does not read them; the border entries of the
 * output next/prev are the input's, copied on the host.  Host buffers
 * should be pinned (cudaHostAlloc) for full copy speed; any host memory
 * works.  Capacities of the outputs: seeds T, offsets T+1, he_list and
 * v_list 3T, next and prev H.  *n_polygons and *n_frontier receive P and
 * N_F.  Synchronizes stream (and the context's side stream) before
 * returning; not available while a graph is captured.
 */
typedef struct {
    const double *coords;
    const int32_t *origin, *twin, *next, *prev;
} polylla_host_mesh;
typedef struct {
    int32_t *seeds, *offsets, *he_list, *v_list;
    int32_t *next, *prev;
    int32_t n_polygons, n_frontier;
} polylla_host_result;
int polylla_create_host(polylla_ctx **out, int32_t n_vertices, int32_t n_triangles,
                        int32_t n_halfedges, const polylla_options *opt);
int polylla_generate_host(polylla_ctx *ctx, const polylla_host_mesh *in,
                          polylla_host_result *out, int32_t validate, polylla_stream stream);

/*
 * Per-stage timing.  With timing enabled, generate records a pair of CUDA
 * events around each stage it runs (on the generate stream);
 * polylla_get_stage_times synchronizes and writes the milliseconds of up to
 * n stages of the last generate (0 for a stage that did not run: the
 * batch stage on a single mesh), returning how many it wrote, or 0 when
 * the last generate was not timed (timing off, or a captured graph).
 * polylla_stage_name gives the name of stage i: the seven kernels of the
 * method ("longest_edge", "label_relink", "chords", "chord_links",
 * "poly_count", "tile_scan", "poly_list"), then "batch_meta" (the serving
 * loop's per-mesh metadata).
 * polylla_launch_count gives the number of kernels the last generate
 * launched (7 for a mesh or a batch, 8 for a served batch).
 */
int polylla_set_timing(polylla_ctx *ctx, int32_t enable);
int polylla_get_stage_times(polylla_ctx *ctx, float *ms, int32_t n);
int polylla_stage_count(void);
const char *polylla_stage_name(int32_t i);
int polylla_launch_count(polylla_ctx *ctx);

/*
 * Batches (no counterpart in the paper, whose method takes one mesh).
 *
 * n independent triangulations, each in the single-mesh layout above with
 * its own local indices (vertex ids from 0, interior half-edges [0, 3T_i),
 * border half-edges [3T_i, H_i)), concatenated: mesh i's vertices are rows
 * [vertex_offset[i], vertex_offset[i+1]) of coords and its half-edges
 * entries [halfedge_offset[i], halfedge_offset[i+1]) of origin/twin/next/
 * prev.  The offset arrays are HOST prefix sums with n+1 entries starting
 * at 0 (copied at create); every mesh has V_i >= 3, T_i >= 1,
 * H_i >= 3 T_i + 3; the totals obey the single-mesh limits.
 *
 * polylla_batch_create validates every mesh (as polylla_create, plus range
 * checks of each local index) and allocates for the whole batch: scratch
 * as for one mesh of the total size plus 16 bytes per half-edge for the
 * batch's union.  The device arrays are not copied and must stay valid.
 * polylla_generate on a batch context runs the method once over all meshes
 * -- one launch per stage, not one per mesh, reading each mesh's own
 * arrays (no copy into the union) -- and gives each mesh exactly
 * what polylla_generate gives it alone: next/prev of its interior half-
 * edges are rewritten in its local indices; polylla_get_polygons returns
 * one CSR for the batch, ordered by mesh and then by seed, with seeds,
 * he_list and v_list in each mesh's local indices and offsets into the
 * batch's he_list.  polylla_batch_polygon_offsets hands out a device array
 * of n+1 entries, valid after a generate completes: mesh i owns polygons
 * [poly_offset[i], poly_offset[i+1]).  polylla_get_labels reports the
 * union's labels (triangles in batch order).  polylla_generate_host does
 * not take a batch context.
 */
typedef struct {
    int32_t n_meshes;
    const int32_t *vertex_offset;   /* HOST [n+1] */
    const int32_t *triangle_offset; /* HOST [n+1] */
    const int32_t *halfedge_offset; /* HOST [n+1] */
    const double *coords;           /* DEVICE [V_total][2], 16-byte aligned */
    const int32_t *origin, *twin;   /* DEVICE [H_total], local indices */
    int32_t *next, *prev;           /* DEVICE [H_total], local; interior entries rewritten */
} polylla_batch;
int polylla_batch_create(polylla_ctx **out, const polylla_batch *batch,
                         const polylla_options *opt, polylla_stream stream);
int polylla_batch_polygon_offsets(polylla_ctx *ctx, const int32_t **poly_offset);

/*
 * CUDA graphs.  polylla_capture_graph records one whole generate of the
 * context (its kernels, with the current launch settings) into a CUDA graph
 * on stream (which must not be NULL, the legacy stream cannot be captured);
 * from then on polylla_generate launches that graph, one launch instead of
 * 7 or 9, untimed.  Changing the launch settings (polylla_set_tuning,
 * polylla_autotune) or polylla_release_graph drops the graph.  The graph
 * reads and writes the same device arrays as the captured generate.
 */
int polylla_capture_graph(polylla_ctx *ctx, polylla_stream stream);
int polylla_release_graph(polylla_ctx *ctx);

/*
 * Launch tuning (results never depend on it).  relink_tile is the triangles
 * per CTA of the relink kernel and relink_items the triangles each of its
 * threads labels and links: (64, 1), (128, 1), (256, 1), (256, 2) or
 * (256, 4); longest_edge_items the triangles per lane of the persistent
 * longest-edge kernel (2 or 4) and longest_edge_blocks its grid (blocks,
 * in [1, 64 * SMs]); output_tile the triangles per tile of the output
 * kernels and output_items the triangles each of their threads walks and
 * lists: (1024, 2), (1024, 4), (2048, 2), (2048, 4) or (4096, 4) (blocks
 * of tile / items threads).
 * polylla_autotune times whole generates (reps per setting, median of the
 * stage's CUDA-event time), tries the candidates of one setting at a time in
 * stage order and keeps the fastest, applies the result to the context,
 * stores it in a process-wide table per device and size bucket
 * (floor(log2 T), T the mesh's or batch's triangle count) that contexts
 * created later start from, and writes it to *out (may be NULL).  It runs
 * generate on the context's mesh (idempotent) and synchronizes stream.
 * polylla_tuning_cache_clear empties the table.
 */
typedef struct {
    int32_t relink_tile;
    int32_t relink_items;
    int32_t longest_edge_blocks;
    int32_t longest_edge_items;
    int32_t output_tile;
    int32_t output_items;
} polylla_tuning;
int polylla_get_tuning(polylla_ctx *ctx, polylla_tuning *out);
int polylla_set_tuning(polylla_ctx *ctx, const polylla_tuning *tuning);
int polylla_autotune(polylla_ctx *ctx, int32_t reps, polylla_tuning *out, polylla_stream stream);
int polylla_tuning_cache_clear(void);

/*
 * Convexification (post-processing; Section 4.2 keeps every half-edge of
 * the triangulation, relinking instead of deleting, so that a later step
 * can turn non-convex polygons into convex ones -- the paper gives no
 * method, so this is the library's own rule).  polylla_convexify runs on the
 * context's last generate (same stream, after it) and splits every reflex
 * corner of every polygon with the fewest edges of the triangulation
 * itself:
 *   - the corner at a frontier half-edge e is (e, x = next(e)) at
 *     v = target(e); with directions leaving v (dir(h) = target(h) - v,
 *     the corner's first side twin(e), dir = origin(e) - v) and
 *     cross(a, b) = a.x b.y - a.y b.x in binary64 (each operation rounded
 *     to nearest, no FMA), the corner is reflex iff cross(dir twin e,
 *     dir x) > 0;
 *   - from cur = twin(e), the last of the corner's interior half-edges
 *     (clockwise from the triangle's next of e, the relink's rotation)
 *     within a half turn clockwise of cur (cross <= 0) becomes a chord and
 *     the new cur, until x lies within a half turn of cur.
 * Both halves of every chord join the frontier (flags bits 0-2 of
 * polylla_get_labels then hold this frontier), next/prev around the chord
 * ends are relinked as by the repair, and polylla_get_polygons returns the
 * convex polygons (same canonical order).  Every corner of the result
 * turns by at most a half turn.  The first call allocates its chord and
 * reflex-corner lists (2 x 4 x 3T bytes); later calls allocate nothing.  Single-mesh contexts only
 * (INVALID_ARGUMENT on a batch).  Asynchronous; device errors through
 * polylla_last_error.  polylla_convex_chords gives the chosen half-edges of
 * the last convexify (device pointer owned by the context, *n of them, each
 * leaving its corner's vertex; one host synchronization).
 */
int polylla_convexify(polylla_ctx *ctx, polylla_stream stream);
int polylla_convex_chords(polylla_ctx *ctx, const int32_t **chords, int32_t *n, polylla_stream stream);

/*
 * Longest-edge propagation paths (Definition 1, Section 3.1; Section 1
 * lists a data-parallel Lepp among the paper's contributions, as a building
 * block for Lepp-based refinement).  Lepp(t0) = t0, t1, ...: t_i is the
 * neighbour of t_{i-1} across the longest edge of t_{i-1}; the path ends at
 * the terminal edge, the longest edge of both of its triangles (both are
 * listed), or at a longest edge on the border.  Both calls use the longest
 * edges of the context's last generate (so they follow it on the same
 * stream), are asynchronous, and report a device error (NONTERMINATING,
 * CAPACITY, INVALID_MESH for a query outside [0, T)) through
 * polylla_last_error until the next generate.  Single-mesh contexts only
 * (INVALID_ARGUMENT on a batch).
 *
 * polylla_lepp_terminal: for every triangle t, terminal[t] = the seed
 *   half-edge of the terminal edge its Lepp ends on -- the smaller half of
 *   an interior terminal edge, the interior half of a border one -- which
 *   names t's terminal-edge region (Definition 2); length[t] (may be NULL)
 *   = the number of triangles in Lepp(t).  Device arrays of T int32.
 * polylla_lepp_paths: the paths of n query triangles tri[0..n) (device,
 *   1 <= n <= T): offsets[n+1] (device) gets the exclusive prefix of the
 *   path lengths, offsets[n] the total, and paths[capacity] (device) the
 *   triangles of every path in query order; past the capacity paths are
 *   cut and CAPACITY is reported.
 */
int polylla_lepp_terminal(polylla_ctx *ctx, int32_t *terminal, int32_t *length, polylla_stream stream);
int polylla_lepp_paths(polylla_ctx *ctx, const int32_t *tri, int32_t n, int32_t *offsets, int32_t *paths,
                       int64_t capacity, polylla_stream stream);

/*
 * Serving (no counterpart in the paper): a request loop with continuous
 * batching.  Requests are meshes in host memory (pinned for full copy
 * speed); a scheduler thread owned by the server admits them, in arrival
 * order, into batches as batch slots and their device memory free up, and
 * runs each batch as one batched generate (see polylla_batch_create) on the
 * slot's own stream: copies in, the method, copies out.  Slots overlap on
 * the device (one copies in while another computes and a third copies
 * out), and requests that arrive while batches are in flight join the next
 * batch a slot forms -- no request waits for a fixed batch to fill.
 *
 * Memory: the server holds at most memory_budget bytes of device memory,
 * split into the lane (below) and n_slots copy-engine slots of equal
 * capacity (triangles, vertices, half-edges, meshes), all allocated at
 * create; a batch is admitted into a slot only while it fits the slot's
 * capacity.  A request larger than a copy-engine slot (and not a lane
 * request) completes with POLYLLA_ERR_TOO_LARGE.
 *
 * A request's result is exactly what polylla_generate_host gives for the
 * mesh alone, whatever it was batched with: CSR and next/prev in the
 * mesh's own indices, written to the request's host buffers (capacities as
 * polylla_generate_host).  The host arrays of a request must stay valid
 * and unchanged until it completes.  In a copy-engine batch each request
 * completes as soon as its own results have landed (an event after its
 * copies out; up to 32 per batch, consecutive requests sharing one beyond
 * that), not when the whole batch's have.
 *
 * Copies: the copy engines run one direction's copies in issue order across
 * all streams, so a small batch's copies would wait behind a large one's.
 * Unless lane_triangles < 0 the server adds a low-latency lane (slot 0) to
 * the n_slots copy-engine slots: a small slot (room for 16 requests of
 * lane_triangles, within budget / (n_slots + 1)) that batches only
 * requests of at most lane_triangles triangles whose nine device-touched
 * arrays (coords, origin, twin and the six results) are pinned host
 * memory, runs on the device's highest-priority stream, and moves their
 * data with kernels through host-mapped memory, never through a copy
 * engine.  The copy-engine slots split the rest of the budget and take the
 * remaining requests in arrival order (and lane requests that have waited
 * more than 5 ms); their data goes through the copy engines (full duplex),
 * while offsets, metadata and control blocks of every batch move by
 * kernel.  Pageable requests are served too, through the copy engines.
 *
 * Requests are not layout-checked (that would cost a pass per batch), but
 * the longest-edge kernel range-checks every interior origin and twin (the
 * only entries the method reads): an index outside its mesh is replaced by
 * one inside it, so no kernel reads outside the batch's arrays, and the
 * batch completes with POLYLLA_ERR_INVALID_MESH (every request in it:
 * device errors are per batch).  The same holds for polylla_generate on a
 * batch created without validation.
 */
typedef struct polylla_server polylla_server;
typedef struct {
    int64_t memory_budget;     /* device bytes the server may hold (> 0)        */
    int32_t n_slots;           /* copy-engine batches in flight, 1..16 (0: 3);
                                  the lane, when on, is one more slot          */
    int32_t max_batch_meshes;  /* meshes per batch, >= 1 (0: 4096)               */
    int32_t max_rotation;      /* as polylla_options (0: 4096)                   */
    int32_t max_batch_triangles; /* a batch stops growing past this many
                                    triangles (0: the slot's capacity); a single
                                    larger request still runs, alone          */
    int32_t lane_triangles;    /* largest request of the low-latency lane
                                  (0: 65,536; negative: no lane)              */
} polylla_server_options;
typedef struct {
    int32_t n_vertices, n_triangles, n_halfedges;
    polylla_host_mesh mesh;      /* inputs (host)                                  */
    polylla_host_result result;  /* outputs (host); n_polygons/n_frontier set at completion */
} polylla_request;
typedef struct {
    int32_t status;              /* POLYLLA_OK or the request's error              */
    int32_t n_polygons, n_frontier;
    int32_t batch_meshes;        /* meshes in the batch the request ran in         */
    double t_submit, t_admit, t_done; /* seconds on the server's steady clock      */
} polylla_request_info;
typedef struct {
    int32_t n_slots;             /* slots, the lane included                       */
    int32_t slot_triangles;      /* capacity of one copy-engine slot               */
    int64_t device_bytes;        /* device memory held                             */
    int64_t batches, requests_done;
    double busy_seconds;         /* time with at least one batch in flight         */
    double mean_in_ms;           /* per batch, on its stream: copies in,           */
    double mean_run_ms;          /*   kernels and metadata readback,               */
    double mean_out_ms;          /*   from metadata landed to results out          */
    double max_batch_ms;         /* the slowest batch (in + run + out on its stream) */
    int64_t max_batch_triangles; /*   its triangles                                */
    int32_t max_batch_requests;  /*   and requests                                 */
    int64_t launches;            /* kernels launched (18 per batch, 19 per lane batch) */
    int64_t lane_batches;        /* batches the lane ran                            */
    int32_t lane_triangles;      /* the lane's request limit (0: no lane)           */
    int32_t lane_slot_triangles; /* capacity of the lane slot (0: no lane)          */
} polylla_server_stats;

/* The slots a server with these options would allocate (host arithmetic
 * only: no CUDA call, usable without a GPU).  device_bytes is the server's
 * own bound on what the slots hold (at most memory_budget); a slot holds at
 * most 500 M triangles, so that its half-edge indices fit int32.  Errors:
 * INVALID_ARGUMENT (NULL, a negative option, more than 16 copy-engine
 * slots, or a budget too small for one triangle per slot). */
typedef struct {
    int32_t n_slots;             /* slots, the lane included                       */
    int32_t slot_triangles;      /* capacity of one copy-engine slot               */
    int32_t lane_triangles;      /* the lane's request limit (0: no lane)           */
    int32_t lane_slot_triangles; /* capacity of the lane slot (0: no lane)          */
    int64_t device_bytes;
} polylla_server_plan;
int polylla_server_plan_slots(const polylla_server_options *opt, polylla_server_plan *out);

/* Create a server on the current device (allocates all slots; starts the
 * scheduler thread).  Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
int polylla_server_create(polylla_server **out, const polylla_server_options *opt);
/* Queue a request (the struct is copied; the arrays are not); *ticket
 * identifies it.  Never blocks on the GPU. */
int polylla_server_submit(polylla_server *srv, const polylla_request *req, int64_t *ticket);
/* Block until the ticket's request completes; fill *info (may be NULL) and
 * forget the ticket.  Returns the request's status. */
int polylla_server_wait(polylla_server *srv, int64_t ticket, polylla_request_info *info);
/* Open-loop replay: submit reqs[k] at arrival_s[k] seconds (ascending)
 * after the call starts, from a native thread, wait for all, and write each
 * request's latency (completion minus its scheduled arrival) to
 * latency_s[k] and its info to infos[k] (may be NULL).  Returns the first
 * failing status, or POLYLLA_OK. */
int polylla_server_replay(polylla_server *srv, int32_t n, const polylla_request *reqs,
                          const double *arrival_s, double *latency_s, polylla_request_info *infos);
int polylla_server_get_stats(polylla_server *srv, polylla_server_stats *out);

/* One completed batch, for tracing where a request's time goes.  Host times
 * are seconds on the server's clock (the one polylla_request_info uses);
 * stream times are CUDA-event milliseconds on the slot's stream;
 * t_stream_start and t_meta_landed are stream events placed on the
 * server's clock through one reference event recorded at create (within a
 * few microseconds). */
typedef struct polylla_batch_record {
    double t_form;         /* scheduler starts forming the batch             */
    double t_enqueued;     /* copies in, kernels and metadata copy enqueued  */
    double t_meta_seen;    /* scheduler saw the metadata land                */
    double t_out_enqueued; /* result copies enqueued                         */
    double t_done;         /* scheduler saw the results land                 */
    float in_ms;           /* stream: copies in                              */
    float run_ms;          /* stream: kernels and metadata copy              */
    float idle_ms;         /* stream: metadata landed -> result copies start */
    float out_ms;          /* stream: result copies                          */
    int64_t n_triangles;
    int32_t n_requests;
    int32_t slot;
    int32_t lane;          /* 1: ran in the low-latency lane (kernel copies) */
    double t_stream_start; /* the slot's stream began the batch          */
    double t_meta_landed;  /* the stream finished kernels and metadata   */
} polylla_batch_record;

/* Copy the most recent min(capacity, kept) completed batches, oldest first,
 * to records (host array of capacity entries; may be NULL when capacity is
 * 0); *n_out receives how many were written and *n_total (may be NULL) how
 * many batches completed since create.  The server keeps the last 65,536.
 * Errors: INVALID_ARGUMENT (NULL srv or n_out, negative capacity). */
int polylla_server_get_batch_log(polylla_server *srv, polylla_batch_record *records, int32_t capacity,
                                 int32_t *n_out, int64_t *n_total);
/* Finish every queued request, stop the scheduler, free everything. */
void polylla_server_destroy(polylla_server *srv);

/*
 * polylla_generate_noalloc -- the whole method, allocating nothing.
 *
 * (No counterpart in the paper: this is a deployment convenience.)  For
 * callers that cannot call cudaMalloc: a serving loop that must not
 * allocate once it runs (an allocation can block on, or fail against,
 * memory other work holds), or a process whose device memory belongs to
 * another allocator that a stray cudaMalloc would fragment or bypass.  It
 * runs the same kernels as polylla_generate, but their scratch (labels, tip
 * lists, output tile words, counters) lives in one static device array of
 * fixed size that every GPU loading the library holds until the process
 * exits (about 1.7 MB), so no context, no cudaMalloc and no cudaFree.
 *
 *   mesh    device arrays as for polylla_create; must satisfy the layout
 *           polylla_create checks (no check is made here);
 *           next/prev of [0, 3T) are rewritten as by polylla_generate.
 *   seeds, offsets, he_list, v_list
 *           caller-owned device outputs with capacities T, T+1, 3T, 3T.
 *   status3 caller-owned device int32[3]: receives P, N_F and the device
 *           error bits of this call (0 = success; 1 a rotation or walk hit
 *           its cap, 2 a capacity was exceeded, 4 a wait gave up).
 *   stream  everything is enqueued on it; the call does not synchronize.
 * Returns POLYLLA_ERR_TOO_LARGE (nothing launched) when T exceeds
 * POLYLLA_NOALLOC_MAX_TRIANGLES or V exceeds it by more than 2,
 * POLYLLA_ERR_INVALID_ARGUMENT for NULL or misaligned pointers,
 * POLYLLA_ERR_CUDA (nothing launched, the error left pending for the caller)
 * when a CUDA error of earlier work is already pending on the calling
 * thread, otherwise POLYLLA_OK or POLYLLA_ERR_CUDA.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory limits; make
 * that first call before any stream capture begins.
 * Every call shares the one array and it keeps the last call's contents:
 * calls that overlap on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.
 */
#define POLYLLA_NOALLOC_MAX_TRIANGLES 131072
int polylla_generate_noalloc(const polylla_mesh *mesh, int32_t *seeds, int32_t *offsets,
                             int32_t *he_list, int32_t *v_list, int32_t *status3,
                             polylla_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* POLYLLA_H */
