// Serving runtime (no counterpart in the paper): a request loop with
// continuous batching over the batched generate.
//
// One scheduler thread owns every CUDA call.  Requests wait in a FIFO queue
// in host memory; whenever a slot is free the scheduler takes, in arrival
// order, as many waiting requests as fit the slot's capacity (meshes,
// triangles, vertices, half-edges), copies their coords, origin and twin
// into the slot's device arena (the method never reads next/prev), runs the
// batch (the method's stages, per-mesh metadata) and moves
// the per-mesh metadata to pinned host memory.  When that has landed it
// copies each request's CSR slices and interior next/prev back into the
// request's host buffers (border entries are the input's, copied on the
// host); when those land the requests complete.  Each slot has its own
// stream, so one slot's copies overlap another's kernels.
// Slots and arenas are allocated once, at create, within the memory budget:
// admission against device memory is admission into a slot.
//
// The copy engines run one direction's copies in issue order across all
// streams, so a small batch's copies wait behind a large batch's.  Unless
// disabled, slot 0 is therefore a low-latency lane, one more (small) slot
// beside the copy-engine slots: it takes only requests of at most
// lane_triangles triangles whose buffers are pinned, runs on the device's
// highest-priority stream, and moves their data with SM kernels through
// host-mapped memory (kernels_serve.cu), so no copy engine queue is ever in
// its path.  The copy-engine slots take every other request in arrival
// order, and a lane request that has waited longer than kStealSeconds.
// Offsets, metadata and control blocks of every batch move by kernel too.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "polylla_serve.cuh"
#include "serve_policy.h"

using namespace polylla;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxCeSlots = 16;           // copy-engine slots
constexpr int kMaxSlots = kMaxCeSlots + 1; // and the lane
constexpr int64_t kLaneBatch = 16;        // the lane slot holds 16 requests of the lane's largest size
constexpr int kGroups = 32;          // completion groups of a copy-engine batch
constexpr size_t kLogKeep = 65536;  // completed batches kept for polylla_server_get_batch_log
constexpr int32_t kLaneDefault = 65536;  // lane_triangles when the option is 0
constexpr double kStealSeconds = 0.005;  // a lane request older than this may join any batch
// kernels per batch; the run is 8 (the method 7, metadata 1)
constexpr int32_t kLaunchesCE = 11;      // per batch: offsets, mesh table, the run, metadata out
constexpr int32_t kLaunchesLane = 12;    // per lane batch: gather, offsets, mesh table, the run, scatter

struct Req {
    polylla_request r{};
    int64_t ticket = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = POLYLLA_OK;
    int32_t P = 0, NF = 0, batch_meshes = 0;
    bool done = false;
    int8_t mapped = -1;  // -1 not checked yet; 1: every buffer pinned (tab holds their device addresses)
    ServeTab tab{};
};

struct Slot {
    polylla_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_meta = nullptr, ev_out = nullptr;
    // timing of the batch in flight: start, inputs in, metadata out, results out
    cudaEvent_t ev_t0 = nullptr, ev_in = nullptr, ev_tm = nullptr, ev_o0 = nullptr, ev_to = nullptr;
    polylla_batch_record rec{};  // host times of the batch in flight
    double *coords = nullptr;  // device arena: concatenated local arrays
    int32_t *origin = nullptr, *twin = nullptr, *next = nullptr, *prev = nullptr;
    int32_t *h_off = nullptr;  // pinned [4 (n_cap + 1)]: v, t, h, b prefix sums
    int32_t *h_meta = nullptr; // pinned [4 n_cap]
    DevCtrl *h_ctrl = nullptr; // pinned
    ServeTab *h_tab = nullptr; // pinned [n_cap]: the lane batch's request buffers
    // device addresses of the pinned arrays above
    int32_t *d_off = nullptr, *d_meta = nullptr;
    DevCtrl *d_ctrl = nullptr;
    ServeTab *d_tab = nullptr;
    // copy-engine slots: one event after the result copies of each group of
    // consecutive requests (one request per group up to kGroups requests),
    // so a request completes when its own results have landed instead of
    // when the whole batch's have
    cudaEvent_t ev_grp[kGroups] = {};
    int32_t grp_end[kGroups] = {};  // group g: requests [grp_end[g - 1], grp_end[g])
    int32_t n_grp = 0, grp_done = 0;
    int32_t n_done = 0;             // requests [0, n_done) of the batch completed
    bool lane = false;         // the low-latency lane (slot 0 when enabled)
    int32_t n_cap = 0, V_cap = 0, T_cap = 0, H_cap = 0;
    std::vector<Req *> reqs;
    int state = 0;             // 0 free, 1 batch running, 2 copying results out
};

// Device bytes of one slot of triangle capacity T (arena, union, scratch,
// metadata), following the allocations of serve_reserve and the arena.
int64_t slot_bytes(int64_t n, int64_t V, int64_t T, int64_t H) {
    const int64_t arena = 16 * V + 16 * H;
    const int64_t uni = 16 * H + 20 * (n + 1) + 4 * seg_count(T);
    const int64_t meta = 16 * n + 4 * (T + n + 1);
    const int64_t Tpad = (T + 15) / 16 * 16;
    const int64_t work = 2 * Tpad + 8 * V + 16 * ((T + OUT_TILE_MIN - 1) / OUT_TILE_MIN) + 16 * ((T + OUT_TILE_MIN - 1) / OUT_TILE_MIN / 1024 + 1) + 8 * out_rec_count(T) + 8 * out_warp_count(T) +
                         4 * T + 4 * (T + 1) + 24 * T + 256;
    const int64_t lepp = 16 * ((T + 1023) / 1024 + 1) + 8;  // path-scan totals of the Lepp primitive
    return arena + uni + meta + work + lepp + 64 * 256;      // + small allocations and their rounding
}

}  // namespace

struct polylla_server {
    int device = 0;
    int32_t max_batch = 4096;
    int32_t max_rotation = 0;
    int64_t max_batch_tri = 0;  // 0: slot capacity
    int32_t lane_tri = 0;       // 0: no lane; else the lane is slots[0]
    int n_slots = 0;
    Slot slots[kMaxSlots];
    int64_t device_bytes = 0;
    Clock::time_point t0;
    cudaEvent_t ev_ref = nullptr;  // recorded at create; puts stream events on the server's clock
    double t_ref = 0;

    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<int64_t, Req *> reqs;
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread sched;

    int64_t batches = 0, done_count = 0, timed_batches = 0;
    double busy = 0.0;
    double t_in = 0, t_run = 0, t_out = 0;  // summed ms: copies in, kernels + metadata, results out
    double slowest_ms = 0;                  // the slowest batch on its stream, and its size
    int64_t slowest_tri = 0;
    int32_t slowest_n = 0;
    std::vector<polylla_batch_record> log;  // ring of the last kLogKeep batches
    int64_t log_total = 0;
    int64_t launches = 0, lane_batches = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void loop();
    bool launch(Slot &s);
    void copy_out(Slot &s);
    void finish(Slot &s, int status);
    void complete(Req *q, int status);
    bool lane_ok(Req *q);
};

// Whether every buffer the device touches for q is pinned host memory, and
// their device addresses (checked once per request).
bool polylla_server::lane_ok(Req *q) {
    if (q->mapped < 0) {
        const void *p[9] = {q->r.mesh.coords,   q->r.mesh.origin,  q->r.mesh.twin,
                            q->r.result.seeds,  q->r.result.offsets, q->r.result.he_list,
                            q->r.result.v_list, q->r.result.next,  q->r.result.prev};
        void *d[9] = {};
        bool ok = true;
        for (int k = 0; k < 9 && ok; k++) {
            cudaPointerAttributes a{};
            ok = cudaPointerGetAttributes(&a, p[k]) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                 a.devicePointer != nullptr;
            d[k] = ok ? a.devicePointer : nullptr;
        }
        cudaGetLastError();  // an unregistered pointer leaves no error behind
        if (ok) {
            q->tab.coords = static_cast<const double *>(d[0]);
            q->tab.origin = static_cast<const int32_t *>(d[1]);
            q->tab.twin = static_cast<const int32_t *>(d[2]);
            q->tab.seeds = static_cast<int32_t *>(d[3]);
            q->tab.offsets = static_cast<int32_t *>(d[4]);
            q->tab.he_list = static_cast<int32_t *>(d[5]);
            q->tab.v_list = static_cast<int32_t *>(d[6]);
            q->tab.next = static_cast<int32_t *>(d[7]);
            q->tab.prev = static_cast<int32_t *>(d[8]);
        }
        q->mapped = ok ? 1 : 0;
    }
    const Slot &l = slots[0];
    return q->mapped == 1 && q->r.n_triangles <= lane_tri && q->r.n_vertices <= l.V_cap &&
           q->r.n_halfedges <= l.H_cap;
}

void polylla_server::complete(Req *q, int status) {
    std::lock_guard<std::mutex> g(mu);
    q->status = status;
    q->t_done = now();
    q->done = true;
    done_count++;
    cv_done.notify_all();
}

void polylla_server::finish(Slot &s, int status) {
    for (size_t i = (size_t)s.n_done; i < s.reqs.size(); i++) complete(s.reqs[i], status);
    s.reqs.clear();
    s.n_done = s.n_grp = s.grp_done = 0;
    s.state = 0;
}

// Form a batch from the head of the queue and enqueue it on the slot.
// Returns true when a batch was launched.
bool polylla_server::launch(Slot &s) {
    std::vector<Req *> take;
    {
        std::lock_guard<std::mutex> g(mu);
        const policy::SlotView sv{s.V_cap, s.T_cap, s.H_cap, std::min(s.n_cap, max_batch), s.lane};
        auto view = [this](Req *q) {
            return policy::ReqView{q->r.n_vertices, q->r.n_triangles, q->r.n_halfedges, lane_tri > 0 && lane_ok(q),
                                   q->t_submit};
        };
        // larger than any slot (the copy-engine slots are identical and the
        // largest) and not a lane request: fails now
        auto fail = [this](Req *q) {
            q->status = POLYLLA_ERR_TOO_LARGE;
            q->t_admit = q->t_done = now();
            q->done = true;
            done_count++;
            cv_done.notify_all();
        };
        policy::form_batch(pending, sv, lane_tri > 0, now(), kStealSeconds, max_batch_tri, view, fail, take);
    }
    if (take.empty()) return false;
    const int32_t n = (int32_t)take.size();
    int32_t *vo = s.h_off, *to = vo + (n + 1), *ho = to + (n + 1), *bo = ho + (n + 1);
    vo[0] = to[0] = ho[0] = bo[0] = 0;
    for (int32_t i = 0; i < n; i++) {
        const polylla_request &r = take[i]->r;
        vo[i + 1] = vo[i] + r.n_vertices;
        to[i + 1] = to[i] + r.n_triangles;
        ho[i + 1] = ho[i] + r.n_halfedges;
        bo[i + 1] = ho[i + 1] - 3 * to[i + 1];
    }
    const double t = now();
    s.rec = polylla_batch_record{};
    s.rec.t_form = t;
    s.rec.n_requests = n;
    s.rec.n_triangles = to[n];
    s.reqs = take;
    s.n_done = s.n_grp = s.grp_done = 0;
    for (Req *q : take) {
        q->t_admit = t;
        q->batch_meshes = n;
    }
    // lane batches: blocks per request of the copy kernels, from the largest request
    int32_t bx = 1;
    cudaError_t e = cudaEventRecord(s.ev_t0, s.stream);
    if (s.lane) {
        int32_t h_max = 0;
        for (int32_t i = 0; i < n; i++) {
            const Req *q = take[i];
            s.h_tab[i] = q->tab;
            h_max = std::max(h_max, q->r.n_halfedges);
            // border next/prev are the input's (the method leaves them as they are)
            const size_t n_int = 3 * (size_t)q->r.n_triangles, n_b = (size_t)q->r.n_halfedges - n_int;
            memcpy(q->r.result.next + n_int, q->r.mesh.next + n_int, 4 * n_b);
            memcpy(q->r.result.prev + n_int, q->r.mesh.prev + n_int, 4 * n_b);
        }
        bx = std::max(1, std::min(64, h_max / 8192));
        if (e == cudaSuccess) {
            launch_serve_gather(s.d_tab, s.d_off, n, bx, s.coords, s.origin, s.twin, s.stream);
            e = cudaGetLastError();
        }
    } else {
        for (int32_t i = 0; i < n && e == cudaSuccess; i++) {
            const polylla_request &r = take[i]->r;
            const size_t Hb = 4 * (size_t)r.n_halfedges;
            e = cudaMemcpyAsync(s.coords + 2 * (size_t)vo[i], r.mesh.coords, 16 * (size_t)r.n_vertices,
                                cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(s.origin + ho[i], r.mesh.origin, Hb, cudaMemcpyHostToDevice, s.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(s.twin + ho[i], r.mesh.twin, Hb, cudaMemcpyHostToDevice, s.stream);
            // next/prev are not read by the method (their interior entries are
            // rewritten, border entries go back from the host input)
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(s.ev_in, s.stream);
    int rc = e == cudaSuccess ? serve_run(s.ctx, n, vo[n], to[n], ho[n], s.d_off, s.stream) : POLYLLA_ERR_CUDA;
    if (rc == POLYLLA_OK) {
        ServeOutputs o;
        serve_outputs(s.ctx, &o);
        if (s.lane) {
            // results straight into the requests' host buffers
            e = cudaEventRecord(s.ev_tm, s.stream);
            if (e == cudaSuccess) e = cudaEventRecord(s.ev_o0, s.stream);
            if (e == cudaSuccess) {
                launch_serve_scatter(s.d_tab, s.d_off, n, bx, o, s.next, s.prev, to[n], s.d_meta, s.d_ctrl,
                                     s.stream);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(s.ev_to, s.stream);
            if (e == cudaSuccess) e = cudaEventRecord(s.ev_out, s.stream);
        } else {
            launch_serve_meta_out(o, n, s.d_meta, s.d_ctrl, s.stream);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(s.ev_meta, s.stream);
            if (e == cudaSuccess) e = cudaEventRecord(s.ev_tm, s.stream);
        }
        if (e != cudaSuccess) rc = POLYLLA_ERR_CUDA;
    }
    if (rc != POLYLLA_OK) {
        cudaStreamSynchronize(s.stream);
        finish(s, rc);
        return true;
    }
    s.state = s.lane ? 2 : 1;
    s.rec.t_enqueued = now();
    if (s.lane) s.rec.t_meta_seen = s.rec.t_out_enqueued = s.rec.t_enqueued;
    s.rec.lane = s.lane ? 1 : 0;
    {
        std::lock_guard<std::mutex> g(mu);
        batches++;
        launches += s.lane ? kLaunchesLane : kLaunchesCE;
        lane_batches += s.lane ? 1 : 0;
    }
    return true;
}

// The batch's metadata has landed: copy every request's results out.
void polylla_server::copy_out(Slot &s) {
    const int status = serve_status(*s.h_ctrl);
    if (status != POLYLLA_OK) {
        finish(s, status);
        return;
    }
    ServeOutputs o;
    serve_outputs(s.ctx, &o);
    const int32_t n = (int32_t)s.reqs.size();
    const int32_t *ho = s.h_off + 2 * (n + 1);
    const int32_t G = std::min(n, kGroups);
    for (int32_t g = 0; g < G; g++) s.grp_end[g] = (int32_t)(((int64_t)(g + 1) * n) / G);
    int32_t g = 0;
    cudaError_t e = cudaEventRecord(s.ev_o0, s.stream);
    for (int32_t i = 0; i < n && e == cudaSuccess; i++) {
        Req *q = s.reqs[i];
        polylla_host_result &out = q->r.result;
        const int32_t P = s.h_meta[4 * i], NF = s.h_meta[4 * i + 1];
        const int32_t p0 = s.h_meta[4 * i + 2], c0 = s.h_meta[4 * i + 3];
        q->P = P;
        q->NF = NF;
        const size_t Hb = 4 * (size_t)q->r.n_halfedges;
        e = cudaMemcpyAsync(out.seeds, o.seeds + p0, 4 * (size_t)P, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out.offsets, o.local_offsets + p0 + i, 4 * (size_t)(P + 1), cudaMemcpyDeviceToHost,
                                s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.he_list, o.he_list + c0, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.v_list, o.v_list + c0, 4 * (size_t)NF, cudaMemcpyDeviceToHost, s.stream);
        const size_t HIb = 12 * (size_t)q->r.n_triangles;
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.next, s.next + ho[i], HIb, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.prev, s.prev + ho[i], HIb, cudaMemcpyDeviceToHost, s.stream);
        if (Hb > HIb) {
            const size_t n_int = 3 * (size_t)q->r.n_triangles;
            memcpy(out.next + n_int, q->r.mesh.next + n_int, Hb - HIb);
            memcpy(out.prev + n_int, q->r.mesh.prev + n_int, Hb - HIb);
        }
        if (e == cudaSuccess && i + 1 == s.grp_end[g]) e = cudaEventRecord(s.ev_grp[g++], s.stream);
    }
    s.n_grp = e == cudaSuccess ? G : 0;
    if (e == cudaSuccess) e = cudaEventRecord(s.ev_out, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev_to, s.stream);
    s.rec.t_out_enqueued = now();
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s.stream);
        finish(s, POLYLLA_ERR_CUDA);
        return;
    }
    s.state = 2;
}

void polylla_server::loop() {
    cudaSetDevice(device);
    double busy_since = -1.0;
    for (;;) {
        bool progressed = false;
        int in_flight = 0;
        for (int k = 0; k < n_slots; k++) {
            Slot &s = slots[k];
            if (s.state == 1) {
                const cudaError_t q = cudaEventQuery(s.ev_meta);
                if (q == cudaSuccess) {
                    s.rec.t_meta_seen = now();
                    copy_out(s);
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    finish(s, POLYLLA_ERR_CUDA);
                    progressed = true;
                }
            }
            if (s.state == 2 && !s.lane) {
                // requests whose own results have landed complete now
                while (s.grp_done < s.n_grp && cudaEventQuery(s.ev_grp[s.grp_done]) == cudaSuccess) {
                    const int32_t end = s.grp_end[s.grp_done++];
                    for (; s.n_done < end; s.n_done++) {
                        Req *r = s.reqs[(size_t)s.n_done];
                        r->r.result.n_polygons = r->P;
                        r->r.result.n_frontier = r->NF;
                        complete(r, POLYLLA_OK);
                    }
                    progressed = true;
                }
            }
            if (s.state == 2) {
                const cudaError_t q = cudaEventQuery(s.ev_out);
                if (q == cudaSuccess || q != cudaErrorNotReady) {
                    if (q == cudaSuccess) {
                        float a = 0, b = 0, c = 0, d = 0, i = 0;
                        if (cudaEventElapsedTime(&a, s.ev_t0, s.ev_in) == cudaSuccess &&
                            cudaEventElapsedTime(&b, s.ev_in, s.ev_tm) == cudaSuccess &&
                            cudaEventElapsedTime(&c, s.ev_tm, s.ev_to) == cudaSuccess &&
                            cudaEventElapsedTime(&i, s.ev_tm, s.ev_o0) == cudaSuccess &&
                            cudaEventElapsedTime(&d, s.ev_o0, s.ev_to) == cudaSuccess) {
                            const int64_t tri = s.rec.n_triangles;
                            s.rec.t_done = now();
                            s.rec.in_ms = a;
                            s.rec.run_ms = b;
                            s.rec.idle_ms = i;
                            s.rec.out_ms = d;
                            s.rec.slot = k;
                            float r0 = 0, r1 = 0;
                            if (ev_ref && cudaEventElapsedTime(&r0, ev_ref, s.ev_t0) == cudaSuccess &&
                                cudaEventElapsedTime(&r1, ev_ref, s.ev_tm) == cudaSuccess) {
                                s.rec.t_stream_start = t_ref + 1e-3 * r0;
                                s.rec.t_meta_landed = t_ref + 1e-3 * r1;
                            }
                            std::lock_guard<std::mutex> g(mu);
                            if (log.size() < kLogKeep) log.push_back(s.rec);
                            else log[(size_t)(log_total % (int64_t)kLogKeep)] = s.rec;
                            log_total++;
                            t_in += a;
                            t_run += b;
                            t_out += c;
                            timed_batches++;
                            if (a + b + c > slowest_ms) {
                                slowest_ms = a + b + c;
                                slowest_tri = tri;
                                slowest_n = (int32_t)s.reqs.size();
                            }
                        }
                    }
                    if (s.lane && q == cudaSuccess) {
                        // the scatter wrote the metadata and control block to pinned memory
                        const int st = serve_status(*s.h_ctrl);
                        for (size_t i = 0; i < s.reqs.size(); i++) {
                            Req *r = s.reqs[i];
                            r->P = s.h_meta[4 * i];
                            r->NF = s.h_meta[4 * i + 1];
                            r->r.result.n_polygons = r->P;
                            r->r.result.n_frontier = r->NF;
                            complete(r, st != POLYLLA_OK ? st : r->P < 0 ? POLYLLA_ERR_CAPACITY : POLYLLA_OK);
                        }
                        s.reqs.clear();
                        s.state = 0;
                    } else {
                        for (size_t i = (size_t)s.n_done; i < s.reqs.size(); i++) {
                            Req *r = s.reqs[i];
                            r->r.result.n_polygons = r->P;
                            r->r.result.n_frontier = r->NF;
                        }
                        finish(s, q == cudaSuccess ? POLYLLA_OK : POLYLLA_ERR_CUDA);
                    }
                    progressed = true;
                }
            }
        }
        for (int k = 0; k < n_slots; k++)
            if (slots[k].state == 0 && launch(slots[k])) progressed = true;
        for (int k = 0; k < n_slots; k++) in_flight += slots[k].state != 0;
        const double t = now();
        if (in_flight && busy_since < 0) busy_since = t;
        if (!in_flight && busy_since >= 0) {
            std::lock_guard<std::mutex> g(mu);
            busy += t - busy_since;
            busy_since = -1.0;
        }
        if (progressed) continue;
        std::unique_lock<std::mutex> g(mu);
        if (stop && pending.empty() && !in_flight) break;
        if (in_flight) {
            // batches on the GPU: poll their events again shortly
            g.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
            cv_submit.wait_for(g, std::chrono::milliseconds(5), [&] { return stop || !pending.empty(); });
        }
    }
    if (busy_since >= 0) {
        std::lock_guard<std::mutex> g(mu);
        busy += now() - busy_since;
    }
}

static void free_slot(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.ctx) polylla_destroy(s.ctx);
    if (s.coords) cudaFree(s.coords);
    if (s.origin) cudaFree(s.origin);
    if (s.twin) cudaFree(s.twin);
    if (s.next) cudaFree(s.next);
    if (s.prev) cudaFree(s.prev);
    if (s.h_off) cudaFreeHost(s.h_off);
    if (s.h_meta) cudaFreeHost(s.h_meta);
    if (s.h_ctrl) cudaFreeHost(s.h_ctrl);
    if (s.h_tab) cudaFreeHost(s.h_tab);
    if (s.ev_meta) cudaEventDestroy(s.ev_meta);
    for (cudaEvent_t ev : {s.ev_t0, s.ev_in, s.ev_tm, s.ev_o0, s.ev_to})
        if (ev) cudaEventDestroy(ev);
    if (s.ev_out) cudaEventDestroy(s.ev_out);
    for (cudaEvent_t ev : s.ev_grp)
        if (ev) cudaEventDestroy(ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// Slot capacities for a budget (host arithmetic only): the lane first,
// kLaneBatch requests of its largest size within budget / (n + 1), then n
// copy-engine slots splitting the rest; each capacity is the largest T
// whose slot, with V <= T + 2m and H <= 4T + 2m for m meshes (bounds for
// triangulated disks), fits its share.
struct SlotPlan {
    int n_ce = 0;
    int64_t meshes = 0, T_ce = 0, T_lane = 0, lane_tri = 0, bytes = 0;
};

static int plan_slots(const polylla_server_options *opt, SlotPlan *p) {
    if (!opt || opt->memory_budget <= 0 || opt->n_slots < 0 || opt->n_slots > kMaxCeSlots || opt->max_batch_meshes < 0 ||
        opt->max_rotation < 0 || opt->max_batch_triangles < 0)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    const int n_ce = opt->n_slots ? opt->n_slots : 3;
    const int64_t m = opt->max_batch_meshes ? opt->max_batch_meshes : 4096;
    const int64_t lane_req = opt->lane_triangles < 0 ? 0 : opt->lane_triangles ? opt->lane_triangles : kLaneDefault;
    auto fit = [m](int64_t bytes, int64_t t_max) {
        int64_t lo = 0, hi = t_max;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (slot_bytes(m, mid + 2 * m, mid, 4 * mid + 2 * m) <= bytes) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto bytes_of = [m](int64_t T) { return slot_bytes(m, T + 2 * m, T, 4 * T + 2 * m); };
    const int64_t T_lane = lane_req > 0 ? fit(opt->memory_budget / (n_ce + 1), kLaneBatch * lane_req) : 0;
    const int64_t lane_bytes = T_lane > 0 ? bytes_of(T_lane) : 0;
    const int64_t T_ce = fit((opt->memory_budget - lane_bytes) / n_ce, 500000000);
    if (T_ce < 1) return POLYLLA_ERR_INVALID_ARGUMENT;
    p->n_ce = n_ce;
    p->meshes = m;
    p->T_ce = T_ce;
    p->T_lane = T_lane;
    p->lane_tri = T_lane > 0 ? std::min(lane_req, T_lane) : 0;
    p->bytes = lane_bytes + n_ce * bytes_of(T_ce);
    return POLYLLA_OK;
}

static int make_slot(polylla_server *srv, Slot &s, int32_t n, int32_t V, int32_t T, int32_t H, bool lane) {
    s.n_cap = n;
    s.V_cap = V;
    s.T_cap = T;
    s.H_cap = H;
    s.lane = lane;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    // the lane's kernels go first whenever SMs free up
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, lane ? greatest : least);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_meta, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_in);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_tm);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_o0);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_to);
    for (int g = 0; g < kGroups && e == cudaSuccess && !lane; g++)
        e = cudaEventCreateWithFlags(&s.ev_grp[g], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.coords, 16 * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.origin, 4 * (size_t)H);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.twin, 4 * (size_t)H);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.next, 4 * (size_t)H);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.prev, 4 * (size_t)H);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s.h_off, sizeof(int32_t) * 4 * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s.h_meta, sizeof(int32_t) * 4 * (size_t)n);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s.h_ctrl, sizeof(DevCtrl));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s.h_tab, sizeof(ServeTab) * (size_t)n);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s.d_off, s.h_off, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s.d_meta, s.h_meta, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s.d_ctrl, s.h_ctrl, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s.d_tab, s.h_tab, 0);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? POLYLLA_ERR_OUT_OF_MEMORY : POLYLLA_ERR_CUDA;
    const int rc = serve_reserve(&s.ctx, n, V, T, H, s.coords, s.origin, s.twin, s.next, s.prev, srv->max_rotation);
    if (rc) return rc;
    srv->device_bytes += 16 * (int64_t)V + 16 * (int64_t)H + (int64_t)serve_bytes(s.ctx);
    return POLYLLA_OK;
}

extern "C" {

int polylla_server_create(polylla_server **out, const polylla_server_options *opt) {
    if (!out) return POLYLLA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    SlotPlan plan;
    const int prc = plan_slots(opt, &plan);
    if (prc) return prc;
    polylla_server *srv = new (std::nothrow) polylla_server();
    if (!srv) return POLYLLA_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return POLYLLA_ERR_CUDA;
    }
    srv->max_batch = (int32_t)plan.meshes;
    srv->max_rotation = opt->max_rotation;
    srv->max_batch_tri = opt->max_batch_triangles;
    srv->lane_tri = (int32_t)plan.lane_tri;
    srv->n_slots = plan.n_ce + (srv->lane_tri > 0 ? 1 : 0);
    const int64_t n = plan.meshes, T_lane = plan.T_lane;
    const int32_t T = (int32_t)plan.T_ce, V = (int32_t)(plan.T_ce + 2 * n), H = (int32_t)(4 * plan.T_ce + 2 * n);
    int rc = POLYLLA_OK;
    for (int k = 0; k < srv->n_slots && !rc; k++) {
        if (k == 0 && srv->lane_tri > 0)
            rc = make_slot(srv, srv->slots[k], (int32_t)n, (int32_t)(T_lane + 2 * n), (int32_t)T_lane,
                           (int32_t)(4 * T_lane + 2 * n), true);
        else
            rc = make_slot(srv, srv->slots[k], (int32_t)n, V, T, H, false);
    }
    if (rc) {
        for (int k = 0; k < srv->n_slots; k++) free_slot(srv->slots[k]);
        delete srv;
        return rc;
    }
    srv->t0 = Clock::now();
    // reference event: its completion, seen by a synchronize, is t_ref on the server's clock
    if (cudaEventCreate(&srv->ev_ref) == cudaSuccess && cudaEventRecord(srv->ev_ref, srv->slots[0].stream) == cudaSuccess &&
        cudaEventSynchronize(srv->ev_ref) == cudaSuccess) {
        srv->t_ref = srv->now();
    } else {
        if (srv->ev_ref) cudaEventDestroy(srv->ev_ref);
        srv->ev_ref = nullptr;
        cudaGetLastError();
    }
    srv->sched = std::thread([srv] { srv->loop(); });
    *out = srv;
    return POLYLLA_OK;
}

int polylla_server_plan_slots(const polylla_server_options *opt, polylla_server_plan *out) {
    if (!out) return POLYLLA_ERR_INVALID_ARGUMENT;
    SlotPlan p;
    const int rc = plan_slots(opt, &p);
    if (rc) return rc;
    out->n_slots = p.n_ce + (p.lane_tri > 0 ? 1 : 0);
    out->slot_triangles = (int32_t)p.T_ce;
    out->lane_triangles = (int32_t)p.lane_tri;
    out->lane_slot_triangles = p.lane_tri > 0 ? (int32_t)p.T_lane : 0;
    out->device_bytes = p.bytes;
    return POLYLLA_OK;
}

int polylla_server_submit(polylla_server *srv, const polylla_request *req, int64_t *ticket) {
    if (!srv || !req || !ticket) return POLYLLA_ERR_INVALID_ARGUMENT;
    const polylla_request &r = *req;
    if (r.n_vertices < 3 || r.n_triangles < 1 || (int64_t)r.n_halfedges < 3 * (int64_t)r.n_triangles + 3)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    if (!r.mesh.coords || !r.mesh.origin || !r.mesh.twin || !r.mesh.next || !r.mesh.prev || !r.result.seeds ||
        !r.result.offsets || !r.result.he_list || !r.result.v_list || !r.result.next || !r.result.prev)
        return POLYLLA_ERR_INVALID_ARGUMENT;
    Req *q = new (std::nothrow) Req();
    if (!q) return POLYLLA_ERR_OUT_OF_MEMORY;
    q->r = r;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        q->ticket = srv->next_ticket++;
        q->t_submit = srv->now();
        srv->reqs[q->ticket] = q;
        srv->pending.push_back(q);
    }
    srv->cv_submit.notify_one();
    *ticket = q->ticket;
    return POLYLLA_OK;
}

int polylla_server_wait(polylla_server *srv, int64_t ticket, polylla_request_info *info) {
    if (!srv) return POLYLLA_ERR_INVALID_ARGUMENT;
    std::unique_lock<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return POLYLLA_ERR_INVALID_ARGUMENT;
    Req *q = it->second;
    srv->cv_done.wait(g, [&] { return q->done; });
    srv->reqs.erase(it);
    g.unlock();
    if (info) {
        info->status = q->status;
        info->n_polygons = q->P;
        info->n_frontier = q->NF;
        info->batch_meshes = q->batch_meshes;
        info->t_submit = q->t_submit;
        info->t_admit = q->t_admit;
        info->t_done = q->t_done;
    }
    const int st = q->status;
    delete q;
    return st;
}

int polylla_server_replay(polylla_server *srv, int32_t n, const polylla_request *reqs, const double *arrival_s,
                          double *latency_s, polylla_request_info *infos) {
    if (!srv || n < 0 || (n > 0 && (!reqs || !arrival_s || !latency_s))) return POLYLLA_ERR_INVALID_ARGUMENT;
    std::vector<int64_t> tickets((size_t)n);
    std::vector<double> sched((size_t)n);
    const double start = srv->now();
    int first_err = POLYLLA_OK;
    for (int32_t k = 0; k < n; k++) {
        const double at = start + arrival_s[k];
        sched[k] = at;
        // sleep to within 200 us of the arrival, then spin
        for (;;) {
            const double left = at - srv->now();
            if (left <= 0) break;
            if (left > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(left - 1.5e-4));
        }
        const int rc = polylla_server_submit(srv, &reqs[k], &tickets[k]);
        if (rc) {
            tickets[k] = 0;
            if (!first_err) first_err = rc;
            latency_s[k] = -1.0;
        }
    }
    for (int32_t k = 0; k < n; k++) {
        if (!tickets[k]) continue;
        polylla_request_info info;
        const int rc = polylla_server_wait(srv, tickets[k], &info);
        if (rc && !first_err) first_err = rc;
        latency_s[k] = info.t_done - sched[k];
        info.t_submit = sched[k];
        if (infos) infos[k] = info;
    }
    return first_err;
}

int polylla_server_get_stats(polylla_server *srv, polylla_server_stats *out) {
    if (!srv || !out) return POLYLLA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> g(srv->mu);
    out->n_slots = srv->n_slots;
    out->slot_triangles = srv->slots[srv->n_slots - 1].T_cap;  // a copy-engine slot
    out->device_bytes = srv->device_bytes;
    out->batches = srv->batches;
    out->requests_done = srv->done_count;
    out->busy_seconds = srv->busy;
    const double nb = srv->timed_batches > 0 ? (double)srv->timed_batches : 1.0;
    out->mean_in_ms = srv->t_in / nb;
    out->mean_run_ms = srv->t_run / nb;
    out->mean_out_ms = srv->t_out / nb;
    out->max_batch_ms = srv->slowest_ms;
    out->max_batch_triangles = srv->slowest_tri;
    out->max_batch_requests = srv->slowest_n;
    out->launches = srv->launches;
    out->lane_batches = srv->lane_batches;
    out->lane_triangles = srv->lane_tri;
    out->lane_slot_triangles = srv->lane_tri > 0 ? srv->slots[0].T_cap : 0;
    return POLYLLA_OK;
}

int polylla_server_get_batch_log(polylla_server *srv, polylla_batch_record *records, int32_t capacity,
                                 int32_t *n_out, int64_t *n_total) {
    if (!srv || !n_out || capacity < 0 || (capacity > 0 && !records)) return POLYLLA_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> g(srv->mu);
    const int64_t kept = (int64_t)srv->log.size();
    const int64_t m = std::min<int64_t>(kept, capacity);
    // oldest kept record: index 0 until the ring wraps, then the next slot to overwrite
    const int64_t first = kept < (int64_t)kLogKeep ? 0 : srv->log_total % (int64_t)kLogKeep;
    for (int64_t i = 0; i < m; i++) records[i] = srv->log[(size_t)((first + kept - m + i) % kept)];
    *n_out = (int32_t)m;
    if (n_total) *n_total = srv->log_total;
    return POLYLLA_OK;
}

void polylla_server_destroy(polylla_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_submit.notify_all();
    if (srv->sched.joinable()) srv->sched.join();
    for (int k = 0; k < srv->n_slots; k++) free_slot(srv->slots[k]);
    if (srv->ev_ref) cudaEventDestroy(srv->ev_ref);
    for (auto &kv : srv->reqs) delete kv.second;
    delete srv;
}

}  // extern "C"
