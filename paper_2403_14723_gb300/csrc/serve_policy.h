// Admission policy of the serving loop (no counterpart in the paper): which
// waiting requests a free slot takes into its next batch.  Plain C++ with
// no CUDA, so that the policy is tested on the CPU exactly as the server
// runs it.
//
// The queue is scanned front to back.  With a low-latency lane on, the
// lane slot takes only lane requests, and the copy-engine slots leave lane
// requests to it until they have waited steal_s.  A request that fits no
// copy-engine slot fails at once, unless the lane can take it.  A batch
// stops growing at the first request that would overflow the slot (or the
// batch triangle cap), so requests keep their arrival order among those a
// slot may take.
#pragma once

#include <cstdint>
#include <deque>
#include <vector>

namespace polylla {
namespace policy {

struct ReqView {
    int64_t V, T, H;   // vertices, triangles, half-edges of the request
    bool small;        // a lane request (small enough, buffers pinned)
    double t_submit;   // seconds, server clock
};

struct SlotView {
    int64_t V_cap, T_cap, H_cap;
    int32_t n_cap;     // meshes per batch
    bool lane;         // the low-latency lane
};

enum class Decision { Take, Skip, Fail, Stop };

struct BatchSoFar {
    int64_t V = 0, T = 0, H = 0;
    int32_t n = 0;
};

// What a forming batch on slot s does with request r at time now.
inline Decision admit(const ReqView &r, const SlotView &s, bool lane_on, double now, double steal_s,
                      int64_t max_batch_tri, const BatchSoFar &b) {
    if (lane_on && s.lane != r.small && (s.lane || now - r.t_submit < steal_s))
        return Decision::Skip;  // the lane takes lane requests only; the others leave them to it for a while
    if (r.V > s.V_cap || r.T > s.T_cap || r.H > s.H_cap)
        return r.small ? Decision::Skip : Decision::Fail;  // a lane request may still fit the lane
    if (b.V + r.V > s.V_cap || b.T + r.T > s.T_cap || b.H + r.H > s.H_cap) return Decision::Stop;
    if (b.n > 0 && max_batch_tri > 0 && b.T + r.T > max_batch_tri) return Decision::Stop;
    return Decision::Take;
}

// Form one batch for slot s from the queue: taken requests move to take
// (in queue order), failed ones are erased and handed to on_fail, skipped
// ones stay.  view(q) gives a request's ReqView.
template <class Q, class View, class OnFail>
void form_batch(std::deque<Q> &pending, const SlotView &s, bool lane_on, double now, double steal_s,
                int64_t max_batch_tri, View view, OnFail on_fail, std::vector<Q> &take) {
    BatchSoFar b;
    for (auto it = pending.begin(); it != pending.end() && b.n < s.n_cap;) {
        const ReqView r = view(*it);
        switch (admit(r, s, lane_on, now, steal_s, max_batch_tri, b)) {
        case Decision::Take:
            b.V += r.V;
            b.T += r.T;
            b.H += r.H;
            b.n++;
            take.push_back(*it);
            it = pending.erase(it);
            break;
        case Decision::Skip:
            ++it;
            break;
        case Decision::Fail:
            on_fail(*it);
            it = pending.erase(it);
            break;
        case Decision::Stop:
            return;
        }
    }
}

}  // namespace policy
}  // namespace polylla
