// Internal interface between the serving runtime (polylla_server.cu) and
// the context code (polylla_api.cu): a batch context with fixed capacities
// whose meshes change on every run.
#pragma once

#include "../../include/polylla.h"
#include "polylla_internal.cuh"

namespace polylla {

// A batch context able to hold up to n_cap meshes of V_cap, T_cap, H_cap in
// total, over the caller's device arena (concatenated local arrays of those
// capacities).  No mesh is bound yet.
int serve_reserve(polylla_ctx **out, int32_t n_cap, int32_t V_cap, int32_t T_cap, int32_t H_cap,
                  const double *coords, const int32_t *origin, const int32_t *twin, int32_t *next, int32_t *prev,
                  int32_t max_rotation);

// Device bytes the context holds.
size_t serve_bytes(const polylla_ctx *c);

// Bind n meshes of V, T, H in total and enqueue the whole run on s: a
// kernel copy of the prefix sums off4 = {v[n+1], t[n+1], h[n+1], b[n+1]}
// (the device address of pinned host memory that must stay valid until the
// run completes), the method's stages and the per-mesh metadata.
int serve_run(polylla_ctx *c, int32_t n, int32_t V, int32_t T, int32_t H, const int32_t *off4, cudaStream_t s);

// Device outputs of the last run (valid once it completes, until the next).
struct ServeOutputs {
    const int32_t *seeds;          // batch order, mesh-local values
    const int32_t *local_offsets;  // mesh i: [first polygon + i, ... + P_i + 1)
    const int32_t *he_list;        // mesh-local values
    const int32_t *v_list;
    const int32_t *meta;           // [4 n]: P_i, N_F,i, first polygon, first CSR entry
    const DevCtrl *ctrl;
};
void serve_outputs(const polylla_ctx *c, ServeOutputs *o);

// Status a run's control block reports (POLYLLA_OK or a device error).
int serve_status(const DevCtrl &h);

// One request's host buffers, as device addresses of pinned host memory
// (what cudaPointerGetAttributes reports as the device pointer).
struct ServeTab {
    const double *coords;
    const int32_t *origin, *twin;
    int32_t *seeds, *offsets, *he_list, *v_list, *next, *prev;
};

// Copies moved by SM kernels through host-mapped pinned memory instead of
// the copy engines: copy-engine copies in one direction run in the order
// they were issued, whatever their stream, so a small copy issued behind a
// large one waits for it, while these kernels are scheduled like any other.
//   gather: request i's coords, origin and twin into the arena at its
//           offsets (off4 as for serve_run, device address of pinned host
//           memory); blocks_x blocks per request.
//   scatter: request i's CSR slices and interior next/prev from the run's
//           outputs into its host buffers; the metadata (P_i, N_F,i, first
//           polygon, first entry) goes to meta_host, with P_i = -1 where it
//           does not fit the request's capacities or the outputs, and the
//           control block to ctrl_host.
//   meta_out: the metadata and the control block only.
void launch_serve_gather(const ServeTab *tab, const int32_t *off4, int32_t n, int32_t blocks_x, double *coords,
                         int32_t *origin, int32_t *twin, cudaStream_t s);
void launch_serve_scatter(const ServeTab *tab, const int32_t *off4, int32_t n, int32_t blocks_x,
                          const ServeOutputs &o, const int32_t *next, const int32_t *prev, int32_t T_tot,
                          int32_t *meta_host, DevCtrl *ctrl_host, cudaStream_t s);
void launch_serve_meta_out(const ServeOutputs &o, int32_t n, int32_t *meta_host, DevCtrl *ctrl_host, cudaStream_t s);
void launch_serve_offsets(const int32_t *off4, int32_t n, int32_t *v_off, int32_t *t_off, int32_t *h_off,
                          int32_t *b_off, cudaStream_t s);

}  // namespace polylla
