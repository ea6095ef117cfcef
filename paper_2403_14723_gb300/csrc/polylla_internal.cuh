// Internal declarations of the GB300 Polylla kernels (sm_103a).
//
// Layout of the work arrays in HBM (all sized at create, reused by every
// generate; nothing is allocated on the hot path):
//   le      [T]   uint8  local index of each triangle's longest half-edge
//   flags   [T]   uint8  bits 0-2 F1 (frontier after repair) of 3t+k,
//                        bits 3-5 F0 (frontier of the label phase),
//                        bit 6 the triangle's longest half-edge is a seed
//   tips    [V]   int32  F0 half-edge leaving each barrier tip
//   chords  [V]   int32  chord half-edge leaving each barrier tip
//   tile_status [n_tiles] u64  look-back words of the polygon scan
//   seeds [T], offsets [T+1], he_list [3T], v_list [3T]   CSR output
//   ctrl          DevCtrl       counters and the device error word
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace polylla {

// device error bits (ORed into DevCtrl::error)
enum : int32_t {
    DEV_ERR_NONTERMINATING = 1,
    DEV_ERR_CAPACITY = 2,
    DEV_ERR_TIMEOUT = 4,
};

struct DevCtrl {
    int32_t error;       // OR of DEV_ERR_* bits of this generate
    int32_t n_tips;      // barrier tips found by the relink
    int32_t ticket;      // next tile of the polygon kernel
    int32_t n_polygons;  // P, written by the last polygon tile
    int32_t n_frontier;  // N_F, written by the last polygon tile
    int32_t pad[3];
};

struct MeshView {
    int32_t V, T, H;
    const double2 *xy;
    const int32_t *origin;
    const int32_t *twin;
    int32_t *next;
    int32_t *prev;
};

struct Work {
    uint8_t *le;
    uint8_t *flags;
    int32_t *tips;
    int32_t *chords;
    int32_t tip_cap;
    unsigned long long *tile_status;
    int32_t n_tiles;
    int32_t *seeds;
    int32_t *offsets;
    int32_t *he_list;
    int32_t *v_list;
    DevCtrl *ctrl;
    int32_t max_rot;
    int32_t persistent_blocks;   // grid of the sparse (tip) kernels
};

// polygon kernel tiling: 256 threads x 8 consecutive half-edges
constexpr int POLY_THREADS = 256;
constexpr int POLY_ITEMS = 8;
constexpr int POLY_TILE = POLY_THREADS * POLY_ITEMS;

// ---- implicit triangle layout (paper Section 4.2) -------------------------
__device__ __forceinline__ int32_t tri_of(int32_t e) { return e / 3; }
__device__ __forceinline__ int32_t loc_of(int32_t e) { return e - 3 * (e / 3); }
__device__ __forceinline__ int32_t nx_of(int32_t e) {
    int32_t b = 3 * (e / 3);
    int32_t k = e - b;
    return b + (k == 2 ? 0 : k + 1);
}
__device__ __forceinline__ int32_t pv_of(int32_t e) {
    int32_t b = 3 * (e / 3);
    int32_t k = e - b;
    return b + (k == 0 ? 2 : k - 1);
}

// launchers (each enqueues one kernel on stream)
void launch_validate(const MeshView &m, int32_t *bad, cudaStream_t s);
void launch_longest_edge(const MeshView &m, const Work &w, cudaStream_t s);
void launch_label_relink(const MeshView &m, const Work &w, cudaStream_t s);
void launch_chords(const MeshView &m, const Work &w, cudaStream_t s);
void launch_chord_links(const MeshView &m, const Work &w, cudaStream_t s);
void launch_polygons(const MeshView &m, const Work &w, cudaStream_t s);

}  // namespace polylla
