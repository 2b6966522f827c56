// Launch description of the persistent backprojection kernel (backproject.cu).
#pragma once

#include <cuda_fp16.h>

#include "fbp_internal.h"

namespace fbp {

// Shared-memory ring: stages of `chunk` angles (of every slice of an item), 64
// window rows in flight, at least two stages.
__host__ __device__ constexpr int bp_stages(int chunk, int group)
{
    return chunk * group >= 32 ? 2 : 64 / (chunk * group);
}
constexpr int kBpMaxSlices = 64;  // slices per batched launch (tensor maps in the parameters)

// One work-list entry of a launch: a slice, or (group = 2) two slices of the
// same plan that share every index computation.
struct BpSlice {
    const double2 *trig64;  // (cos, sin) / tau per angle
    float *image;           // [n][n]
    float *image2;          // second slice of a group (group = 2), else unused
    int n;
    int A;
    int wp;       // detector window per tile and angle, in (mid, slope) pairs
    int tiles_x;  // tiles per image row
    float scale;  // pi / A
    int tiles;    // tiles of the slice (work items: tiles, or tiles / 2 for point pairs)
    double half_n;  // (n - 1) / 2
    double half_d;  // (n_det - 1) / 2
};

// Kernel parameters: one tensor map per slice (over that slice's filtered
// pairs [A][pitch]) and the work list, implicit in the slice order: item j
// is tile j - tile_end[s-1] of the slice s with tile_end[s-1] <= j < tile_end[s].
// The host orders slices by angle count, most first, so the costliest tiles
// are handed out first.
template <int MAXS>
struct BpLaunch {
    CUtensorMap maps[2 * MAXS];  // entry s, slice g of its group: maps[group * s + g]
    BpSlice slices[MAXS];
    int tile_end[MAXS];  // inclusive prefix sums of the slices' tile counts
    int n_slices;
    int n_items;  // = tile_end[n_slices - 1]
    int wp_max;   // largest wp over the slices (sizes the shared-memory rows)
    int *status;
    // Work distribution: NULL = CTA b takes items b, b + grid, ...; otherwise
    // two ints {next item, CTAs done}, zero before the launch and left at zero
    // by it, from which CTAs take items as they get room (one counter per
    // launch in flight).
    int *sched;
};

// Template choice: tile = (8 wx) x (32 wy) pixels, wx*wy consumer warps.
struct BpConfig {
    int wx;
    int wy;
    int chunk;        // angles per stage: 8, 16 or 32
    bool half_pairs;  // FP16-stored (mid, slope) pairs
    bool kahan;       // Kahan-compensated sum over angles
    int group;        // slices per work item: 1, or 2 (same plan)
    bool point_pairs; // work item = a tile and its point-symmetric partner (one slice)
};

// The kernel configuration of a plan's slices (api.cu).
BpConfig bp_config(const Plan &p);

cudaError_t launch_backproject(const BpLaunch<1> &P, const BpConfig &c, cudaStream_t s);
cudaError_t launch_backproject_batch(const BpLaunch<kBpMaxSlices> &P, const BpConfig &c,
                                     int grid_limit, cudaStream_t s);

}  // namespace fbp
