// Batched clouds: many FLA clouds of different sizes, meshes and carriers
// advanced and deposited together, a few launches per window for all of them.
//
// The clouds share one global cell space: cloud k's cells occupy
// [cell_off_k, cell_off_k + n_cells_k), so one key pass and one radix sort
// (with the bin starts) bin every droplet of every cloud, and each cloud's sorted
// records are contiguous.  Clouds are ordered by group (dim, kernel), so each
// group's records are contiguous too and live in a record array of the
// group's width.  Per-cloud parameters come from a device table.  The window
// start step is read from a device counter that the window's last kernel
// advances, so a captured graph of several windows replays without host work.
#pragma once

#include "fla_internal.cuh"

namespace fla {

constexpr int kBatchGroups = 4;   // (2D, ISO), (2D, ANISO), (3D, ISO), (3D, ANISO)
__host__ __device__ constexpr int batch_group(int dim, int kernel) { return (dim - 2) * 2 + kernel; }

struct BatchCloud {
    int dim, kernel, N, per_cell;
    int n_batches, plain, group, pad;
    int64_t n, drop_off, n_cells, cell_off, n_nodes, node_off;
    float* state;
    uint32_t* meta;
    const fla_batch* batches;
    float* nodes;
    float* s_mass;
    float* s_mom;
    float* dsum;
    double delta, h_min, h_max, p, window_dt;
    fla_carrier_desc car;
};

// One CTA tile of a cloud's mesh for the batched gather (origin in cells).
struct BatchTile {
    int cloud, x0, y0, z0;
};

// Device-side tables and run state (all in the caller's workspace).
struct BatchDev {
    const BatchCloud* clouds;     // n_clouds, group-ordered
    int n_clouds;
    int64_t n_total;              // droplets of all clouds
    int64_t cells_total;
    int64_t nodes_total;
    const int64_t* drop_pre;      // n_clouds + 1 droplet offsets
    const int64_t* node_pre;      // n_clouds + 1 node offsets
    int* step;                    // [0] first step of the next window; [1] 1 when perm and
                                  // bin_start hold the binning of the window before it
    unsigned int* ext_max;        // per cloud: max squared support radius (float bits)
    unsigned int* tile_counter;   // per group
    void* cargs;                  // per cloud carrier arguments of the current window
    const uint32_t* perm;         // sorted droplet order (global indices) of the current deposit
    const uint32_t* bin_start;    // cells_total + 1
    void* rec[kBatchGroups];      // records per group
    int group_first[kBatchGroups + 1];   // clouds [group_first[g], group_first[g+1]) form group g
    int64_t group_cells[kBatchGroups + 1];   // global cell ranges of the groups
    int64_t group_drops[kBatchGroups];       // droplets of each group's clouds
    const BatchTile* tiles[kBatchGroups];    // gather tiles per group, in the tuned order
    int n_tiles[kBatchGroups];
    uint32_t* tile_cand[kBatchGroups];       // per tile: candidates (gather plan)
    uint32_t* tile_items[kBatchGroups];      // per tile: first work item (n_tiles + 1)
    unsigned long long* cloud_cand;          // per cloud: candidates of its tiles (zero between plans)
    unsigned int* plan_done;                 // per group: plan CTAs finished
    void* item_temp[kBatchGroups];           // partial sums of each group's work items
};

// index k with pre[k] <= v < pre[k + 1] (pre ascending, n + 1 entries)
__device__ __forceinline__ int batch_find(const int64_t* __restrict__ pre, int n, int64_t v)
{
    int lo = 0, hi = n;   // invariant: pre[lo] <= v < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

size_t batch_carrier_args_bytes();
cudaError_t batch_prepare_gathers();
cudaError_t batch_prepare_advance();
cudaError_t launch_batch_carrier(const BatchDev& b, double dt, cudaStream_t s);
cudaError_t launch_batch_advance(const BatchDev& b, int dim, int64_t n_dim, int nsteps, double dt, bool reset,
                                 int threads, DevStatus* st, cudaStream_t s);
// Keys, sort and bin starts (cells_total + 1 words) of all clouds: one kernel.
cudaError_t launch_batch_binning(const BatchDev& b, const BinWork& w, uint32_t* bin_start, DevStatus* st,
                                 cudaStream_t s);
cudaError_t launch_batch_records(const BatchDev& b, int group, DevStatus* st, cudaStream_t s);
cudaError_t launch_batch_gather(const BatchDev& b, int group, int ctas, DevStatus* st, int num_sms, cudaStream_t s);
cudaError_t launch_batch_step(const BatchDev& b, int nsteps, cudaStream_t s);

}  // namespace fla
