// One persistent launch per window of the batched clouds.
//
// k_batch_window (window.cu) is a cooperative kernel (every CTA resident)
// that runs a whole window of every cloud as phases separated by grid
// barriers: carrier arguments, carrier nodes, the advance of both
// dimensions, the binning (keys, stable radix sort, bin starts; its own
// barriers), the records of each group, the gather plan, the work items and
// the combine of each group, and the step counter.  Each phase is the code of
// the corresponding kernel of the launch-per-phase window, compiled a second
// time from the same source file into relocatable device code with the
// namespace renamed (-Dfla=fla_w -DFLA_WINDOW_PHASES), where each file adds
// the device functions below: every phase keeps its own file's compilation
// (records without FMA contraction), and the launch-per-phase kernels keep
// theirs.  A barrier wait gives up after about a second (the binning's
// barrier: abort word, FLA_STATUS_WAIT_TIMEOUT), and every CTA then skips
// the remaining phases.
#pragma once

#include "batch.cuh"

// Opaque argument blocks that a phase file fills on the host and reads on the
// device (its own structures stay private to it).
struct WindowBlob {
    alignas(16) unsigned char b[256];
};

namespace fla {

// Phases, each a grid-stride loop of the calling CTA (256 threads) over its
// share of the work.
__device__ void window_carrier_args(const BatchDev& b, double dt);
__device__ void window_carrier_sample(const BatchDev& b);
// Droplet steps integrated by this thread.
__device__ int window_advance(const BatchDev& b, int dim, int64_t n_dim, int nsteps, double dt, DevStatus* st);
// Keys, sort and bin starts of all clouds (bin_start must be zero).  gen is
// the barrier generation, advanced by the barriers the binning takes; false
// when a wait gave up.  smem: the kernel's dynamic shared memory.
__device__ bool window_binning(const WindowBlob& bin, const BatchDev& b, unsigned int& gen, unsigned char* smem);
__device__ void window_records(const BatchDev& b, int group, DevStatus* st);
// Gather of group g: candidates per tile, item counts (one CTA per group),
// the work items (persistent, from the group's counter), the combine.
__device__ void window_gather_cand(const WindowBlob& nw, int dim);
__device__ void window_gather_plan(const WindowBlob& nw, int dim);
__device__ void window_gather_items(const WindowBlob& nw, int dim, int kernel, unsigned char* smem);
__device__ void window_gather_combine(const WindowBlob& nw, int dim);
// Grid barrier number gen on the binning's barrier words; false when a wait
// gave up (then or before).
__device__ bool window_barrier(const WindowBlob& bin, unsigned int gen, bool arrive);

// Host side of the phase files.
size_t window_bin_blob(WindowBlob* out, const BatchDev& b, const BinWork& w, uint32_t* bin_start, DevStatus* st,
                       void** clear, size_t* clear_bytes);
size_t window_gather_blob(WindowBlob* out, const BatchDev& b, int group, DevStatus* st, uint32_t chunk);
size_t window_binning_smem();
size_t window_items_smem();

}  // namespace fla
