// The persistent window kernel of the batched clouds (window.cuh): one
// cooperative launch per window.  Compiled as relocatable device code with
// the namespace renamed (-Dfla=fla_w); its host entry points are C symbols
// with hidden visibility that batch.cu calls with plain pointers.
#include <string.h>

#include "window.cuh"

namespace fla {
namespace {

constexpr int kWinThreads = 256;

struct WindowArgs {
    BatchDev b;
    WindowBlob bin;
    WindowBlob nw[kBatchGroups];
    int64_t n_dim[2];
    uint32_t* bin_start;
    int64_t n_bins;
    double dt;
    int window;
    int stall;
    DevStatus* st;
};

__device__ __forceinline__ int group_dim(int g) { return 2 + g / 2; }
__device__ __forceinline__ int group_kernel(int g) { return g % 2; }

// Phases in order, each followed by a grid barrier (the binning takes its
// own between its passes).  After a wait gives up every CTA skips the rest.
__global__ void __launch_bounds__(kWinThreads, 1) k_batch_window(const __grid_constant__ WindowArgs w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_sum[kWinThreads / 32];
    unsigned int gen = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;

    // carrier arguments at the window start; bin starts cleared for the counts
    window_carrier_args(w.b, w.dt);
    for (int64_t c = tid; c < w.n_bins; c += stride) w.bin_start[c] = 0u;
    bool ok = window_barrier(w.bin, ++gen, !(w.stall && blockIdx.x == 0));

    if (ok) window_carrier_sample(w.b);
    ok = ok && window_barrier(w.bin, ++gen, true);

    int n = 0;
    if (ok) n = window_advance(w.b, 2, w.n_dim[0], w.window, w.dt, w.st) +
                window_advance(w.b, 3, w.n_dim[1], w.window, w.dt, w.st);
    {
        const int s = __reduce_add_sync(0xffffffffu, n);
        if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
#pragma unroll
            for (int q = 0; q < kWinThreads / 32; ++q) t += s_sum[q];
            if (t) atomicAdd(&w.st->droplet_steps, (unsigned long long)t);
        }
    }
    ok = ok && window_barrier(w.bin, ++gen, true);

    if (ok && w.b.n_total > 0) {
        ok = window_binning(w.bin, w.b, gen, smem);
        ok = ok && window_barrier(w.bin, ++gen, true);
    }

    if (ok)
        for (int g = 0; g < kBatchGroups; ++g)
            if (w.b.group_first[g + 1] > w.b.group_first[g]) window_records(w.b, g, w.st);
    ok = ok && window_barrier(w.bin, ++gen, true);

    if (ok)
        for (int g = 0; g < kBatchGroups; ++g)
            if (w.b.n_tiles[g] > 0) window_gather_cand(w.nw[g], group_dim(g));
    ok = ok && window_barrier(w.bin, ++gen, true);

    if (ok)
        for (int g = 0; g < kBatchGroups; ++g)
            if (w.b.n_tiles[g] > 0 && (int)blockIdx.x == g % (int)gridDim.x) window_gather_plan(w.nw[g], group_dim(g));
    ok = ok && window_barrier(w.bin, ++gen, true);

    if (ok)
        for (int g = 0; g < kBatchGroups; ++g)
            if (w.b.n_tiles[g] > 0) window_gather_items(w.nw[g], group_dim(g), group_kernel(g), smem);
    ok = ok && window_barrier(w.bin, ++gen, true);

    if (ok)
        for (int g = 0; g < kBatchGroups; ++g)
            if (w.b.n_tiles[g] > 0) window_gather_combine(w.nw[g], group_dim(g));
    ok = ok && window_barrier(w.bin, ++gen, true);

    // the next window's start step (every CTA has read this one's)
    if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
        w.b.step[0] += w.window;
        w.b.step[1] = 1;   // this window's binning orders the next launched advance
    }
}

size_t window_smem()
{
    const size_t a = window_binning_smem(), b = window_items_smem();
    return a > b ? a : b;
}

}  // namespace
}  // namespace fla

// ------------------------------------------------------------------ host
// batch.cu passes its fla::BatchDev and fla::BinWork, which have the layout of
// this file's fla_w copies (the same header), as opaque pointers.

// Sets the kernel's shared-memory limit (once, before any capture) and
// returns the CTAs that fit at once on the device (0 on error).
extern "C" __attribute__((visibility("hidden"))) int fla_window_prepare(void)
{
    static int ctas = -1;
    if (ctas < 0) {
        int dev = 0, sms = 0, occ = 0;
        const size_t smem = fla::window_smem();
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaFuncSetAttribute(fla::k_batch_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fla::k_batch_window, fla::kWinThreads, smem) !=
                cudaSuccess)
            return 0;
        ctas = occ * sms;
    }
    return ctas;
}

// One window of every cloud: a memset of the barrier words, then the
// cooperative kernel.  Returns a cudaError_t value.
extern "C" __attribute__((visibility("hidden"))) int fla_window_issue(const void* batch_dev, const void* bin_work,
                                                                    uint32_t* bin_start, void* status, double dt,
                                                                    int window, int64_t n2, int64_t n3, int stall,
                                                                    uint32_t chunk, void* stream)
{
    const int ctas = fla_window_prepare();
    if (ctas < 1) return (int)cudaErrorInvalidConfiguration;
    fla::WindowArgs w;
    memset(&w, 0, sizeof(w));
    memcpy(&w.b, batch_dev, sizeof(w.b));
    fla::BinWork bw;
    memcpy(&bw, bin_work, sizeof(bw));
    fla::DevStatus* st = static_cast<fla::DevStatus*>(status);
    void* clear = nullptr;
    size_t clear_bytes = 0;
    fla::window_bin_blob(&w.bin, w.b, bw, bin_start, st, &clear, &clear_bytes);
    for (int g = 0; g < fla::kBatchGroups; ++g) fla::window_gather_blob(&w.nw[g], w.b, g, st, chunk);
    w.n_dim[0] = n2;
    w.n_dim[1] = n3;
    w.bin_start = bin_start;
    w.n_bins = w.b.cells_total + 1;
    w.dt = dt;
    w.window = window;
    w.stall = stall;
    w.st = st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(clear, 0, clear_bytes, s);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(fla::kWinThreads);
    cfg.dynamicSmemBytes = fla::window_smem();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, fla::k_batch_window, w);
}
