// fla_cell_bins_noalloc: the cell binning of fla_cell_bins for callers that
// cannot allocate device memory.
//
// Some host programs hand this library device pointers to buffers they
// already own but have no way to create new device buffers: a solver's C or
// Fortran coupling layer without a CUDA allocator of its own, or code running
// where cudaMalloc is not allowed because it synchronises the device or
// because another framework has reserved the memory.  For them this entry
// point takes its scratch space from a fixed array compiled into the library
// instead of a caller-provided workspace, and needs no fla_ctx (creating one
// allocates a small status block).
//
// The scratch array lives in device memory of every GPU that loads the
// library, until the process exits.  Its size caps the cloud at
// FLA_NOALLOC_MAX_DROPLETS droplets.
#include <mutex>

#include "fla_internal.cuh"

using namespace fla;

namespace {

constexpr int64_t kMaxDroplets = FLA_NOALLOC_MAX_DROPLETS;
// keys[2][max], vals[2][max], then the binning's scratch, sized for the
// largest cell count a mesh may have (2^31 - 1 cells: the most radix passes)
constexpr size_t kScratchBytes = bin_plan(kMaxDroplets, 2147483646LL).scratch_bytes;
static_assert(bin_plan(kMaxDroplets, 1).scratch_bytes <= kScratchBytes, "scratch sized for the smallest mesh too");
static_assert(bin_plan(kMaxDroplets, 262144).scratch_bytes <= kScratchBytes, "and for a mid-size one");
static_assert(bin_plan(kMaxDroplets, 1LL << 22).scratch_bytes <= kScratchBytes, "and for 2^22 cells");
constexpr int64_t kWords = 4 * kMaxDroplets + (int64_t)(kScratchBytes / 4);

static __device__ __align__(256) uint32_t g_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device;
// the host-side name g_scratch is not a device address).
int scratch_for_current_device(uint32_t** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FLA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FLA_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FLA_OK;
}

}  // namespace

extern "C" int fla_cell_bins_noalloc(const fla_cloud* cloud, const fla_mesh* mesh, uint32_t* keys_sorted_dev,
                                     uint32_t* perm_dev, uint32_t* bin_start_dev, fla_stream_t stream)
{
    // the same checks as fla_cell_bins, so both reject the same clouds
    const int valid = cloud_valid(cloud, mesh);
    if (valid != FLA_OK) return valid;
    if (cloud->n > kMaxDroplets) return FLA_ERR_WORKSPACE;   // beyond the fixed scratch array
    if (!bin_start_dev || (cloud->n > 0 && (!keys_sorted_dev || !perm_dev))) return FLA_ERR_ARG;
    const int64_t nc = mesh->dim == 2 ? (int64_t)mesh->n * mesh->n : (int64_t)mesh->n * mesh->n * mesh->n;
    cudaStream_t s = (cudaStream_t)stream;
    if (cloud->n == 0) return cudaMemsetAsync(bin_start_dev, 0, (size_t)(nc + 1) * 4, s) == cudaSuccess
                                  ? FLA_OK : FLA_ERR_CUDA;
    uint32_t* base = nullptr;
    const int st = scratch_for_current_device(&base);
    if (st != FLA_OK) return st;
    // Every scratch word the binning reads is written earlier in the same call.
    // With no context there is no status block: a barrier wait that runs out
    // ends the call without a report (its bin starts all zero).
    BinWork w{};
    w.keys[0] = base;
    w.keys[1] = base + kMaxDroplets;
    w.vals[0] = base + 2 * kMaxDroplets;
    w.vals[1] = base + 3 * kMaxDroplets;
    w.scratch = base + 4 * kMaxDroplets;
    if (launch_binning(*cloud, *mesh, w, bin_start_dev, nullptr, 0, s) != cudaSuccess) return FLA_ERR_CUDA;
    const int cur = bin_sorted_buffer(bin_plan(cloud->n, nc));
    if (cudaMemcpyAsync(keys_sorted_dev, w.keys[cur], (size_t)cloud->n * 4, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return FLA_ERR_CUDA;
    return cudaMemcpyAsync(perm_dev, w.vals[cur], (size_t)cloud->n * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess
               ? FLA_OK : FLA_ERR_CUDA;
}
