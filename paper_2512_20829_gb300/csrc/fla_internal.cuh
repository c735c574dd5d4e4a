// Internal declarations shared by the translation units of libfla.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fla.h"

struct fla_ctx {
    int device;
    int num_sms;
    fla_device_status* status_dev;   // 64-byte block, zeroed at creation
    // profiling: launch/call counters (always) and CUDA-event phase timing (optional)
    int timing;
    double ms[FLA_PHASE_COUNT];
    long long launches[FLA_PHASE_COUNT];
    long long calls[FLA_PHASE_COUNT];
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    unsigned int stall;   // fla_test_stall bits, cleared when used
};

namespace fla {

constexpr int kMaxPlanes = 7;

// Programmatic dependent launch.  Kernels launched by launch_pdl are set up
// by the GPU while the previous grid in the stream runs, and their CTAs begin
// as soon as it completes, instead of after a full launch round trip.  Every
// kernel starts with pdl_entry(), which waits until the previous grid has
// completed and its writes are visible, so memory accesses keep plain stream
// order.  (No kernel signals its dependents early: CTAs launched ahead and
// left waiting slowed the grids they waited on.)  Outside a programmatic
// launch the wait returns at once.
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch with programmatic stream serialization (the kernel begins with pdl_entry()).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = s == nullptr ? 0 : 1;   // the legacy stream: a plain launch
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// vec4 of the storage type: float4 or a 32-byte pair of double2.
template <typename T> struct V4;
template <> struct V4<float> {
    float4 v;
};
template <> struct V4<double> {
    double2 a, b;
};

// Loads of a kernel's inputs (state, nodes, records, bin starts).  A kernel
// of one phase reads them through the non-coherent read-only path; the
// persistent window kernel (window.cuh), where an earlier phase of the same
// launch wrote them, reads them with plain loads, which a grid barrier's
// fences make coherent.
template <typename T>
__device__ __forceinline__ T ldro(const T* p)
{
#ifdef FLA_WINDOW_PHASES
    return *p;
#else
    return __ldg(p);
#endif
}

template <typename T>
__device__ __forceinline__ void load4(const T* base, int64_t idx4, T out[4]);
template <>
__device__ __forceinline__ void load4<float>(const float* base, int64_t idx4, float out[4])
{
    float4 v = ldro(reinterpret_cast<const float4*>(base) + idx4);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* base, int64_t idx4, double out[4])
{
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx4;
    double2 a = ldro(p), b = ldro(p + 1);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void store4(T* base, int64_t idx4, const T in[4]);
template <>
__device__ __forceinline__ void store4<float>(float* base, int64_t idx4, const float in[4])
{
    reinterpret_cast<float4*>(base)[idx4] = make_float4(in[0], in[1], in[2], in[3]);
}
template <>
__device__ __forceinline__ void store4<double>(double* base, int64_t idx4, const double in[4])
{
    double2* p = reinterpret_cast<double2*>(base) + 2 * idx4;
    p[0] = make_double2(in[0], in[1]);
    p[1] = make_double2(in[2], in[3]);
}

// Values per droplet (before padding) and planes of 4.
__host__ __device__ constexpr int state_values(int kind, int dim)
{
    return kind == FLA_CLOUD_FLA ? 2 * dim + 2 * dim * dim + 1 + dim : 2 * dim + 1 + dim;
}
__host__ __device__ constexpr int state_planes(int kind, int dim) { return (state_values(kind, dim) + 3) / 4; }
__host__ __device__ constexpr int acc_offset(int kind, int dim)
{
    return kind == FLA_CLOUD_FLA ? 2 * dim + 2 * dim * dim : 2 * dim;
}
__host__ __device__ constexpr int node_stride(int dim) { return dim == 2 ? 8 : 12; }
// Double-float (FLA_F32X2) node arrays end with this tail: the largest |value|
// of each component (float bits), from which the split into a + b is formed.
constexpr size_t kNodesX2TailBytes = 256;

// Record of one binned droplet for the kernel-regression gather, in sorted order.
// Single precision (the weight is 2^(c r^2 + lih), resp. 2^(-q log2(e)/2 + lpref)):
//   2D iso   (8 values):  x, y, c, lih | a_m, a_x, a_y, r2max
//   3D iso   (12 values): x, y, z, r2max | c, lih, 0, 0 | a_m, a_x, a_y, a_z
//   2D aniso (12 values): x, y, lpref, ext2 | P00, P01, P11, 0 | a_m, a_x, a_y, 0
//   3D aniso (16 values): x, y, z, lpref | P00, P01, P02, P11 | P12, P22, ext2, 0 | a_m, a_x, a_y, a_z
// with c = -log2(e)/(2 h^2), lih = log2(1/h), lpref = log2(det(Sigma)^-1/2),
// r2max = 9 h^2 and ext2 = 9 tr(Sigma) (squared support radius bounds).
// Double precision keeps the same slots with c = -1/(2 h^2), 1/h in place of lih
// and det(Sigma)^-1/2 in place of lpref (the weight is (1/h) e^(c r^2)).
__host__ __device__ constexpr int record_values(int dim, int kernel)
{
    return (dim == 2 && kernel == FLA_KERNEL_ISO) ? 8 : ((dim == 3 && kernel == FLA_KERNEL_ANISO) ? 16 : 12);
}

// Device status block layout (matches fla_device_status).
// Cell key of droplet i (plane 0 holds the position): floor(x N) per axis in
// the cloud's precision, clamped to N - 1, x fastest; false when the droplet
// is not active or lies outside [0,1]^D.
template <typename T, int D>
__device__ __forceinline__ bool cell_key_of(const T* __restrict__ state, const uint32_t* __restrict__ meta, int64_t i,
                                            int N, uint32_t* key_out)
{
    T x[4];
    load4<T>(state, i, x);
    bool ok = (meta[i] & FLA_META_ACTIVE) != 0;
    uint32_t key = 0, mul = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        ok &= (x[a] >= T(0) && x[a] <= T(1));
        const T s = x[a] * T(N);            // formed in the cloud's precision
        int c = ok ? (int)floor(s) : 0;
        c = c > N - 1 ? N - 1 : c;
        key += (uint32_t)c * mul;
        mul *= (uint32_t)N;
    }
    *key_out = key;
    return ok;
}

struct DevStatus {
    unsigned long long nonfinite, deposited, droplet_steps, pairs, fold_steps;
    unsigned int flags, pad;
};
static_assert(sizeof(DevStatus) == sizeof(fla_device_status), "status block mirrors fla_device_status");
constexpr unsigned int kFlagMlpTimeout = FLA_STATUS_MLP_TIMEOUT;
constexpr unsigned int kFlagWaitTimeout = FLA_STATUS_WAIT_TIMEOUT;

// Waits on words that other CTAs of the same grid publish give up after
// kWaitLimitNs of the GPU's global timer (about a second), or at once when
// another CTA has given up (its abort word is set).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Fold-guard array: planes of 4 doubles holding J[d*d] then W[d*d] (2D 8
// values, 3D 18), then the hand-over list of the advance (n u32) and its
// counter, each on a 16-byte boundary.
__host__ __device__ constexpr int fold_planes(int dim) { return (2 * dim * dim + 3) / 4; }
struct FoldLayout {
    size_t list, count, total;
};
inline FoldLayout fold_layout(int dim, int64_t n)
{
    FoldLayout L{};
    L.list = (size_t)fold_planes(dim) * (size_t)n * 4 * sizeof(double);
    L.count = L.list + (((size_t)n * 4 + 15) & ~(size_t)15);
    L.total = L.count + 16;
    return L;
}

// Cell binning (binning.cu): one cooperative kernel per call over tiles of
// 2,048 keys; radix digits of up to 11 bits (2,048 values) for clouds of up to
// 2^21 droplets, 8 bits beyond.  Scratch besides the key and value buffers:
// per-(pass, tile, digit) histograms, per-(block of 32 tiles, digit) sums,
// per-(pass, digit) totals and per-chunk cell counts of the bin-start scan (all written by the kernel before it reads
// them), then the barrier words, cleared before each call.  Where bin_start
// directly follows the scratch (the workspace layouts place it there), one
// memset clears the barrier words and bin_start.
constexpr int64_t kSortTile = 2048;
constexpr int kSortMaxDigitBits = 11;
constexpr int64_t kBinMaxChunks = 1024;         // chunks of cells of the bin-start scan
constexpr size_t kBinControlBytes = 256;        // barrier counter, abort, done
struct BinPlan {
    int64_t n, n_cells;                         // droplets; cells (the key of droplets without a cell)
    int bits, passes, width, tiles;
    int64_t chunks, chunk_cells;
    int64_t blocks;                             // blocks of 32 tiles of the tile-prefix scans
    size_t off_hist, off_block, off_totals, off_chunk, off_clear, scratch_bytes;   // byte offsets; size
};
__host__ __device__ constexpr int sort_bits_of(uint64_t max_key)
{
    int b = 0;
    while (b < 32 && (max_key >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}
__host__ __device__ constexpr size_t bin_up256(size_t x) { return (x + 255) & ~(size_t)255; }
__host__ __device__ constexpr BinPlan bin_plan(int64_t n, int64_t n_cells)
{
    BinPlan p{};
    p.n = n;
    p.n_cells = n_cells;
    p.bits = sort_bits_of((uint64_t)n_cells);
    const int maxw = n <= (int64_t(1) << 21) ? kSortMaxDigitBits : 8;
    p.passes = (p.bits + maxw - 1) / maxw;
    p.width = (p.bits + p.passes - 1) / p.passes;
    const int64_t nn = n > 0 ? n : 1;
    p.tiles = (int)((nn + kSortTile - 1) / kSortTile);
    const int64_t cells = n_cells + 1;
    const int64_t blocks = (cells + kSortTile - 1) / kSortTile;
    const int64_t per = (blocks + kBinMaxChunks - 1) / kBinMaxChunks;
    p.chunk_cells = per * kSortTile;
    p.chunks = (cells + p.chunk_cells - 1) / p.chunk_cells;
    const size_t ndw = (size_t)1 << p.width;
    p.blocks = (p.tiles + 31) / 32;
    p.off_hist = 0;
    p.off_block = bin_up256((size_t)p.passes * ndw * (size_t)p.tiles * 4);
    p.off_totals = p.off_block + bin_up256((size_t)p.blocks * ndw * 4);
    p.off_chunk = p.off_totals + bin_up256((size_t)p.passes * ndw * 4);
    p.off_clear = p.off_chunk + bin_up256((size_t)p.chunks * 4);
    p.scratch_bytes = p.off_clear + kBinControlBytes;
    return p;
}

struct BinWork {
    uint32_t* keys[2];
    uint32_t* vals[2];
    void* scratch;         // BinPlan::scratch_bytes
};

// Argument checks shared by the entry points: mesh shape and size; a cloud's
// kind, dtype, counts, pointers, alignment, release table and fold guard.
bool mesh_valid(const fla_mesh* m);
int cloud_valid(const fla_cloud* c, const fla_mesh* m);

// ---------------------------------------------------------------- launches
cudaError_t launch_carrier_sample(const fla_carrier_desc& c, const fla_mesh& m, double t, int dtype, void* nodes,
                                  cudaStream_t s);
cudaError_t launch_advance(const fla_cloud& cl, const fla_mesh& m, const void* nodes, int step0, int nsteps,
                           double dt, bool reset, DevStatus* st, int num_sms, cudaStream_t s,
                           const uint32_t* order = nullptr);
// Binning of one cloud with n > 0 (one memset, one kernel): cell keys, the
// stable sort of (key, index) and bin_start (n_cells + 1 words).  The sorted
// keys and permutation end in buffer bin_sorted_buffer(plan).  zero[0, nzero)
// (nzero <= 256) is cleared too: counters of the caller's later kernels.
// stall (a test hook) keeps one CTA from arriving at the grid barrier after
// the key phase, so that the others' waits run out.
cudaError_t launch_binning(const fla_cloud& cl, const fla_mesh& m, const BinWork& w, uint32_t* bin_start,
                           DevStatus* st, int stall, cudaStream_t s, uint32_t* zero = nullptr, int nzero = 0);
inline int bin_sorted_buffer(const BinPlan& p) { return p.passes & 1; }
cudaError_t launch_records(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg,
                           const uint32_t* perm, const uint32_t* bin_start, int64_t n_cells, void* rec,
                           unsigned int* ext_max, DevStatus* st, cudaStream_t s, float* aux = nullptr);
cudaError_t launch_learn_backward(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg,
                                  const uint32_t* perm, const uint32_t* bin_start, int64_t n_cells,
                                  const float* dldc, float* partial, int n_parts, DevStatus* st, cudaStream_t s);
// Candidates per work item: 4,096 in single precision; 64 in double
// precision, whose candidates cost many times more, so that a small mesh
// still spreads over many SMs (on a 64^2 Taylor-Green cloud the FP64 gather
// took 27.3 / 11.5 / 7.5 / 4.8 / 3.6 / 3.5 ms per run at 2,048 / 512 / 256 /
// 128 / 64 / 32 candidates).
constexpr uint32_t kItemChunkF32 = 4096, kItemChunkF64 = 64;
__host__ __device__ inline uint32_t nw_chunk(size_t elem) { return elem == 8 ? kItemChunkF64 : kItemChunkF32; }

// Work-item buffers of the tile gather (in the caller's workspace).
struct NwWork {
    uint32_t* tile_cand;               // tiles
    uint32_t* tile_items;              // tiles + 1
    unsigned long long* cand_total;    // zero before the launch
    unsigned int* done;                // zero before the launch (reset by the plan)
    unsigned int* counter;
    void* temp;                        // nw_temp_bytes
};
int nw_tiles(int dim, int N);
int64_t nw_item_budget(int dim, int N, int64_t n, size_t elem);
size_t nw_temp_bytes(int dim, int N, int64_t n, size_t elem);
cudaError_t launch_nw_gather(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg, const void* rec,
                             const uint32_t* bin_start, const unsigned int* ext_max, const NwWork& w,
                             const fla_sources& out, DevStatus* st, int num_sms, cudaStream_t s);
int gather2d_tiles(int N);
uint32_t gather2d_item_budget(int N, int64_t n);
size_t gather2d_temp_bytes(int N, int64_t n);
cudaError_t launch_gather2d(const fla_mesh& m, const fla_deposit_cfg& cfg, const void* rec, const uint32_t* bin_start,
                            const unsigned int* ext_max, uint32_t* tile_cand, uint32_t* tile_items,
                            unsigned int* counter, void* temp, uint32_t budget, const fla_sources& out,
                            DevStatus* st, int num_sms, cudaStream_t s);
cudaError_t launch_psicell(const fla_cloud& cl, const fla_mesh& m, double window_dt, int per_cell,
                           const uint32_t* perm, const uint32_t* bin_start, void* rec, const fla_psicell_out& out,
                           DevStatus* st, cudaStream_t s);
cudaError_t launch_cic(const fla_cloud& cl, const fla_mesh& m, double window_dt, int per_cell, const uint32_t* perm,
                       const uint32_t* bin_start, void* rec, const fla_psicell_out& out, DevStatus* st, cudaStream_t s);

}  // namespace fla
