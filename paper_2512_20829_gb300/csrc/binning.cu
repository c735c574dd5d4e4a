// Cell binning: integer cell keys, a stable LSD radix sort of (key, index)
// and the per-cell bin starts.  All integer work: bit-exact and deterministic.
//
// The sort processes tiles of 2,048 keys (256 threads x 8).  Per pass of a
// digit of up to 11 bits: (1) per-tile digit histograms, (2) per-digit
// exclusive scans over tiles, (3) a stable scatter in which each warp ranks
// its keys with __match_any_sync and per-warp running digit counters, so a
// key's destination depends only on the input order.
#include "batch.cuh"

namespace fla {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // 2,048 keys per tile
static_assert(RS_TILE == kSortTile, "tile size shared with the scratch sizes");
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_MAX_DIGITS = 2048;               // digits of up to 11 bits

template <typename T, int D>
__global__ void __launch_bounds__(256) k_cell_keys(const T* __restrict__ state, const uint32_t* __restrict__ meta,
                                                   int64_t n, int N, uint32_t sentinel, uint32_t* __restrict__ keys,
                                                   uint32_t* __restrict__ zero, int nzero)
{
    pdl_entry();
    // words the caller's later kernels need at zero (counters), cleared here
    // instead of by a separate memset in the stream
    if (blockIdx.x == 0 && (int)threadIdx.x < nzero) zero[threadIdx.x] = 0u;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key;
    keys[i] = cell_key_of<T, D>(state, meta, i, N, &key) ? key : sentinel;
}

// Batched clouds: global key = the cloud's cell offset + its cell key;
// droplets without a cell get the sentinel cells_total.
__global__ void __launch_bounds__(256) k_batch_keys(BatchDev b, uint32_t* __restrict__ keys)
{
    pdl_entry();
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= b.n_total) return;
    const int k = batch_find(b.drop_pre, b.n_clouds, g);
    const BatchCloud& c = b.clouds[k];
    const int64_t i = g - b.drop_pre[k];
    uint32_t key;
    const bool ok = c.dim == 2 ? cell_key_of<float, 2>(c.state, c.meta, i, c.N, &key)
                               : cell_key_of<float, 3>(c.state, c.meta, i, c.N, &key);
    keys[g] = ok ? (uint32_t)(c.cell_off + key) : (uint32_t)b.cells_total;
}

__global__ void k_batch_step(int* step, int nsteps)
{
    pdl_entry();
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += nsteps;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                           int width, uint32_t* __restrict__ counts, int tiles)
{
    pdl_entry();
    __shared__ uint32_t h[RS_MAX_DIGITS];
    const int nd = 1 << width;
    for (int t = threadIdx.x; t < nd; t += RS_THREADS) h[t] = 0;
    __syncthreads();
    const int64_t base = blockIdx.x * (int64_t)RS_TILE;
    const int lane = threadIdx.x & 31;
    uint32_t kv[RS_ITEMS];   // all of this thread's loads in flight before the ranking
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = base + k * RS_THREADS + threadIdx.x;
        kv[k] = j < n ? __ldg(keys + j) : 0u;
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = base + k * RS_THREADS + threadIdx.x;
        const bool valid = j < n;
        const uint32_t dg = valid ? (kv[k] >> shift) & (uint32_t)(nd - 1) : 0xFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += RS_THREADS) counts[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < RS_WARPS ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < RS_WARPS) s_warp[lane] = t;
    }
    __syncthreads();
    total = s_warp[RS_WARPS - 1];
    const uint32_t before = w > 0 ? s_warp[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

// One block per digit: exclusive scan of the digit's per-tile counts, and the digit total.
__global__ void __launch_bounds__(RS_THREADS) k_radix_scan(uint32_t* __restrict__ counts, int tiles,
                                                           uint32_t* __restrict__ totals)
{
    pdl_entry();
    __shared__ uint32_t s_warp[RS_WARPS];
    uint32_t* row = counts + (int64_t)blockIdx.x * tiles;
    uint32_t running = 0;
    for (int base = 0; base < tiles; base += RS_THREADS) {
        const int t = base + threadIdx.x;
        const uint32_t v = t < tiles ? row[t] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, s_warp, tot);
        if (t < tiles) row[t] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = running;
}

__global__ void __launch_bounds__(RS_THREADS, 1) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                              int64_t n, int shift, int width,
                                                              const uint32_t* __restrict__ counts,
                                                              const uint32_t* __restrict__ totals, int tiles)
{
    pdl_entry();
    __shared__ uint32_t s_base[RS_MAX_DIGITS];
    __shared__ uint16_t s_cnt[RS_WARPS][RS_MAX_DIGITS];
    __shared__ uint32_t s_warp[RS_WARPS];
    const int nd = 1 << width;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // this warp's keys and values, loaded before anything else so that their
    // latency overlaps the digit bases below
    const int64_t wbase = blockIdx.x * (int64_t)RS_TILE + w * (RS_ITEMS * 32);
    uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = wbase + k * 32 + lane;
        const bool valid = j < n;
        key[k] = valid ? __ldg(kin + j) : 0u;
        val[k] = valid ? (vin ? __ldg(vin + j) : (uint32_t)j) : 0u;
    }
    // digit bases: exclusive scan of the digit totals plus this tile's offset
    {
        constexpr int PER = RS_MAX_DIGITS / RS_THREADS;   // 8 digits per thread
        uint32_t v[PER], c[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {   // both loads issued before the scan
            const int d = tid * PER + q;
            v[q] = d < nd ? __ldg(totals + d) : 0u;
            c[q] = d < nd ? __ldg(counts + (int64_t)d * tiles + blockIdx.x) : 0u;
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) sum += v[q];
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(sum, s_warp, tot);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int d = tid * PER + q;
            if (d < nd) s_base[d] = ex + c[q];
            ex += v[q];
        }
    }
    for (int q = tid; q < RS_WARPS * RS_MAX_DIGITS; q += RS_THREADS) (&s_cnt[0][0])[q] = 0;
    __syncthreads();

    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = wbase + k * 32 + lane;
        const bool valid = j < n;
        const uint32_t kk = key[k];
        const uint32_t dg = valid ? (kk >> shift) & (uint32_t)(nd - 1) : 0xFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t before = valid ? s_cnt[w][dg] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) s_cnt[w][dg] = (uint16_t)(before + (uint32_t)__popc(peers));
        __syncwarp();
        rank[k] = valid ? before + (uint32_t)__popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    for (int d = tid; d < nd; d += RS_THREADS) {   // exclusive scan across warps, per digit
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            const uint32_t c = s_cnt[ww][d];
            s_cnt[ww][d] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        if (rank[k] == 0xffffffffu) continue;
        const uint32_t dg = (key[k] >> shift) & (uint32_t)(nd - 1);
        const uint32_t pos = s_base[dg] + s_cnt[w][dg] + rank[k];
        kout[pos] = key[k];
        vout[pos] = val[k];
    }
}

// bin_start[c] = first sorted position whose key is >= c, for c in [0, n_cells].
__global__ void __launch_bounds__(256) k_bin_start(const uint32_t* __restrict__ keys, int64_t n, int64_t n_cells,
                                                   uint32_t* __restrict__ bin_start)
{
    pdl_entry();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c > n_cells) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(keys + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    bin_start[c] = (uint32_t)lo;
}

}  // namespace

int sort_bits(uint32_t max_key)
{
    int b = 0;
    while (b < 32 && (max_key >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

int radix_tiles(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

// Digits of up to 11 bits (2 passes for the meshes used here) while the per-tile
// digit counts stay small next to the keys; 8-bit digits for very large clouds.
static int max_digit_bits(int64_t n) { return sort_digit_values(n) == 2048 ? 11 : 8; }

int sort_passes(int bits) { return (bits + 10) / 11; }

int sort_passes_n(int bits, int64_t n)
{
    const int w = max_digit_bits(n);
    return (bits + w - 1) / w;
}

cudaError_t launch_cell_keys(const fla_cloud& cl, const fla_mesh& m, uint32_t* keys, cudaStream_t s, uint32_t* zero,
                             int nzero)
{
    if (nzero > 256) return cudaErrorInvalidValue;
    if (cl.n == 0) return cudaSuccess;
    const int64_t nc = m.dim == 2 ? (int64_t)m.n * m.n : (int64_t)m.n * m.n * m.n;
    const unsigned blocks = (unsigned)((cl.n + 255) / 256);
    if (cl.dtype != FLA_F64) {   // FLA_F32X2: the key is formed from the hi planes
        if (m.dim == 2) launch_pdl(k_cell_keys<float, 2>, dim3(blocks), dim3(256), 0, s, (const float*)cl.state_dev, cl.meta_dev, cl.n, m.n, (uint32_t)nc, keys, zero, nzero);
        else launch_pdl(k_cell_keys<float, 3>, dim3(blocks), dim3(256), 0, s, (const float*)cl.state_dev, cl.meta_dev, cl.n, m.n, (uint32_t)nc, keys, zero, nzero);
    } else {
        if (m.dim == 2) launch_pdl(k_cell_keys<double, 2>, dim3(blocks), dim3(256), 0, s, (const double*)cl.state_dev, cl.meta_dev, cl.n, m.n, (uint32_t)nc, keys, zero, nzero);
        else launch_pdl(k_cell_keys<double, 3>, dim3(blocks), dim3(256), 0, s, (const double*)cl.state_dev, cl.meta_dev, cl.n, m.n, (uint32_t)nc, keys, zero, nzero);
    }
    return cudaGetLastError();
}

// Sorts keys[first] (values: the identity) into buffer first ^ (passes & 1).
cudaError_t launch_radix_sort(SortWork w, int64_t n, int bits, int first, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int passes = sort_passes_n(bits, n);
    const int width = (bits + passes - 1) / passes;
    const int tiles = radix_tiles(n);
    int cur = first;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * width;
        const int wp = (bits - shift) < width ? (bits - shift) : width;
        const int nd = 1 << wp;
        launch_pdl(k_radix_hist, dim3(tiles), dim3(RS_THREADS), 0, s, w.keys[cur], n, shift, wp, w.counts, tiles);
        launch_pdl(k_radix_scan, dim3(nd), dim3(RS_THREADS), 0, s, w.counts, tiles, w.totals);
        launch_pdl(k_radix_scatter, dim3(tiles), dim3(RS_THREADS), 0, s, w.keys[cur], p == 0 ? nullptr : w.vals[cur], w.keys[cur ^ 1],
                                                     w.vals[cur ^ 1], n, shift, wp, w.counts, w.totals, tiles);
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_start(const uint32_t* keys_sorted, int64_t n, int64_t n_cells, uint32_t* bin_start,
                             cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n_cells + 1 + 255) / 256);
    launch_pdl(k_bin_start, dim3(blocks), dim3(256), 0, s, keys_sorted, n, n_cells, bin_start);
    return cudaGetLastError();
}

cudaError_t launch_batch_keys(const BatchDev& b, uint32_t* keys, cudaStream_t s)
{
    if (b.n_total == 0) return cudaSuccess;
    launch_pdl(k_batch_keys, dim3((unsigned)((b.n_total + 255) / 256)), dim3(256), 0, s, b, keys);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchDev& b, int nsteps, cudaStream_t s)
{
    launch_pdl(k_batch_step, dim3(1), dim3(32), 0, s, b.step, nsteps);
    return cudaGetLastError();
}

}  // namespace fla
