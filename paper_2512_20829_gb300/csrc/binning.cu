// Cell binning: integer cell keys, a stable LSD radix sort of (key, index)
// and the per-cell bin starts.  All integer work: bit-exact and deterministic.
//
// A memset clears the per-cell counts (bin_start) and the barrier words; then
// one cooperative kernel (every CTA resident) runs these phases, separated by
// grid barriers, over tiles of 2,048 droplets:
//   B  per tile: the cell keys, the tile's histogram of the first digit and
//      the per-cell counts (one add per run of equal keys in a warp);
//   C  per digit: exclusive scan of its per-tile counts in tile order (the
//      tile prefixes) and the digit's total; on the first pass, per chunk of
//      cells: its count;
//   D  per tile: the stable scatter of the pass.  Each warp ranks its keys
//      with __match_any_sync and running per-digit counters (a key's place
//      depends only on the input order), the tile is reordered by digit in
//      shared memory and written out in runs of equal digits.  On the first
//      pass, per chunk of cells: the bin starts, an exclusive scan of the
//      counts;
//   H  before each further pass, per tile of the previous pass's output: its
//      histogram of the pass's digit; then C and D again.
// A barrier wait ends when every CTA has arrived, when another CTA has given
// up (the abort word), or after about a second, when it gives up itself: it
// sets the abort word and FLA_STATUS_WAIT_TIMEOUT.  The call's output is then
// not valid, and its bin starts are cleared (no cell holds a droplet, so later
// kernels read nothing of the sorted arrays).  Data written in the kernel is
// read back with L2-only loads (ld.cg): an SM's L1 may hold stale lines.
#include "batch.cuh"

namespace fla {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;    // 2,048 keys per tile
static_assert(RS_TILE == kSortTile, "tile size shared with the scratch sizes");
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_MAX_DIGITS = 1 << kSortMaxDigitBits;
constexpr int RS_PER = RS_MAX_DIGITS / RS_THREADS;             // digits per thread: 8
// shared memory: s_off, s_loc, s_key, s_val (u32 x 2,048 each), s_cnt (u16 x 8 x 2,048)
constexpr size_t RS_SMEM = 4 * RS_MAX_DIGITS * 4 + RS_WARPS * RS_MAX_DIGITS * 2;

struct BinArgs {
    int64_t n, n_cells;
    int bits, passes, width, tiles;
    int64_t chunks, chunk_cells, blocks;
    int stall;
    uint32_t* keys[2];
    uint32_t* vals[2];
    unsigned int* bar;         // barrier arrivals
    unsigned int* abort;
    unsigned int* done;        // CTAs that have finished
    uint32_t* totals;          // passes x 2^width digit totals
    uint32_t* hist;            // passes x tiles x 2^width: per-tile digit counts, then tile prefixes
    uint32_t* block_sum;       // blocks x 2^width: digit counts of each block of 32 tiles
    uint32_t* chunk_sum;       // chunks: cell counts per chunk
    uint32_t* bin_start;       // n_cells + 1: per-cell counts, then bin starts
    uint32_t* zero;            // caller's counters cleared by the call
    int nzero;
    DevStatus* status;
};

BinArgs bin_args(const BinPlan& p, const BinWork& w, uint32_t* bin_start, DevStatus* st, int stall, uint32_t* zero,
                 int nzero)
{
    BinArgs a{};
    a.n = p.n;
    a.n_cells = p.n_cells;
    a.bits = p.bits;
    a.passes = p.passes;
    a.width = p.width;
    a.tiles = p.tiles;
    a.chunks = p.chunks;
    a.chunk_cells = p.chunk_cells;
    a.blocks = p.blocks;
    a.stall = stall;
    for (int b = 0; b < 2; ++b) {
        a.keys[b] = w.keys[b];
        a.vals[b] = w.vals[b];
    }
    char* z = static_cast<char*>(w.scratch);
    a.bar = reinterpret_cast<unsigned int*>(z + p.off_clear);
    a.abort = a.bar + 1;
    a.done = a.bar + 2;
    a.totals = reinterpret_cast<uint32_t*>(z + p.off_totals);
    a.hist = reinterpret_cast<uint32_t*>(z + p.off_hist);
    a.block_sum = reinterpret_cast<uint32_t*>(z + p.off_block);
    a.chunk_sum = reinterpret_cast<uint32_t*>(z + p.off_chunk);
    a.bin_start = bin_start;
    a.zero = zero;
    a.nzero = nzero;
    a.status = st;
    return a;
}

// Cell keys of a single cloud and of the batched clouds (global cell space).
template <typename T, int D>
struct CloudKeys {
    const T* state;
    const uint32_t* meta;
    int N;
    uint32_t sentinel;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const
    {
        uint32_t key;
        return cell_key_of<T, D>(state, meta, i, N, &key) ? key : sentinel;
    }
};

struct BatchKeys {
    BatchDev b;
    __device__ __forceinline__ uint32_t operator()(int64_t g) const
    {
        const int c = batch_find(b.drop_pre, b.n_clouds, g);
        const BatchCloud& cl = b.clouds[c];
        const int64_t i = g - b.drop_pre[c];
        uint32_t key;
        const bool ok = cl.dim == 2 ? cell_key_of<float, 2>(cl.state, cl.meta, i, cl.N, &key)
                                    : cell_key_of<float, 3>(cl.state, cl.meta, i, cl.N, &key);
        return ok ? (uint32_t)(cl.cell_off + key) : (uint32_t)b.cells_total;
    }
};

// Grid barrier number gen (1, 2, ...): returns false when a wait gave up.
__device__ bool grid_barrier(const BinArgs& a, unsigned int gen, bool arrive = true)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = gen * gridDim.x;
        // the CTA's writes (ordered before thread 0 by the CTA barrier) are
        // made visible before the arrival, and the other CTAs' writes before
        // this CTA's later reads
        __threadfence();
        if (arrive) atomicAdd(a.bar, 1u);
        int ok = 1;
        unsigned long long t0 = 0;
        for (unsigned int poll = 0;; ++poll) {
            if (*reinterpret_cast<volatile unsigned int*>(a.bar) >= target) break;
            if (*reinterpret_cast<volatile unsigned int*>(a.abort)) {
                ok = 0;
                break;
            }
            if (poll < 256) continue;   // tight spin first: most barriers complete within a few microseconds
            const unsigned long long now = global_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitLimitNs) {
                atomicExch(a.abort, 1u);
                if (a.status) atomicOr(&a.status->flags, kFlagWaitTimeout);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

__device__ __forceinline__ int pass_digits(const BinArgs& a, int p)
{
    const int shift = p * a.width;
    return 1 << (a.bits - shift < a.width ? a.bits - shift : a.width);
}

// The histogram of pass p's digit over one tile's keys (kv[k]: droplet
// t * 2,048 + k * 256 + threadIdx.x), written to hist without atomics.
__device__ void tile_hist(const BinArgs& a, int p, int64_t t, const uint32_t kv[RS_ITEMS], uint32_t* h)
{
    const int nd = pass_digits(a, p);
    const int shift = p * a.width;
    const int lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < nd; q += RS_THREADS) h[q] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = t * RS_TILE + k * RS_THREADS + threadIdx.x;
        const bool valid = j < a.n;
        const uint32_t dg = valid ? (kv[k] >> shift) & (uint32_t)(nd - 1) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    uint32_t* row = a.hist + ((int64_t)p * a.tiles + t) * (1 << a.width);
    for (int q = threadIdx.x; q < nd; q += RS_THREADS) row[q] = h[q];
    __syncthreads();
}

// Phase B for one tile: keys, the first pass's histogram and cell counts.
template <typename KF>
__device__ void key_tile(const BinArgs& a, const KF& kf, int64_t t, uint32_t* h)
{
    const int lane = threadIdx.x & 31;
    uint32_t kv[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = t * RS_TILE + k * RS_THREADS + threadIdx.x;
        kv[k] = 0u;
        if (j < a.n) {
            kv[k] = kf(j);
            a.keys[0][j] = kv[k];
        }
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = t * RS_TILE + k * RS_THREADS + threadIdx.x;
        const bool cell = j < a.n && (int64_t)kv[k] < a.n_cells;
        const unsigned run = __match_any_sync(0xffffffffu, cell ? kv[k] : 0xffffffffu);
        if (cell && (__ffs(run) - 1) == lane) atomicAdd(a.bin_start + kv[k], (uint32_t)__popc(run));
    }
    tile_hist(a, 0, t, kv, h);
}

// Phase H for one tile of pass p's input (the previous pass's output).
__device__ void input_tile_hist(const BinArgs& a, int p, int64_t t, uint32_t* h)
{
    const uint32_t* kin = a.keys[p & 1];
    uint32_t kv[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t j = t * RS_TILE + k * RS_THREADS + threadIdx.x;
        kv[k] = j < a.n ? __ldcg(kin + j) : 0u;
    }
    tile_hist(a, p, t, kv, h);
}

// Phase C for up to kScanTilesInCta tiles: one CTA per 32 digits (lane =
// digit), its warps splitting the tiles: each sums its share, the shares are
// scanned across warps, and each warp rescans its share from its offset, in
// place; warp 0 writes the digit totals.
constexpr int64_t kScanTilesInCta = 256;
__device__ void tile_prefixes_cta(const BinArgs& a, int p, uint32_t (*s_part)[32])
{
    const int nd = pass_digits(a, p);
    const int ndw = 1 << a.width;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* hp = a.hist + (int64_t)p * a.tiles * ndw;
    const int64_t per = (a.tiles + RS_WARPS - 1) / RS_WARPS;   // at most 32
    const int64_t t0 = w * per;
    const int64_t t1 = t0 + per < a.tiles ? t0 + per : a.tiles;
    for (int g = blockIdx.x; g * 32 < nd; g += gridDim.x) {
        const int d = g * 32 + lane;
        const bool on = d < nd;
        uint32_t sum = 0;
        for (int h = 0; h < 2; ++h) {
            uint32_t v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int64_t t = t0 + 16 * h + k;
                v[k] = on && t < t1 ? __ldcg(hp + t * ndw + d) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) sum += v[k];
        }
        s_part[w][lane] = sum;
        __syncthreads();
        uint32_t run = 0, total = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            const uint32_t c = s_part[ww][lane];
            run += ww < w ? c : 0u;
            total += c;
        }
        __syncthreads();
        for (int h = 0; h < 2; ++h) {
            uint32_t v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int64_t t = t0 + 16 * h + k;
                v[k] = on && t < t1 ? __ldcg(hp + t * ndw + d) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int64_t t = t0 + 16 * h + k;
                if (on && t < t1) hp[t * ndw + d] = run;
                run += v[k];
            }
        }
        if (w == 0 && on) a.totals[p * ndw + d] = total;
    }
}

// Phase C in two steps, one warp per (32 digits, block of 32 tiles), lane =
// digit.  C1: the block's count of each digit.  C2 (after a barrier): the
// counts of the earlier blocks, then the exclusive scan over the block's
// tiles in tile order, in place; the last block also writes the digit totals.
__device__ void block_sums(const BinArgs& a, int p)
{
    const int nd = pass_digits(a, p);
    const int ndw = 1 << a.width;
    const int lane = threadIdx.x & 31;
    const uint32_t* hp = a.hist + (int64_t)p * a.tiles * ndw;
    const int64_t groups = (nd + 31) / 32, tasks = groups * a.blocks;
    const int64_t warps = (int64_t)gridDim.x * RS_WARPS;
    for (int64_t task = (int64_t)blockIdx.x * RS_WARPS + (threadIdx.x >> 5); task < tasks; task += warps) {
        const int64_t b = task / groups;
        const int d = (int)(task % groups) * 32 + lane;
        const int64_t t0 = b * 32, t1 = t0 + 32 < a.tiles ? t0 + 32 : a.tiles;
        uint32_t sum = 0;
        if (d < nd) {
#pragma unroll 8
            for (int64_t t = t0; t < t1; ++t) sum += __ldcg(hp + t * ndw + d);
            a.block_sum[b * ndw + d] = sum;
        }
    }
}

__device__ void tile_prefixes(const BinArgs& a, int p)
{
    const int nd = pass_digits(a, p);
    const int ndw = 1 << a.width;
    const int lane = threadIdx.x & 31;
    uint32_t* hp = a.hist + (int64_t)p * a.tiles * ndw;
    const int64_t groups = (nd + 31) / 32, tasks = groups * a.blocks;
    const int64_t warps = (int64_t)gridDim.x * RS_WARPS;
    for (int64_t task = (int64_t)blockIdx.x * RS_WARPS + (threadIdx.x >> 5); task < tasks; task += warps) {
        const int64_t b = task / groups;
        const int d = (int)(task % groups) * 32 + lane;
        if (d >= nd) continue;
        uint32_t run = 0;
#pragma unroll 8
        for (int64_t bb = 0; bb < b; ++bb) run += __ldcg(a.block_sum + bb * ndw + d);
        const int64_t t0 = b * 32, t1 = t0 + 32 < a.tiles ? t0 + 32 : a.tiles;
        for (int h = 0; h < 2; ++h) {
            const int64_t th = t0 + 16 * h;
            uint32_t v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = th + k < t1 ? __ldcg(hp + (th + k) * ndw + d) : 0u;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (th + k < t1) hp[(th + k) * ndw + d] = run;
                run += v[k];
            }
        }
        if (b == a.blocks - 1) a.totals[p * ndw + d] = run;
    }
}

// Phase C, first pass: the count of each chunk of cells.
__device__ void chunk_counts(const BinArgs& a, uint32_t* s_warp)
{
    const int64_t cells = a.n_cells + 1;
    for (int64_t c = blockIdx.x; c < a.chunks; c += gridDim.x) {
        const int64_t c0 = c * a.chunk_cells;
        const int64_t c1 = c0 + a.chunk_cells < cells ? c0 + a.chunk_cells : cells;
        uint32_t sum = 0;
        for (int64_t i = c0 + threadIdx.x; i < c1; i += RS_THREADS) sum += __ldcg(a.bin_start + i);
        uint32_t tot;
        block_exclusive_scan(sum, s_warp, tot);
        if (threadIdx.x == 0) a.chunk_sum[c] = tot;
    }
}

// Phase D, first pass: bin starts of each chunk of cells.
__device__ void chunk_starts(const BinArgs& a, uint32_t* s_warp)
{
    const int64_t cells = a.n_cells + 1;
    for (int64_t c = blockIdx.x; c < a.chunks; c += gridDim.x) {
        uint32_t pre = 0;
        for (int64_t i = threadIdx.x; i < c; i += RS_THREADS) pre += __ldcg(a.chunk_sum + i);
        uint32_t run;
        block_exclusive_scan(pre, s_warp, run);   // run = sum of the earlier chunks' counts
        const int64_t c0 = c * a.chunk_cells;
        const int64_t c1 = c0 + a.chunk_cells < cells ? c0 + a.chunk_cells : cells;
        for (int64_t b0 = c0; b0 < c1; b0 += RS_TILE) {
            uint32_t v[RS_ITEMS], s = 0;
#pragma unroll
            for (int k = 0; k < RS_ITEMS; ++k) {
                const int64_t i = b0 + threadIdx.x * RS_ITEMS + k;
                v[k] = i < c1 ? __ldcg(a.bin_start + i) : 0u;
                s += v[k];
            }
            uint32_t btot;
            uint32_t ex = run + block_exclusive_scan(s, s_warp, btot);
#pragma unroll
            for (int k = 0; k < RS_ITEMS; ++k) {
                const int64_t i = b0 + threadIdx.x * RS_ITEMS + k;
                if (i < c1) a.bin_start[i] = ex;
                ex += v[k];
            }
            run += btot;
        }
    }
}

struct ScatterSmem {
    uint32_t* off;                      // global start of each digit's run of this tile
    uint32_t* loc;                      // tile-local start of each digit's run
    uint32_t* key;                      // the tile's keys and values in digit order
    uint32_t* val;
    uint16_t (*cnt)[RS_MAX_DIGITS];     // per warp and digit: running counts, then warp offsets
};

// Phase D: the stable scatter of pass p from buffer p & 1 into the other.
__device__ void scatter_pass(const BinArgs& a, int p, const ScatterSmem& sm, uint32_t* s_warp)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int ndw = 1 << a.width;
    const int shift = p * a.width;
    const int nd = pass_digits(a, p);
    const int cur = p & 1;
    const uint32_t* hp = a.hist + (int64_t)p * a.tiles * ndw;
    // digit bases of this pass (the same for every tile): thread owns digits
    // tid * 8 + q, q < 8
    uint32_t base[RS_PER];
    {
        uint32_t v[RS_PER], sum = 0;
#pragma unroll
        for (int q = 0; q < RS_PER; ++q) {
            const int d = tid * RS_PER + q;
            v[q] = d < nd ? __ldcg(a.totals + p * ndw + d) : 0u;
            sum += v[q];
        }
        uint32_t all;
        uint32_t ex = block_exclusive_scan(sum, s_warp, all);
#pragma unroll
        for (int q = 0; q < RS_PER; ++q) {
            base[q] = ex;
            ex += v[q];
        }
    }
    const uint32_t* kin = a.keys[cur];
    const uint32_t* vin = a.vals[cur];
    uint32_t* kout = a.keys[cur ^ 1];
    uint32_t* vout = a.vals[cur ^ 1];
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
        const int64_t wbase = t * RS_TILE + w * (RS_ITEMS * 32);
        uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
        for (int k = 0; k < RS_ITEMS; ++k) {
            const int64_t j = wbase + k * 32 + lane;
            const bool valid = j < a.n;
            key[k] = valid ? __ldcg(kin + j) : 0u;
            val[k] = valid ? (p == 0 ? (uint32_t)j : __ldcg(vin + j)) : 0u;
        }
#pragma unroll
        for (int q = 0; q < RS_PER; ++q) {
            const int d = tid * RS_PER + q;
            if (d < nd) sm.off[d] = base[q] + __ldcg(hp + t * ndw + d);
        }
        for (int q = tid; q < RS_WARPS * RS_MAX_DIGITS / 8; q += RS_THREADS)
            reinterpret_cast<uint4*>(&sm.cnt[0][0])[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        // ranks within the warp, in (k, lane) order
#pragma unroll
        for (int k = 0; k < RS_ITEMS; ++k) {
            const int64_t j = wbase + k * 32 + lane;
            const bool valid = j < a.n;
            const uint32_t dg = valid ? (key[k] >> shift) & (uint32_t)(nd - 1) : 0xFFFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const uint32_t before = valid ? sm.cnt[w][dg] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) sm.cnt[w][dg] = (uint16_t)(before + (uint32_t)__popc(peers));
            __syncwarp();
            rank[k] = valid ? before + (uint32_t)__popc(peers & lt) : 0xffffffffu;
        }
        __syncthreads();
        for (int d = tid; d < nd; d += RS_THREADS) {   // per digit: offsets of the warps, the tile's count
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < RS_WARPS; ++ww) {
                const uint32_t c = sm.cnt[ww][d];
                sm.cnt[ww][d] = (uint16_t)run;
                run += c;
            }
            sm.loc[d] = run;
        }
        __syncthreads();
        {   // tile-local digit starts: exclusive scan of the counts
            uint32_t c[RS_PER], sum = 0;
#pragma unroll
            for (int q = 0; q < RS_PER; ++q) {
                const int d = tid * RS_PER + q;
                c[q] = d < nd ? sm.loc[d] : 0u;
                sum += c[q];
            }
            uint32_t all;
            uint32_t ex = block_exclusive_scan(sum, s_warp, all);
#pragma unroll
            for (int q = 0; q < RS_PER; ++q) {
                const int d = tid * RS_PER + q;
                if (d < nd) sm.loc[d] = ex;
                ex += c[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RS_ITEMS; ++k) {
            if (rank[k] == 0xffffffffu) continue;
            const uint32_t dg = (key[k] >> shift) & (uint32_t)(nd - 1);
            const uint32_t lp = sm.loc[dg] + sm.cnt[w][dg] + rank[k];
            sm.key[lp] = key[k];
            sm.val[lp] = val[k];
        }
        __syncthreads();
        // write out in digit order: consecutive threads, consecutive positions of a run
        const int64_t rem = a.n - t * RS_TILE;
        const int tile_n = rem < RS_TILE ? (int)rem : RS_TILE;
        for (int i = tid; i < tile_n; i += RS_THREADS) {
            const uint32_t k = sm.key[i];
            const uint32_t dg = (k >> shift) & (uint32_t)(nd - 1);
            const uint32_t g = sm.off[dg] + ((uint32_t)i - sm.loc[dg]);
            kout[g] = k;
            vout[g] = sm.val[i];
        }
        __syncthreads();   // shared memory is rewritten by the next tile
    }
}

// The phases B, C, D and H over the calling CTA's tiles; gen is the barrier
// generation (advanced by each barrier).  Returns false when a wait gave up.
// stall_first: this CTA does not arrive at the first barrier (test hook).
template <typename KF>
__device__ bool binning_phases(const BinArgs& a, const KF& kf, unsigned char* smem_raw, unsigned int& gen,
                               bool stall_first)
{
    ScatterSmem sm;
    sm.off = reinterpret_cast<uint32_t*>(smem_raw);
    sm.loc = sm.off + RS_MAX_DIGITS;
    sm.key = sm.loc + RS_MAX_DIGITS;
    sm.val = sm.key + RS_MAX_DIGITS;
    sm.cnt = reinterpret_cast<uint16_t (*)[RS_MAX_DIGITS]>(sm.val + RS_MAX_DIGITS);
    __shared__ uint32_t s_warp[RS_WARPS];
    __shared__ uint32_t s_part[RS_WARPS][32];
    bool ok = true;

    // B: keys, first-pass tile histograms, cell counts (bin_start starts at
    // zero: cleared before the phase)
    if (blockIdx.x == 0 && (int)threadIdx.x < a.nzero) a.zero[threadIdx.x] = 0u;
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) key_tile(a, kf, t, sm.off);
    ok = grid_barrier(a, ++gen, !stall_first);
    for (int p = 0; ok && p < a.passes; ++p) {
        if (p > 0) {
            // H: the pass's tile histograms of the previous pass's output
            for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) input_tile_hist(a, p, t, sm.off);
            ok = grid_barrier(a, ++gen);
            if (!ok) break;
        }
        // C: tile prefixes and digit totals of this pass; chunk counts of the cells
        if (a.tiles <= kScanTilesInCta) {
            tile_prefixes_cta(a, p, s_part);
            if (p == 0) chunk_counts(a, s_warp);
            ok = grid_barrier(a, ++gen);
            if (!ok) break;
        } else {
            block_sums(a, p);
            if (p == 0) chunk_counts(a, s_warp);
            ok = grid_barrier(a, ++gen);
            if (!ok) break;
            tile_prefixes(a, p);
            ok = grid_barrier(a, ++gen);
            if (!ok) break;
        }
        // D: scatter; bin starts
        scatter_pass(a, p, sm, s_warp);
        if (p == 0) chunk_starts(a, s_warp);
        if (p + 1 < a.passes) ok = grid_barrier(a, ++gen);
    }
    return ok;
}

template <typename KF>
__global__ void __launch_bounds__(RS_THREADS) k_binning(BinArgs a, KF kf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_last;
    unsigned int gen = 0;
    binning_phases(a, kf, smem_raw, gen, a.stall && blockIdx.x == 0);

    // After a wait gave up, the permutation and the bin starts may disagree:
    // the last CTA to finish then clears bin_start, so that every cell is
    // empty and later kernels read nothing of the sorted arrays.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (*reinterpret_cast<volatile unsigned int*>(a.abort))
            for (int64_t c = threadIdx.x; c <= a.n_cells; c += RS_THREADS) a.bin_start[c] = 0u;
    }
}

// Cooperative launch of k_binning<KF> over as many CTAs as the work has, at
// most the number that can be resident at once.
template <typename KF>
cudaError_t launch_coop(const BinPlan& p, const BinArgs& a, const KF& kf, cudaStream_t s)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_binning<KF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_binning<KF>, RS_THREADS, RS_SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t want = p.tiles;
    want = p.chunks > want ? p.chunks : want;
    const int64_t digit_ctas = ((((int64_t)1 << p.width) + 31) / 32 * p.blocks + RS_WARPS - 1) / RS_WARPS;
    want = digit_ctas > want ? digit_ctas : want;
    const int64_t cap = (int64_t)occ * sms;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    // barrier words and (where it follows directly) bin_start: one memset; else two
    char* clear = reinterpret_cast<char*>(a.bar);
    const size_t clear_bytes = p.scratch_bytes - p.off_clear;
    const size_t bins = ((size_t)p.n_cells + 1) * 4;
    if (reinterpret_cast<char*>(a.bin_start) == clear + clear_bytes) {
        e = cudaMemsetAsync(clear, 0, clear_bytes + bins, s);
    } else {
        e = cudaMemsetAsync(clear, 0, clear_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.bin_start, 0, bins, s);
    }
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(RS_THREADS);
    cfg.dynamicSmemBytes = RS_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_binning<KF>, a, kf);
}

__global__ void k_batch_step(int* step, int nsteps)
{
    pdl_entry();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        step[0] += nsteps;
        step[1] = 1;   // this window's binning orders the next window's advance
    }
}

}  // namespace

cudaError_t launch_binning(const fla_cloud& cl, const fla_mesh& m, const BinWork& w, uint32_t* bin_start,
                           DevStatus* st, int stall, cudaStream_t s, uint32_t* zero, int nzero)
{
    if (nzero > 256) return cudaErrorInvalidValue;
    if (cl.n == 0) return cudaSuccess;
    const int64_t nc = m.dim == 2 ? (int64_t)m.n * m.n : (int64_t)m.n * m.n * m.n;
    const BinPlan p = bin_plan(cl.n, nc);
    const BinArgs a = bin_args(p, w, bin_start, st, stall, zero, nzero);
    const uint32_t sentinel = (uint32_t)nc;
    if (cl.dtype != FLA_F64) {   // FLA_F32X2: the key is formed from the hi planes
        const float* x = (const float*)cl.state_dev;
        if (m.dim == 2) return launch_coop(p, a, CloudKeys<float, 2>{x, cl.meta_dev, m.n, sentinel}, s);
        return launch_coop(p, a, CloudKeys<float, 3>{x, cl.meta_dev, m.n, sentinel}, s);
    }
    const double* x = (const double*)cl.state_dev;
    if (m.dim == 2) return launch_coop(p, a, CloudKeys<double, 2>{x, cl.meta_dev, m.n, sentinel}, s);
    return launch_coop(p, a, CloudKeys<double, 3>{x, cl.meta_dev, m.n, sentinel}, s);
}

cudaError_t launch_batch_binning(const BatchDev& b, const BinWork& w, uint32_t* bin_start, DevStatus* st,
                                 cudaStream_t s)
{
    if (b.n_total == 0) return cudaSuccess;
    const BinPlan p = bin_plan(b.n_total, b.cells_total);
    return launch_coop(p, bin_args(p, w, bin_start, st, 0, nullptr, 0), BatchKeys{b}, s);
}

cudaError_t launch_batch_step(const BatchDev& b, int nsteps, cudaStream_t s)
{
    launch_pdl(k_batch_step, dim3(1), dim3(32), 0, s, b.step, nsteps);
    return cudaGetLastError();
}

}  // namespace fla

#ifdef FLA_WINDOW_PHASES
// Phase and barrier of the persistent window kernel (window.cuh).
#include "window.cuh"
namespace fla {

static_assert(sizeof(BinArgs) <= sizeof(WindowBlob), "binning arguments fit the window's blob");

__device__ bool window_binning(const WindowBlob& bin, const BatchDev& b, unsigned int& gen, unsigned char* smem)
{
    const BinArgs& a = *reinterpret_cast<const BinArgs*>(bin.b);
    return binning_phases(a, BatchKeys{b}, smem, gen, false);
}

__device__ bool window_barrier(const WindowBlob& bin, unsigned int gen, bool arrive)
{
    return grid_barrier(*reinterpret_cast<const BinArgs*>(bin.b), gen, arrive);
}

// The binning's arguments for all clouds and the control words (barrier
// arrivals, abort, done) that must be zero before the window kernel.
size_t window_bin_blob(WindowBlob* out, const BatchDev& b, const BinWork& w, uint32_t* bin_start, DevStatus* st,
                       void** clear, size_t* clear_bytes)
{
    const BinPlan p = bin_plan(b.n_total > 0 ? b.n_total : 1, b.cells_total);
    BinArgs a = bin_args(p, w, bin_start, st, 0, nullptr, 0);
    if (b.n_total == 0) a.n = 0;
    memset(out, 0, sizeof(*out));
    memcpy(out->b, &a, sizeof(a));
    *clear = a.bar;
    *clear_bytes = p.scratch_bytes - p.off_clear;
    return sizeof(a);
}

size_t window_binning_smem() { return RS_SMEM; }

}  // namespace fla
#endif
