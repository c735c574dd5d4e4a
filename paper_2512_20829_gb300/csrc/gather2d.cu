// Kernel-regression gather for 2D clouds with the spherical kernel in single
// precision (Eqs. 13-16): the load-balanced, lane-per-record form.
//
// Work decomposition.  The mesh is cut into 16x16-cell tiles.  The candidate
// records of a tile are the records of the cells within R of it (R from the
// largest support in the cloud); because records are sorted by cell, they are
// the concatenation of one contiguous segment per neighbourhood row.  A plan
// kernel counts each tile's candidates and cuts the list into work items of
// at most kChunk candidates, so that a dense cluster of droplets (a caustic)
// is spread over many CTAs instead of stalling one.
//
// Evaluation.  Persistent warps take (work item, 4x4 cell block) units from a
// counter, independently of each other (no CTA barriers).  A warp streams the item's
// candidates from the row segments that can reach its block, keeps (by ballot)
// the records whose support reaches the block, queues them in shared memory
// (records covering the whole block and the others in two queues, so each batch
// takes one path) and, 32 at a time, lets each lane evaluate one record against
// all 16 cells of the block.  The Gaussian is separable, so a lane needs 4 + 4 ex2
// per record instead of one per cell: w = 2^(c dx^2) * 2^(c dy^2 + log2(1/h)).
// The truncation test keeps the single-precision form r^2 = fma(dy, dy, dx*dx)
// <= 9 h^2.  Each lane accumulates its own records; the 32 lane partials of a
// cell are then summed in a fixed lane order, written per work item, and a
// combine kernel adds the items of a tile in item order (Neumaier-compensated)
// and divides.  Every step has a fixed order: the result does not depend on
// timing.
#include "fla_internal.cuh"

namespace fla {
namespace {

constexpr int kTile = 16;          // tile edge in cells
constexpr int kBlocks = 16;        // 4 x 4 blocks of 4 x 4 cells per tile
constexpr int kWarps = 16;         // warps per CTA (one CTA per SM; 8 / 12 warps measured slower)
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 2048;       // candidates per work item (2,048-3,072 measured best on the 512^2 jet)
constexpr int kRing = 64;          // queued records per warp
constexpr int kScratchFloats = 32 * 33;  // per-warp reduction scratch (padded rows)

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int support_cells(const unsigned int* ext_max, int N)
{
    const float ext2max = __uint_as_float(__ldg(ext_max));
    // rounded explicitly: the plan and the gather must agree on R to the bit
    return (int)floorf(__fadd_rn(__fmul_rn(__fsqrt_rn(ext2max), (float)N), 0.5f)) + 1;
}

struct PlanArgs {
    const uint32_t* bin_start;
    const unsigned int* ext_max;
    uint32_t* tile_cand;
    uint32_t* tile_items;      // n_tiles + 1
    int N, tiles_x, n_tiles;
    uint32_t budget;           // maximum number of work items (temp buffer size)
    unsigned int* done;        // CTAs of the plan that have finished (the last one scans; reset by it)
};

// Exclusive scan of the per-tile item counts by one CTA; if the total exceeds
// the budget, every non-empty tile gets a single item instead.
__device__ void scan_items(const PlanArgs& a)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t running = 0;
        for (int base = 0; base < a.n_tiles; base += blockDim.x) {
            const int t = base + tid;
            uint32_t v = 0;
            if (t < a.n_tiles) v = pass == 0 ? a.tile_items[t] : (a.tile_cand[t] ? 1u : 0u);
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_warp[w] = x;
            __syncthreads();
            if (w == 0) {
                uint32_t sw = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, sw, o);
                    if (lane >= o) sw += y;
                }
                if (lane < nw) s_warp[lane] = sw;
            }
            __syncthreads();
            const uint32_t excl = running + (w > 0 ? s_warp[w - 1] : 0) + x - v;
            if (t < a.n_tiles) a.tile_items[t] = excl;
            running += s_warp[nw - 1];
            __syncthreads();
        }
        if (tid == 0) {
            a.tile_items[a.n_tiles] = running;
            s_total = running;
        }
        __syncthreads();
        if (pass == 0 && s_total <= a.budget) break;
    }
}

// Candidates of each tile (one warp per tile, lanes over the neighbourhood
// rows) and the number of work items it needs; the last CTA to finish scans
// the item counts into item offsets.
__global__ void __launch_bounds__(256) k_plan2d(PlanArgs a)
{
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (t < a.n_tiles) {
        const int N = a.N, R = support_cells(a.ext_max, N);
        const int tx0 = (t % a.tiles_x) * kTile, ty0 = (t / a.tiles_x) * kTile;
        const int xlo = max(tx0 - R, 0), xhi = min(tx0 + kTile - 1 + R, N - 1);
        const int ylo = max(ty0 - R, 0), yhi = min(ty0 + kTile - 1 + R, N - 1);
        uint32_t cand = 0;
        for (int y = ylo + lane; y <= yhi; y += 32) {
            const int64_t rb = (int64_t)y * N;
            cand += __ldg(a.bin_start + rb + xhi + 1) - __ldg(a.bin_start + rb + xlo);
        }
        cand = __reduce_add_sync(0xffffffffu, cand);
        if (lane == 0) {
            a.tile_cand[t] = cand;
            a.tile_items[t] = cand ? (cand + kChunk - 1) / kChunk : 0;
        }
    }
    // the last CTA to finish does the scan
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    scan_items(a);
    if (threadIdx.x == 0) *a.done = 0u;
}

struct G2Args {
    const float4* rec;          // 2 float4 per record: x, y, c, lih | a_m, a_x, a_y, r2max
    const uint32_t* bin_start;
    const unsigned int* ext_max;
    const uint32_t* tile_cand;
    const uint32_t* tile_items;
    unsigned int* counter;
    float4* temp;               // [item][256 cells] of (D, N_m, N_x, N_y)
    unsigned long long* pairs;
    int N, tiles_x, n_tiles;
};

__global__ void __launch_bounds__(kThreads, 1) k_gather2d_items(G2Args a)
{
    pdl_entry();
    extern __shared__ __align__(16) float4 smem4[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* ring = smem4 + warp * (kScratchFloats / 4 + 8);   // per-warp region (two rings, then scratch)
    const int N = a.N;
    const float fN = (float)N;
    const int R = support_cells(a.ext_max, N);
    const uint32_t total = __ldg(a.tile_items + a.n_tiles) * kBlocks;   // (item, block) units
    const unsigned lt = (1u << lane) - 1u;
    unsigned npairs = 0;

    for (;;) {
        // each warp takes one (work item, 4x4 block) unit at a time: no CTA barriers
        uint32_t unit = 0;
        if (lane == 0) unit = atomicAdd(a.counter, 1u);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= total) break;
        const uint32_t item = unit / kBlocks;
        const int blk = (int)(unit % kBlocks);
        // tile of this item: last t with tile_items[t] <= item
        int lo = 0, hi = a.n_tiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.tile_items + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const int t = lo;
        const uint32_t i0 = __ldg(a.tile_items + t), ni = __ldg(a.tile_items + t + 1) - i0;
        const uint32_t cand = __ldg(a.tile_cand + t);
        const uint32_t csize = (cand + ni - 1) / ni;
        const uint32_t c0 = (item - i0) * csize, c1 = min(c0 + csize, cand);
        const int tx0 = (t % a.tiles_x) * kTile, ty0 = (t / a.tiles_x) * kTile;
        const int xlo = max(tx0 - R, 0), xhi = min(tx0 + kTile - 1 + R, N - 1);
        const int ylo = max(ty0 - R, 0), yhi = min(ty0 + kTile - 1 + R, N - 1);
        // the 4x4 block of cells
        const int bx0 = tx0 + 4 * (blk & 3), by0 = ty0 + 4 * (blk >> 2);
        const bool live = bx0 < N && by0 < N;
        const int bx1 = min(bx0 + 3, N - 1), by1 = min(by0 + 3, N - 1);
        float xc[4], yc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xc[i] = ((float)(bx0 + i) + 0.5f) / fN;
            yc[i] = ((float)(by0 + i) + 0.5f) / fN;
        }
        const float bxl = ((float)bx0 + 0.5f) / fN, bxh = ((float)bx1 + 0.5f) / fN;
        const float byl = ((float)by0 + 0.5f) / fN, byh = ((float)by1 + 0.5f) / fN;
        const int wxlo = max(bx0 - R, xlo), wxhi = min(bx1 + R, xhi);
        const int wylo = by0 - R, wyhi = by1 + R;

        float acc[16][4];
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][q] = 0.0f;

        // Evaluation of one record against the 16 cells.  FULL: the record's
        // truncated support covers the whole block (decided when it was queued),
        // so no per-cell test is needed.
        auto eval = [&](const float4 ra, const float4 rb, const bool full) {
            float dxx[4], ex[4], dyv[4], ey[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float dx = __fsub_rn(xc[i], ra.x);
                dxx[i] = __fmul_rn(dx, dx);
                ex[i] = ex2_approx(dxx[i] * ra.z);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                dyv[j] = __fsub_rn(yc[j], ra.y);
                ey[j] = ex2_approx(fmaf(dyv[j] * dyv[j], ra.z, ra.w));
            }
            if (full) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float w = ex[i] * ey[j];
                        float* c = acc[4 * j + i];
                        c[0] += w;
                        c[1] = fmaf(w, rb.x, c[1]);
                        c[2] = fmaf(w, rb.y, c[2]);
                        c[3] = fmaf(w, rb.z, c[3]);
                    }
                npairs += 16;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float r2 = __fmaf_rn(dyv[j], dyv[j], dxx[i]);   // single-precision decision
                        const bool in = r2 <= rb.w;
                        const float w = in ? ex[i] * ey[j] : 0.0f;
                        float* c = acc[4 * j + i];
                        c[0] += w;
                        c[1] = fmaf(w, rb.x, c[1]);
                        c[2] = fmaf(w, rb.y, c[2]);
                        c[3] = fmaf(w, rb.z, c[3]);
                        npairs += in;
                    }
            }
        };

        // Two queues: records covering the whole block (ring 0) and the others
        // (ring 1), so that each batch of 32 takes one path for the whole warp.
        uint32_t wr0 = 0, rd0 = 0, wr1 = 0, rd1 = 0;
        float4* ring0 = ring;
        float4* ring1 = ring + 2 * kRing;
        auto stream = [&](const float4 ra, const float4 rb, const bool valid) {
            bool ov = false, full = false;
            if (valid) {
                const float dl = fmaxf(fmaxf(bxl - ra.x, ra.x - bxh), 0.0f);
                const float dm = fmaxf(fmaxf(byl - ra.y, ra.y - byh), 0.0f);
                ov = dl * dl + dm * dm <= rb.w * 1.0009765625f;
                // the computed r^2 grows with |dx| and |dy| (each rounding is monotone):
                // if the farthest cell passes the single-precision test, every cell does
                const float dxe = fmaxf(fabsf(__fsub_rn(xc[0], ra.x)), fabsf(__fsub_rn(xc[3], ra.x)));
                const float dye = fmaxf(fabsf(__fsub_rn(yc[0], ra.y)), fabsf(__fsub_rn(yc[3], ra.y)));
                full = ov && __fmaf_rn(dye, dye, __fmul_rn(dxe, dxe)) <= rb.w;
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, full);
            const unsigned m1 = __ballot_sync(0xffffffffu, ov && !full);
            if (full) {
                const uint32_t slot = (wr0 + __popc(m0 & lt)) & (kRing - 1);
                ring0[2 * slot] = ra;
                ring0[2 * slot + 1] = rb;
            } else if (ov) {
                const uint32_t slot = (wr1 + __popc(m1 & lt)) & (kRing - 1);
                ring1[2 * slot] = ra;
                ring1[2 * slot + 1] = rb;
            }
            wr0 += __popc(m0);
            wr1 += __popc(m1);
            __syncwarp();
            if (wr0 - rd0 >= 32) {
                const uint32_t slot = (rd0 + lane) & (kRing - 1);
                eval(ring0[2 * slot], ring0[2 * slot + 1], true);
                rd0 += 32;
                __syncwarp();
            }
            if (wr1 - rd1 >= 32) {
                const uint32_t slot = (rd1 + lane) & (kRing - 1);
                eval(ring1[2 * slot], ring1[2 * slot + 1], false);
                rd1 += 32;
                __syncwarp();
            }
        };

        // Row segments, 32 rows at a time: lane l reads the bin offsets of row l so
        // that the offsets of all rows arrive together.  Rows before this block's
        // window enter only through the scan of the row lengths (the item's
        // candidate offsets); rows after it end the walk.
        uint32_t offset = 0;
        for (int yg = ylo; yg <= yhi && yg <= wyhi && offset < c1; yg += 32) {
            const int yl = yg + lane;
            uint32_t beg = 0, len = 0, wb = 0, we = 0;
            if (yl <= yhi) {
                const int64_t rowb = (int64_t)yl * N;
                beg = __ldg(a.bin_start + rowb + xlo);
                len = __ldg(a.bin_start + rowb + xhi + 1) - beg;
                if (wxlo <= wxhi) {
                    wb = __ldg(a.bin_start + rowb + wxlo);
                    we = __ldg(a.bin_start + rowb + wxhi + 1);
                }
            }
            uint32_t incl = len;   // inclusive scan of the row lengths across lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int nrows = min(32, yhi - yg + 1);
            const int r1 = min(nrows, wyhi - yg + 1);
            for (int r = live ? max(0, wylo - yg) : r1; r < r1; ++r) {
                const uint32_t rbeg = __shfl_sync(0xffffffffu, beg, r);
                const uint32_t rlen = __shfl_sync(0xffffffffu, len, r);
                const uint32_t rwb = __shfl_sync(0xffffffffu, wb, r);
                const uint32_t rwe = __shfl_sync(0xffffffffu, we, r);
                const uint32_t roff = offset + __shfl_sync(0xffffffffu, incl, r) - rlen;
                if (roff >= c1) break;
                const int y = yg + r;
                if (!live || y < wylo || y > wyhi || roff + rlen <= c0 || wxlo > wxhi) continue;
                const uint32_t s0 = max(rbeg + (c0 > roff ? c0 - roff : 0u), rwb);
                const uint32_t e = min(rbeg + min(c1 - roff, rlen), rwe);
                // stream the segment 32 records at a time, loading one batch ahead
                float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
                if (s0 + lane < e) {
                    ra = __ldg(a.rec + 2 * (int64_t)(s0 + lane));
                    rb = __ldg(a.rec + 2 * (int64_t)(s0 + lane) + 1);
                }
                for (uint32_t j0 = s0; j0 < e; j0 += 32) {
                    const uint32_t jn = j0 + 32 + lane;
                    float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
                    if (jn < e) {
                        na = __ldg(a.rec + 2 * (int64_t)jn);
                        nb = __ldg(a.rec + 2 * (int64_t)jn + 1);
                    }
                    stream(ra, rb, j0 + lane < e);
                    ra = na;
                    rb = nb;
                }
            }
            offset += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (live && lane < wr0 - rd0) {
            const uint32_t slot = (rd0 + lane) & (kRing - 1);
            eval(ring0[2 * slot], ring0[2 * slot + 1], true);
        }
        if (live && lane < wr1 - rd1) {
            const uint32_t slot = (rd1 + lane) & (kRing - 1);
            eval(ring1[2 * slot], ring1[2 * slot + 1], false);
        }
        __syncwarp();

        // combine the 32 lane partials of each value, 32 values at a time through
        // the warp's scratch (rows padded to 33): four running sums over lanes
        // l = 0, 4, 8, ... / 1, 5, 9, ... in lane order, then (s0 + s1) + (s2 + s3).
        // The order is fixed, and the rounding (at most 31 u of the sum of the
        // partials' magnitudes) is far below that of a lane's own plain sum.
        float* scr = reinterpret_cast<float*>(ring);
        float4* out = a.temp + (int64_t)item * (kTile * kTile);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
            for (int v = 0; v < 32; ++v) scr[lane * 33 + v] = acc[(32 * half + v) >> 2][v & 3];
            __syncwarp();
            float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int l = 0; l < 32; ++l) s4[l & 3] += scr[l * 33 + lane];
            __syncwarp();
            const int f = 32 * half + lane;      // value f of the block: cell f/4, component f%4
            const int k = f >> 2;
            const int local = (4 * (blk & 3) + (k & 3)) + kTile * (4 * (blk >> 2) + (k >> 2));
            reinterpret_cast<float*>(out + local)[f & 3] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
        __syncwarp();
    }
    // pairs inside the truncation (cells of partial blocks at the mesh edge included):
    // one atomic per warp
    const unsigned wsum = __reduce_add_sync(0xffffffffu, npairs);
    if (lane == 0 && wsum) atomicAdd(a.pairs, (unsigned long long)wsum);
}

struct CombineArgs {
    const float4* temp;
    const uint32_t* tile_items;
    int N, tiles_x;
    float scale;
    float* s_mass;
    float* s_mom;
    float* dsum;
};

// Sum a cell's work-item partials in item order (compensated) and divide.
__global__ void __launch_bounds__(256) k_combine2d(CombineArgs a)
{
    pdl_entry();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int N = a.N;
    const int64_t nc = (int64_t)N * N;
    if (c >= nc) return;
    const int cx = (int)(c % N), cy = (int)(c / N);
    const int t = (cy / kTile) * a.tiles_x + cx / kTile;
    const int local = (cx % kTile) + kTile * (cy % kTile);
    const uint32_t i0 = __ldg(a.tile_items + t), i1 = __ldg(a.tile_items + t + 1);
    float s[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    for (uint32_t it = i0; it < i1; ++it) {
        const float4 v = __ldg(a.temp + (int64_t)it * (kTile * kTile) + local);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float tt = s[q] + vv[q];
            if (fabsf(s[q]) >= fabsf(vv[q])) cmp[q] += (s[q] - tt) + vv[q];
            else cmp[q] += (vv[q] - tt) + s[q];
            s[q] = tt;
        }
    }
    const float D = s[0] + cmp[0];
    const bool cov = D > 0.0f;
    a.s_mass[c] = cov ? -(s[1] + cmp[1]) / D * a.scale : 0.0f;
    a.s_mom[c] = cov ? -(s[2] + cmp[2]) / D * a.scale : 0.0f;
    a.s_mom[nc + c] = cov ? -(s[3] + cmp[3]) / D * a.scale : 0.0f;
    if (a.dsum) a.dsum[c] = D;
}

}  // namespace

int gather2d_tiles(int N) { return ((N + kTile - 1) / kTile) * ((N + kTile - 1) / kTile); }

uint32_t gather2d_item_budget(int N, int64_t n)
{
    return (uint32_t)(gather2d_tiles(N) + (16 * (n > 0 ? n : 1) + kChunk - 1) / kChunk + 1);
}

size_t gather2d_temp_bytes(int N, int64_t n) { return (size_t)gather2d_item_budget(N, n) * kTile * kTile * 16; }

cudaError_t launch_gather2d(const fla_mesh& m, const fla_deposit_cfg& cfg, const void* rec, const uint32_t* bin_start,
                            const unsigned int* ext_max, uint32_t* tile_cand, uint32_t* tile_items,
                            unsigned int* counter, void* temp, uint32_t budget, const fla_sources& out,
                            DevStatus* st, int num_sms, cudaStream_t s)
{
    const int N = m.n;
    const int tiles_x = (N + kTile - 1) / kTile;
    const int n_tiles = tiles_x * tiles_x;
    PlanArgs p{bin_start, ext_max, tile_cand, tile_items, N, tiles_x, n_tiles, budget, counter + 1};
    // the gather's unit counter and the plan's CTA counter are zero on entry
    cudaError_t e = launch_pdl(k_plan2d, dim3((unsigned)((n_tiles * 32 + 255) / 256)), dim3(256), 0, s, p);
    if (e != cudaSuccess) return e;
    G2Args g{};
    g.rec = (const float4*)rec;
    g.bin_start = bin_start;
    g.ext_max = ext_max;
    g.tile_cand = tile_cand;
    g.tile_items = tile_items;
    g.counter = counter;
    g.temp = (float4*)temp;
    g.pairs = &st->pairs;
    g.N = N;
    g.tiles_x = tiles_x;
    g.n_tiles = n_tiles;
    const size_t smem = (size_t)kWarps * (kScratchFloats / 4 + 8) * sizeof(float4);
    static bool attr_set = false;   // set once, before any stream capture that uses it
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_gather2d_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    launch_pdl(k_gather2d_items, dim3(num_sms), dim3(kThreads), smem, s, g);
    CombineArgs c{};
    c.temp = (const float4*)temp;
    c.tile_items = tile_items;
    c.N = N;
    c.tiles_x = tiles_x;
    const double dx = 1.0 / N;
    c.scale = cfg.per_cell ? (float)(dx * dx) : 1.0f;
    c.s_mass = (float*)out.s_mass_dev;
    c.s_mom = (float*)out.s_mom_dev;
    c.dsum = (float*)out.dsum_dev;
    const int64_t nc = (int64_t)N * N;
    launch_pdl(k_combine2d, dim3((unsigned)((nc + 255) / 256)), dim3(256), 0, s, c);
    return cudaGetLastError();
}

}  // namespace fla
