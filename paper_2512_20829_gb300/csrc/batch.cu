// Batched clouds: plan (device tables in the caller's workspace), one window
// of batched launches, the autotuner and the CUDA graph of several windows.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "batch.cuh"

using namespace fla;

// The persistent window kernel (window.cu, its own compilation of the phases).
extern "C" int fla_window_prepare(void);
extern "C" int fla_window_issue(const void* batch_dev, const void* bin_work, uint32_t* bin_start, void* status,
                                double dt, int window, int64_t n2, int64_t n3, int stall, uint32_t chunk,
                                void* stream);

struct fla_batch_plan {
    BatchDev dev;                       // device tables (pointers into the workspace)
    std::vector<BatchCloud> host;       // host copy of the cloud table
    int n_clouds = 0;
    double dt = 0.0;
    int window = 0;
    int64_t n_dim[2] = {0, 0};          // droplets of the 2D and 3D clouds
    BinPlan bins{};
    BinWork sort{};
    uint32_t* bin_start = nullptr;
    const BatchTile* tiles_order[2][kBatchGroups] = {};   // natural, interleaved
    // tuning
    int advance_threads = 128;
    int gather_ctas_per_sm = 2;
    int tile_order = 0;
    bool tuned = false;
    int mode = FLA_BATCH_AUTO;          // requested window execution
    int persistent = 0;                 // in use: one cooperative kernel per window
    bool persistent_ok = false;         // the window kernel fits the device
    float timed_ms[2] = {0.0f, 0.0f};   // the tuner's window: persistent, launches
    // graph of graph_windows windows
    cudaGraphExec_t exec = nullptr;
    int graph_windows = 0;
    int num_sms = 1;
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BatchLayout {
    size_t clouds, drop_pre, node_pre, misc, ext, cargs, tiles[2][kBatchGroups], keys[2], vals[2], scratch,
        bin_start, rec[kBatchGroups], tile_cand[kBatchGroups], tile_items[kBatchGroups], cloud_cand,
        item_temp[kBatchGroups], total;
    int64_t n_total, cells_total, nodes_total, group_drops[kBatchGroups], group_items[kBatchGroups];
    int n_tiles[kBatchGroups];
};

int64_t cells_of_mesh(const fla_mesh& m) { return m.dim == 2 ? (int64_t)m.n * m.n : (int64_t)m.n * m.n * m.n; }
int64_t nodes_of_mesh(const fla_mesh& m)
{
    const int64_t nn = m.n + 1;
    return m.dim == 2 ? nn * nn : nn * nn * nn;
}
int tiles_of_mesh(const fla_mesh& m)
{
    // tile shapes of the gather: 16 x 16 (2D), 8 x 8 x 4 (3D)
    if (m.dim == 2) return ((m.n + 15) / 16) * ((m.n + 15) / 16);
    return ((m.n + 7) / 8) * ((m.n + 7) / 8) * ((m.n + 3) / 4);
}

int item_ok(const fla_batch_item& it)
{
    const fla_cloud& c = it.cloud;
    const fla_mesh& m = it.mesh;
    if ((m.dim != 2 && m.dim != 3) || m.n < 1 || m.n > 1024) return FLA_ERR_ARG;
    if (c.kind != FLA_CLOUD_FLA || c.dtype != FLA_F32 || c.dim != m.dim || c.fold_dev) return FLA_ERR_ARG;
    if (c.n < 0 || c.n >= 2147483647LL) return FLA_ERR_ARG;
    if (c.n > 0 && (!c.state_dev || !c.meta_dev || !c.batches_dev || c.n_batches < 1 ||
                    ((uintptr_t)c.state_dev % 16) != 0))
        return FLA_ERR_ARG;
    if (!it.nodes_dev || ((uintptr_t)it.nodes_dev % 16) != 0) return FLA_ERR_ARG;
    if (it.carrier.dim != m.dim || it.carrier.n_vortex < 0 || it.carrier.n_vortex > FLA_MAX_VORTICES)
        return FLA_ERR_ARG;
    const fla_deposit_cfg& g = it.cfg;
    if (g.kernel != FLA_KERNEL_ISO && g.kernel != FLA_KERNEL_ANISO) return FLA_ERR_ARG;
    if (!(g.h_min > 0) || !(g.h_max >= g.h_min) || !(g.window_dt > 0) || !(g.p > 0)) return FLA_ERR_ARG;
    if (g.kernel == FLA_KERNEL_ANISO && !(g.h_max * g.h_max > m.dim * g.h_min * g.h_min)) return FLA_ERR_ARG;
    if (g.mlp_dev) return FLA_ERR_UNSUPPORTED;
    if (g.precision != FLA_PREC_MIXED && g.precision != FLA_PREC_PLAIN) return FLA_ERR_ARG;
    if (g.h_max * m.n > 64.0) return FLA_ERR_UNSUPPORTED;
    if (!it.out.s_mass_dev || !it.out.s_mom_dev) return FLA_ERR_ARG;
    return FLA_OK;
}

// clouds in group order (dim, kernel), stable within a group
std::vector<int> group_order(const fla_batch_item* items, int n)
{
    std::vector<int> ord(n);
    for (int k = 0; k < n; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        return batch_group(items[a].mesh.dim, items[a].cfg.kernel) < batch_group(items[b].mesh.dim, items[b].cfg.kernel);
    });
    return ord;
}

BatchLayout batch_layout(const fla_batch_item* items, int n)
{
    BatchLayout L{};
    for (int k = 0; k < n; ++k) {
        const int g = batch_group(items[k].mesh.dim, items[k].cfg.kernel);
        L.n_total += items[k].cloud.n;
        L.cells_total += cells_of_mesh(items[k].mesh);
        L.nodes_total += nodes_of_mesh(items[k].mesh);
        L.group_drops[g] += items[k].cloud.n;
        L.n_tiles[g] += tiles_of_mesh(items[k].mesh);
        L.group_items[g] += nw_item_budget(items[k].mesh.dim, items[k].mesh.n, items[k].cloud.n, 4);
    }
    const size_t nn = (size_t)(L.n_total > 0 ? L.n_total : 1);
    size_t o = 0;
    L.clouds = o; o += up256(sizeof(BatchCloud) * (size_t)n);
    L.drop_pre = o; o += up256(8 * (size_t)(n + 1));
    L.node_pre = o; o += up256(8 * (size_t)(n + 1));
    L.misc = o; o += 256;                                  // step, tile counters
    L.ext = o; o += up256(4 * (size_t)n);
    L.cargs = o; o += up256(batch_carrier_args_bytes() * (size_t)n);
    for (int r = 0; r < 2; ++r)
        for (int g = 0; g < kBatchGroups; ++g) { L.tiles[r][g] = o; o += up256(sizeof(BatchTile) * (size_t)L.n_tiles[g]); }
    for (int b = 0; b < 2; ++b) { L.keys[b] = o; o += up256(nn * 4); }
    for (int b = 0; b < 2; ++b) { L.vals[b] = o; o += up256(nn * 4); }
    L.scratch = o; o += up256(bin_plan(L.n_total, L.cells_total).scratch_bytes);
    L.bin_start = o; o += up256(((size_t)L.cells_total + 1) * 4);
    for (int g = 0; g < kBatchGroups; ++g) {
        const int rv = record_values(g < 2 ? 2 : 3, g & 1);
        L.rec[g] = o;
        o += up256((size_t)L.group_drops[g] * rv * 4);
    }
    for (int g = 0; g < kBatchGroups; ++g) {
        L.tile_cand[g] = o; o += up256(4 * (size_t)L.n_tiles[g]);
        L.tile_items[g] = o; o += up256(4 * ((size_t)L.n_tiles[g] + 1));
    }
    L.cloud_cand = o; o += up256(8 * (size_t)n);
    // item partials, one region per group: the persistent window kernel runs
    // the groups' work items in one phase
    for (int g = 0; g < kBatchGroups; ++g) {
        const int dim = g < 2 ? 2 : 3;
        L.item_temp[g] = o; o += up256((size_t)L.group_items[g] * (size_t)(dim + 2) * 256 * 4);
    }
    L.total = o;
    return L;
}

template <typename P>
P* at(void* base, size_t off) { return reinterpret_cast<P*>(static_cast<char*>(base) + off); }

}  // namespace

namespace {

// The parts of one window of every cloud: carrier sample and advance (acc
// reset); keys, sort, bin starts and records; the gathers; the step counter.
int issue_advance(fla_ctx* ctx, fla_batch_plan* p, int threads, cudaStream_t s)
{
    BatchDev& b = p->dev;
    if (launch_batch_carrier(b, p->dt, s) != cudaSuccess) return FLA_ERR_CUDA;
    for (int d = 0; d < 2; ++d)
        if (launch_batch_advance(b, 2 + d, p->n_dim[d], p->window, p->dt, true, threads, (DevStatus*)ctx->status_dev,
                                 s) != cudaSuccess)
            return FLA_ERR_CUDA;
    return FLA_OK;
}

int issue_records(fla_ctx* ctx, fla_batch_plan* p, cudaStream_t s)
{
    BatchDev& b = p->dev;
    if (b.n_total > 0) {
        if (launch_batch_binning(b, p->sort, p->bin_start, (DevStatus*)ctx->status_dev, s) != cudaSuccess)
            return FLA_ERR_CUDA;
        b.perm = p->sort.vals[bin_sorted_buffer(p->bins)];
    } else if (cudaMemsetAsync(p->bin_start, 0, ((size_t)b.cells_total + 1) * 4, s) != cudaSuccess) {
        return FLA_ERR_CUDA;
    }
    for (int g = 0; g < kBatchGroups; ++g)
        if (b.group_first[g + 1] > b.group_first[g] &&
            launch_batch_records(b, g, (DevStatus*)ctx->status_dev, s) != cudaSuccess)
            return FLA_ERR_CUDA;
    return FLA_OK;
}

int issue_gathers(fla_ctx* ctx, fla_batch_plan* p, int ctas_per_sm, int order, cudaStream_t s)
{
    BatchDev& b = p->dev;
    for (int g = 0; g < kBatchGroups; ++g) b.tiles[g] = p->tiles_order[order][g];
    for (int g = 0; g < kBatchGroups; ++g)
        if (launch_batch_gather(b, g, ctas_per_sm * p->num_sms, (DevStatus*)ctx->status_dev, p->num_sms, s) !=
            cudaSuccess)
            return FLA_ERR_CUDA;
    return FLA_OK;
}

// One window as the persistent kernel (a memset of its barrier words, one
// cooperative launch).
int issue_persistent(fla_ctx* ctx, fla_batch_plan* p, cudaStream_t s)
{
    BatchDev& b = p->dev;
    for (int g = 0; g < kBatchGroups; ++g) b.tiles[g] = p->tiles_order[p->tile_order][g];
    b.perm = p->sort.vals[bin_sorted_buffer(p->bins)];
    const int stall = (ctx->stall & FLA_STALL_BATCH_WINDOW) != 0;
    ctx->stall &= ~FLA_STALL_BATCH_WINDOW;
    return fla_window_issue(&b, &p->sort, p->bin_start, ctx->status_dev, p->dt, p->window, p->n_dim[0],
                            p->n_dim[1], stall, nw_chunk(4), s) == (int)cudaSuccess
               ? FLA_OK
               : FLA_ERR_CUDA;
}

int issue_window(fla_ctx* ctx, fla_batch_plan* p, cudaStream_t s)
{
    if (p->persistent) return issue_persistent(ctx, p, s);
    int st = issue_advance(ctx, p, p->advance_threads, s);
    if (st == FLA_OK) st = issue_records(ctx, p, s);
    if (st == FLA_OK) st = issue_gathers(ctx, p, p->gather_ctas_per_sm, p->tile_order, s);
    if (st == FLA_OK && launch_batch_step(p->dev, p->window, s) != cudaSuccess) st = FLA_ERR_CUDA;
    return st;
}

// Kernel launches of one window (for the caller's launch accounting).
int window_launches(const fla_batch_plan* p)
{
    if (p->persistent) return 1;
    int n = 2 + (p->n_dim[0] > 0) + (p->n_dim[1] > 0) + 1;   // carrier (2), advance, step
    if (p->dev.n_total > 0) n += 1;   // keys, sort and bin starts: one kernel
    for (int g = 0; g < kBatchGroups; ++g) {
        if (p->dev.group_first[g + 1] > p->dev.group_first[g]) n += 1;
        if (p->dev.n_tiles[g] > 0) n += 3;   // gather plan, items, combine
    }
    return n;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~EventPair() { cudaEventDestroy(a); cudaEventDestroy(b); }
    float ms() const
    {
        float t = 1e30f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) return 1e30f;
        return t;
    }
};

// Autotuning on the first windows of a run.  Every knob leaves the results
// unchanged: the advance's block size (droplets are independent), the number
// of persistent gather CTAs and the order of the tile table (a tile's work
// items depend only on its candidates, each is computed whole by one CTA, and
// the items of a tile are combined in their own order).  Window w < 3 advances with 64 << w threads per
// block and times it; the first window also times the gathers for each
// (CTAs per SM, order) pair by repeating them, which rewrites the same
// outputs.  Returns the windows issued, or -1.
int tune(fla_ctx* ctx, fla_batch_plan* p, int n_windows, cudaStream_t s)
{
    static const int kThreads[3] = {64, 128, 256};
    static const int kCtas[3] = {1, 2, 4};
    EventPair ev;
    float best_adv = 1e30f;
    int used = 0;
    for (int w = 0; w < 3 && w < n_windows; ++w) {
        cudaEventRecord(ev.a, s);
        if (issue_advance(ctx, p, kThreads[w], s) != FLA_OK) return -1;
        cudaEventRecord(ev.b, s);
        const float ta = ev.ms();
        if (ta < best_adv) {
            best_adv = ta;
            p->advance_threads = kThreads[w];
        }
        if (issue_records(ctx, p, s) != FLA_OK) return -1;
        if (w == 0) {
            float best = 1e30f;
            for (int o = 0; o < 2; ++o)
                for (int c = 0; c < 3; ++c) {
                    cudaEventRecord(ev.a, s);
                    if (issue_gathers(ctx, p, kCtas[c], o, s) != FLA_OK) return -1;
                    cudaEventRecord(ev.b, s);
                    const float tg = ev.ms();
                    if (tg < best) {
                        best = tg;
                        p->gather_ctas_per_sm = kCtas[c];
                        p->tile_order = o;
                    }
                }
        }
        if (issue_gathers(ctx, p, p->gather_ctas_per_sm, p->tile_order, s) != FLA_OK) return -1;
        if (launch_batch_step(p->dev, p->window, s) != cudaSuccess) return -1;
        ++used;
    }
    // then one whole window as the persistent kernel and one as launches
    if (p->mode == FLA_BATCH_AUTO && p->persistent_ok && n_windows - used >= 2) {
        float t[2];
        for (int m = 0; m < 2; ++m) {
            p->persistent = m == 0;
            cudaEventRecord(ev.a, s);
            if (issue_window(ctx, p, s) != FLA_OK) return -1;
            cudaEventRecord(ev.b, s);
            t[m] = ev.ms();
            ++used;
        }
        p->persistent = t[0] < t[1];
        p->timed_ms[0] = t[0];
        p->timed_ms[1] = t[1];
    } else {
        p->persistent = p->mode == FLA_BATCH_PERSISTENT && p->persistent_ok;
    }
    return used;
}

}  // namespace

extern "C" int fla_batch_workspace_size(const fla_batch_item* items, int32_t n_items, size_t* bytes)
{
    if (!items || !bytes || n_items < 1 || n_items > 65536) return FLA_ERR_ARG;
    for (int k = 0; k < n_items; ++k) {
        const int st = item_ok(items[k]);
        if (st != FLA_OK) return st;
    }
    const BatchLayout L = batch_layout(items, n_items);
    if (L.n_total >= 2147483647LL || L.cells_total >= 2147483647LL) return FLA_ERR_UNSUPPORTED;
    *bytes = L.total;
    return FLA_OK;
}

extern "C" int fla_batch_create(fla_ctx* ctx, const fla_batch_item* items, int32_t n_items, double dt,
                                int32_t window_steps, int32_t step0, void* ws, size_t ws_bytes,
                                fla_batch_plan** out)
{
    if (!ctx || !out || !(dt > 0) || window_steps < 1 || step0 < 0) return FLA_ERR_ARG;
    size_t need = 0;
    int st = fla_batch_workspace_size(items, n_items, &need);
    if (st != FLA_OK) return st;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FLA_ERR_WORKSPACE;
    const BatchLayout L = batch_layout(items, n_items);
    if (batch_prepare_gathers() != cudaSuccess || batch_prepare_advance() != cudaSuccess) return FLA_ERR_CUDA;
    const bool persistent_ok = fla_window_prepare() > 0;
    fla_batch_plan* p = new (std::nothrow) fla_batch_plan();
    if (!p) return FLA_ERR_ARG;
    p->n_clouds = n_items;
    p->dt = dt;
    p->window = window_steps;
    p->num_sms = ctx->num_sms > 0 ? ctx->num_sms : 1;
    const std::vector<int> ord = group_order(items, n_items);
    std::vector<int64_t> drop_pre(n_items + 1, 0), node_pre(n_items + 1, 0);
    p->host.resize(n_items);
    BatchDev& b = p->dev;
    int64_t cell = 0;
    for (int g = 0; g <= kBatchGroups; ++g) b.group_first[g] = 0;
    for (int idx = 0; idx < n_items; ++idx) {
        const fla_batch_item& it = items[ord[idx]];
        BatchCloud& c = p->host[idx];
        memset(&c, 0, sizeof(c));
        c.dim = it.mesh.dim;
        c.kernel = it.cfg.kernel;
        c.N = it.mesh.n;
        c.per_cell = it.cfg.per_cell ? 1 : 0;
        c.n_batches = it.cloud.n_batches;
        c.plain = it.cfg.precision == FLA_PREC_PLAIN ? 1 : 0;
        c.group = batch_group(c.dim, c.kernel);
        c.n = it.cloud.n;
        c.drop_off = drop_pre[idx];
        c.n_cells = cells_of_mesh(it.mesh);
        c.cell_off = cell;
        c.n_nodes = nodes_of_mesh(it.mesh);
        c.node_off = node_pre[idx];
        c.state = (float*)it.cloud.state_dev;
        c.meta = it.cloud.meta_dev;
        c.batches = it.cloud.batches_dev;
        c.nodes = (float*)it.nodes_dev;
        c.s_mass = (float*)it.out.s_mass_dev;
        c.s_mom = (float*)it.out.s_mom_dev;
        c.dsum = (float*)it.out.dsum_dev;
        c.delta = it.cloud.delta;
        c.h_min = it.cfg.h_min;
        c.h_max = it.cfg.h_max;
        c.p = it.cfg.p;
        c.window_dt = it.cfg.window_dt;
        c.car = it.carrier;
        drop_pre[idx + 1] = drop_pre[idx] + c.n;
        node_pre[idx + 1] = node_pre[idx] + c.n_nodes;
        cell += c.n_cells;
        b.group_first[c.group + 1] += 1;
        p->n_dim[c.dim - 2] += c.n;
    }
    for (int g = 0; g < kBatchGroups; ++g) b.group_first[g + 1] += b.group_first[g];
    b.group_cells[0] = 0;
    for (int g = 0; g < kBatchGroups; ++g) {
        int64_t cg = 0;
        for (int k = b.group_first[g]; k < b.group_first[g + 1]; ++k) cg += p->host[k].n_cells;
        b.group_cells[g + 1] = b.group_cells[g] + cg;
        b.group_drops[g] = L.group_drops[g];
        b.n_tiles[g] = L.n_tiles[g];
    }
    // gather tiles per group: natural (cloud by cloud) and interleaved (round robin over the clouds)
    std::vector<BatchTile> nat[kBatchGroups], inter[kBatchGroups];
    for (int g = 0; g < kBatchGroups; ++g) {
        std::vector<std::vector<BatchTile>> per;
        for (int k = b.group_first[g]; k < b.group_first[g + 1]; ++k) {
            const BatchCloud& c = p->host[k];
            const int tx = c.dim == 2 ? 16 : 8, ty = c.dim == 2 ? 16 : 8, tz = c.dim == 2 ? 1 : 4;
            std::vector<BatchTile> v;
            for (int z = 0; z < (c.dim == 2 ? 1 : (c.N + tz - 1) / tz); ++z)
                for (int y = 0; y < (c.N + ty - 1) / ty; ++y)
                    for (int x = 0; x < (c.N + tx - 1) / tx; ++x) v.push_back(BatchTile{k, x * tx, y * ty, z * tz});
            nat[g].insert(nat[g].end(), v.begin(), v.end());
            per.push_back(v);
        }
        size_t longest = 0;
        for (auto& v : per) longest = std::max(longest, v.size());
        for (size_t t = 0; t < longest; ++t)
            for (auto& v : per)
                if (t < v.size()) inter[g].push_back(v[t]);
    }
    // device tables
    bool ok = cudaMemcpy(at<void>(ws, L.clouds), p->host.data(), sizeof(BatchCloud) * n_items,
                         cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(at<void>(ws, L.drop_pre), drop_pre.data(), 8 * (n_items + 1), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy(at<void>(ws, L.node_pre), node_pre.data(), 8 * (n_items + 1), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    for (int g = 0; g < kBatchGroups && ok; ++g) {
        if (nat[g].empty()) continue;
        ok = cudaMemcpy(at<void>(ws, L.tiles[0][g]), nat[g].data(), sizeof(BatchTile) * nat[g].size(),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(at<void>(ws, L.tiles[1][g]), inter[g].data(), sizeof(BatchTile) * inter[g].size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    int misc[64] = {0};
    misc[0] = step0;
    ok = ok && cudaMemcpy(at<void>(ws, L.misc), misc, sizeof(misc), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(at<void>(ws, L.cloud_cand), 0, 8 * (size_t)n_items) == cudaSuccess;
    if (!ok) {
        delete p;
        return FLA_ERR_CUDA;
    }
    b.clouds = at<BatchCloud>(ws, L.clouds);
    b.n_clouds = n_items;
    b.n_total = L.n_total;
    b.cells_total = L.cells_total;
    b.nodes_total = L.nodes_total;
    b.drop_pre = at<int64_t>(ws, L.drop_pre);
    b.node_pre = at<int64_t>(ws, L.node_pre);
    b.step = at<int>(ws, L.misc);
    b.tile_counter = at<unsigned int>(ws, L.misc + 16);
    b.plan_done = at<unsigned int>(ws, L.misc + 32);
    b.cloud_cand = at<unsigned long long>(ws, L.cloud_cand);
    for (int g = 0; g < kBatchGroups; ++g) b.item_temp[g] = at<void>(ws, L.item_temp[g]);
    b.ext_max = at<unsigned int>(ws, L.ext);
    b.cargs = at<void>(ws, L.cargs);
    for (int r = 0; r < 2; ++r)
        for (int g = 0; g < kBatchGroups; ++g) p->tiles_order[r][g] = at<BatchTile>(ws, L.tiles[r][g]);
    for (int g = 0; g < kBatchGroups; ++g) {
        b.tiles[g] = p->tiles_order[0][g];
        b.rec[g] = at<void>(ws, L.rec[g]);
        b.tile_cand[g] = at<uint32_t>(ws, L.tile_cand[g]);
        b.tile_items[g] = at<uint32_t>(ws, L.tile_items[g]);
    }
    for (int k = 0; k < 2; ++k) {
        p->sort.keys[k] = at<uint32_t>(ws, L.keys[k]);
        p->sort.vals[k] = at<uint32_t>(ws, L.vals[k]);
    }
    p->sort.scratch = at<void>(ws, L.scratch);
    p->bin_start = at<uint32_t>(ws, L.bin_start);
    b.bin_start = p->bin_start;
    p->bins = bin_plan(L.n_total, L.cells_total);
    b.perm = p->sort.vals[bin_sorted_buffer(p->bins)];   // the same buffer every window
    p->persistent_ok = persistent_ok;
    *out = p;
    return FLA_OK;
}

extern "C" void fla_batch_destroy(fla_batch_plan* plan)
{
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    delete plan;
}

extern "C" int fla_batch_set_step(fla_batch_plan* plan, int32_t step, fla_stream_t stream)
{
    if (!plan || step < 0) return FLA_ERR_ARG;
    // step[1] = 0: the workspace's binning is not this run's (the next window
    // advances in seed order)
    static thread_local int host_step[2];   // pageable source: the copy is staged at the call
    host_step[0] = step;
    host_step[1] = 0;
    return cudaMemcpyAsync(plan->dev.step, host_step, sizeof(host_step), cudaMemcpyHostToDevice,
                           (cudaStream_t)stream) ==
                   cudaSuccess
               ? FLA_OK
               : FLA_ERR_CUDA;
}

extern "C" int fla_batch_tuning(const fla_batch_plan* plan, int32_t* advance_threads, int32_t* gather_ctas_per_sm,
                                int32_t* tile_order, int32_t* launches_per_window)
{
    if (!plan) return FLA_ERR_ARG;
    if (advance_threads) *advance_threads = plan->advance_threads;
    if (gather_ctas_per_sm) *gather_ctas_per_sm = plan->gather_ctas_per_sm;
    if (tile_order) *tile_order = plan->tile_order;
    if (launches_per_window) *launches_per_window = window_launches(plan);
    return plan->tuned ? FLA_OK : FLA_ERR_UNSUPPORTED;
}

extern "C" int fla_batch_set_tuning(fla_batch_plan* plan, int32_t advance_threads, int32_t gather_ctas_per_sm,
                                    int32_t tile_order)
{
    if (!plan || (advance_threads != 64 && advance_threads != 128 && advance_threads != 256) ||
        gather_ctas_per_sm < 1 || gather_ctas_per_sm > 8 || (tile_order != 0 && tile_order != 1))
        return FLA_ERR_ARG;
    plan->advance_threads = advance_threads;
    plan->gather_ctas_per_sm = gather_ctas_per_sm;
    plan->tile_order = tile_order;
    plan->tuned = true;
    if (plan->exec) {   // the graph holds the old launch shapes
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
        plan->graph_windows = 0;
    }
    return FLA_OK;
}

extern "C" int fla_batch_set_mode(fla_batch_plan* plan, int32_t mode)
{
    if (!plan || (mode != FLA_BATCH_AUTO && mode != FLA_BATCH_LAUNCHES && mode != FLA_BATCH_PERSISTENT))
        return FLA_ERR_ARG;
    if (mode == FLA_BATCH_PERSISTENT && !plan->persistent_ok) return FLA_ERR_UNSUPPORTED;
    plan->mode = mode;
    if (mode != FLA_BATCH_AUTO || plan->tuned) plan->persistent = mode == FLA_BATCH_PERSISTENT;
    if (plan->exec) {   // the graph holds the other form
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
        plan->graph_windows = 0;
    }
    return FLA_OK;
}

extern "C" int fla_batch_mode(const fla_batch_plan* plan, int32_t* mode, float* persistent_ms, float* launches_ms)
{
    if (!plan) return FLA_ERR_ARG;
    if (mode) *mode = plan->tuned || plan->mode != FLA_BATCH_AUTO
                          ? (plan->persistent ? FLA_BATCH_PERSISTENT : FLA_BATCH_LAUNCHES)
                          : FLA_BATCH_AUTO;
    if (persistent_ms) *persistent_ms = plan->timed_ms[0];
    if (launches_ms) *launches_ms = plan->timed_ms[1];
    return FLA_OK;
}

extern "C" int fla_batch_run(fla_ctx* ctx, fla_batch_plan* plan, int32_t n_windows, fla_stream_t stream)
{
    if (!ctx || !plan || n_windows < 0) return FLA_ERR_ARG;
    if (n_windows == 0) return FLA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return FLA_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone || s == nullptr) {
        // inside the caller's capture, or on the legacy stream: plain launches
        for (int w = 0; w < n_windows; ++w) {
            const int st = issue_window(ctx, plan, s);
            if (st != FLA_OK) return st;
        }
        return FLA_OK;
    }
    if (!plan->tuned) {
        const int used = tune(ctx, plan, n_windows, s);
        if (used < 0) return FLA_ERR_CUDA;
        plan->tuned = true;
        n_windows -= used;
        if (n_windows == 0) return FLA_OK;
    }
    if (!plan->exec || plan->graph_windows != n_windows) {
        if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
            plan->exec = nullptr;
        }
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FLA_ERR_CUDA;
        int st = FLA_OK;
        for (int w = 0; w < n_windows && st == FLA_OK; ++w) st = issue_window(ctx, plan, s);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st != FLA_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return st != FLA_OK ? st : FLA_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&plan->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            plan->exec = nullptr;
            return FLA_ERR_CUDA;
        }
        plan->graph_windows = n_windows;
    }
    return cudaGraphLaunch(plan->exec, s) == cudaSuccess ? FLA_OK : FLA_ERR_CUDA;
}
