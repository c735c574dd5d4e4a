// C-ABI entry points: argument validation, workspace carving and launches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "mlp_tc.cuh"

using namespace fla;

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int64_t cells_of(const fla_mesh& m)
{
    return m.dim == 2 ? (int64_t)m.n * m.n : (int64_t)m.n * m.n * m.n;
}

bool mesh_ok(const fla_mesh* m) { return fla::mesh_valid(m); }
int cloud_ok(const fla_cloud* c, const fla_mesh* m) { return fla::cloud_valid(c, m); }

bool dtype_ok(int32_t dtype) { return dtype == FLA_F32 || dtype == FLA_F64 || dtype == FLA_F32X2; }

}  // namespace

namespace fla {

bool mesh_valid(const fla_mesh* m)
{
    if (!m || (m->dim != 2 && m->dim != 3) || m->n < 1 || m->n > (1 << 20)) return false;
    const double nc = m->dim == 2 ? (double)m->n * m->n : (double)m->n * m->n * m->n;
    return nc < 2147483647.0;
}

int cloud_valid(const fla_cloud* c, const fla_mesh* m)
{
    if (!c || !mesh_valid(m)) return FLA_ERR_ARG;
    if (c->dim != m->dim || (c->dtype != FLA_F32 && c->dtype != FLA_F64 && c->dtype != FLA_F32X2))
        return FLA_ERR_ARG;
    if (c->kind != FLA_CLOUD_FLA && c->kind != FLA_CLOUD_LPT) return FLA_ERR_ARG;
    if (c->n < 0 || c->n >= 2147483647LL) return FLA_ERR_ARG;
    if (c->n > 0) {
        if (!c->state_dev || !c->meta_dev || !c->batches_dev || c->n_batches < 1) return FLA_ERR_ARG;
        if (!aligned(c->state_dev, 16) || !aligned(c->batches_dev, 8)) return FLA_ERR_ARG;
        if (c->n_batches > (int32_t)FLA_META_BATCH_MASK + 1) return FLA_ERR_ARG;
    }
    if (!isfinite(c->delta)) return FLA_ERR_ARG;
    if (c->fold_dev) {   // fold guard: single-precision FLA clouds only
        if (c->kind != FLA_CLOUD_FLA || c->dtype != FLA_F32 || !aligned(c->fold_dev, 16)) return FLA_ERR_ARG;
        if (!(c->tau_fold > 0) || !isfinite(c->tau_fold)) return FLA_ERR_ARG;
    }
    return FLA_OK;
}

}  // namespace fla

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
    size_t keys[2], vals[2], scratch, bin_start, misc, rec, tiles, temp, total;
};

// The load-balanced gather serves single-precision 2D clouds with the spherical kernel.
bool use_gather2d(const fla_mesh& m, int dtype, int kernel)
{
    return m.dim == 2 && dtype != FLA_F64 && kernel == FLA_KERNEL_ISO;
}

WsLayout layout(const fla_mesh& m, int dtype, int kernel, int64_t n)
{
    WsLayout L{};
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t T = dtype == FLA_F64 ? 8 : 4;
    const size_t rv = (size_t)record_values(m.dim, kernel);
    const size_t rec_bytes = nn * T * (rv > 4 ? rv : 4);
    size_t o = 0;
    for (int b = 0; b < 2; ++b) { L.keys[b] = o; o += up256(nn * 4); }
    for (int b = 0; b < 2; ++b) { L.vals[b] = o; o += up256(nn * 4); }
    L.scratch = o; o += up256(bin_plan(n, cells_of(m)).scratch_bytes);
    L.bin_start = o; o += up256(((size_t)cells_of(m) + 1) * 4);
    L.misc = o; o += 256;
    L.rec = o; o += up256(rec_bytes);
    L.tiles = o;
    L.temp = o;
    if (use_gather2d(m, dtype, kernel)) {
        o += up256((size_t)(2 * gather2d_tiles(m.n) + 1) * 4);
        L.temp = o;
        o += up256(gather2d_temp_bytes(m.n, n));
    } else {   // the tile gather's work items
        o += up256((size_t)(2 * nw_tiles(m.dim, m.n) + 1) * 4);
        L.temp = o;
        o += up256(nw_temp_bytes(m.dim, m.n, n, T));
    }
    L.total = o;
    return L;
}

// Which of the sort's ping-pong buffers holds the sorted order of a cloud of n.
int sorted_buffer(const fla_mesh& m, int64_t n) { return bin_sorted_buffer(bin_plan(n, cells_of(m))); }

template <typename P>
P* at(void* base, size_t off) { return reinterpret_cast<P*>(static_cast<char*>(base) + off); }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FLA_OK : FLA_ERR_CUDA; }

// Counts a phase's launches and, with timing on, brackets it with CUDA events.
struct PhaseScope {
    fla_ctx* c;
    int ph;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(fla_ctx* ctx, int phase, cudaStream_t stream, int n_launch) : c(ctx), ph(phase), s(stream)
    {
        c->calls[ph] += 1;
        c->launches[ph] += n_launch;
        if (c->timing) {
            a = take();
            if (a && cudaEventRecord(a, s) != cudaSuccess) a = nullptr;
        }
    }
    ~PhaseScope()
    {
        if (!a) return;
        cudaEvent_t b = take();
        if (b && cudaEventRecord(b, s) == cudaSuccess) c->pending.push_back({ph, a, b});
    }
    cudaEvent_t take()
    {
        if (!c->pool.empty()) {
            cudaEvent_t e = c->pool.back();
            c->pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

// Keys, sort and bin starts (into bin_start, n_cells + 1 words) of a cloud
// with n > 0: one kernel; *cur_out = the buffer that holds the sorted keys /
// permutation.
int bin_cloud(fla_ctx* ctx, const fla_cloud& c, const fla_mesh& m, void* ws, const WsLayout& L, uint32_t* bin_start,
              cudaStream_t s, int* cur_out, uint32_t* zero = nullptr, int nzero = 0)
{
    BinWork w{};
    for (int b = 0; b < 2; ++b) {
        w.keys[b] = at<uint32_t>(ws, L.keys[b]);
        w.vals[b] = at<uint32_t>(ws, L.vals[b]);
    }
    w.scratch = at<void>(ws, L.scratch);
    const int stall = (ctx->stall & FLA_STALL_BINNING) != 0;
    ctx->stall &= ~FLA_STALL_BINNING;
    cudaError_t e;
    {
        PhaseScope ps(ctx, FLA_PHASE_SORT, s, 1);   // keys, sort and bin starts
        e = launch_binning(c, m, w, bin_start, (DevStatus*)ctx->status_dev, stall, s, zero, nzero);
    }
    if (e != cudaSuccess) return FLA_ERR_CUDA;
    *cur_out = bin_sorted_buffer(bin_plan(c.n, cells_of(m)));
    return FLA_OK;
}

// Workspace check: `need` bytes from the start of the layout (each entry point
// uses a prefix of it: binning up to the records, PSI-CELL 4 values per record,
// the kernel-regression deposit all of it).
int ws_ok(void* ws, size_t bytes, size_t need)
{
    if (!ws || !aligned(ws, 256)) return FLA_ERR_WORKSPACE;
    if (bytes < need) return FLA_ERR_WORKSPACE;
    return FLA_OK;
}

}  // namespace

extern "C" {

int fla_abi_version(void) { return FLA_ABI_VERSION; }

const char* fla_status_string(int code)
{
    switch (code) {
    case FLA_OK: return "ok";
    case FLA_ERR_ARG: return "invalid argument";
    case FLA_ERR_CUDA: return "CUDA error";
    case FLA_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FLA_ERR_NONFINITE: return "non-finite values found on the device";
    case FLA_ERR_TIMEOUT: return "device wait timed out";
    case FLA_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
    }
}

int fla_create(fla_ctx** out, int device)
{
    if (!out) return FLA_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
        cudaGetLastError();
        return FLA_ERR_CUDA;
    }
    if (device < 0 || device >= count) return FLA_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FLA_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return FLA_ERR_CUDA;
    fla_ctx* c = (fla_ctx*)calloc(1, sizeof(fla_ctx));
    if (!c) return FLA_ERR_ARG;
    c->device = device;
    c->num_sms = sms;
    if (cudaMalloc((void**)&c->status_dev, 64) != cudaSuccess) {
        free(c);
        return FLA_ERR_CUDA;
    }
    if (cudaMemset(c->status_dev, 0, 64) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(c->status_dev);
        free(c);
        return FLA_ERR_CUDA;
    }
    new (&c->pending) std::vector<fla_ctx::Pending>();
    new (&c->pool) std::vector<cudaEvent_t>();
    *out = c;
    return FLA_OK;
}

void fla_destroy(fla_ctx* ctx)
{
    if (!ctx) return;
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    ctx->pending.~vector();
    ctx->pool.~vector();
    if (ctx->status_dev) cudaFree(ctx->status_dev);
    free(ctx);
}

const char* fla_phase_name(int32_t phase)
{
    static const char* names[FLA_PHASE_COUNT] = {"carrier", "advance", "keys", "sort", "bins", "records", "gather",
                                                 "psicell"};
    return (phase >= 0 && phase < FLA_PHASE_COUNT) ? names[phase] : "unknown";
}

int fla_profile_enable(fla_ctx* ctx, int enable, int reset)
{
    if (!ctx || (enable != 0 && enable != 1)) return FLA_ERR_ARG;
    if (reset) {
        for (auto& p : ctx->pending) {
            ctx->pool.push_back(p.a);
            ctx->pool.push_back(p.b);
        }
        ctx->pending.clear();
        for (int i = 0; i < FLA_PHASE_COUNT; ++i) {
            ctx->ms[i] = 0.0;
            ctx->launches[i] = 0;
            ctx->calls[i] = 0;
        }
    }
    ctx->timing = enable;
    return FLA_OK;
}

int fla_profile_read(fla_ctx* ctx, int32_t n_phases, double* ms, int64_t* launches, int64_t* calls)
{
    if (!ctx || n_phases < 0) return FLA_ERR_ARG;
    int rc = FLA_OK;
    for (auto& p : ctx->pending) {
        float t = 0.0f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess)
            rc = FLA_ERR_CUDA;
        else
            ctx->ms[p.phase] += t;
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < n_phases && i < FLA_PHASE_COUNT; ++i) {
        if (ms) ms[i] = ctx->ms[i];
        if (launches) launches[i] = ctx->launches[i];
        if (calls) calls[i] = ctx->calls[i];
    }
    return rc;
}

int fla_state_layout(int32_t kind, int32_t dim, int32_t* n_planes, int32_t* off_x, int32_t* off_v, int32_t* off_J,
                     int32_t* off_W, int32_t* off_acc)
{
    if ((kind != FLA_CLOUD_FLA && kind != FLA_CLOUD_LPT) || (dim != 2 && dim != 3)) return FLA_ERR_ARG;
    if (n_planes) *n_planes = state_planes(kind, dim);
    if (off_x) *off_x = 0;
    if (off_v) *off_v = dim;
    if (off_J) *off_J = kind == FLA_CLOUD_FLA ? 2 * dim : -1;
    if (off_W) *off_W = kind == FLA_CLOUD_FLA ? 2 * dim + dim * dim : -1;
    if (off_acc) *off_acc = acc_offset(kind, dim);
    return FLA_OK;
}

size_t fla_carrier_nodes_bytes(const fla_mesh* mesh, int32_t dtype)
{
    if (!mesh_ok(mesh) || !dtype_ok(dtype)) return 0;
    const size_t nn = (size_t)mesh->n + 1;
    const size_t nodes = mesh->dim == 2 ? nn * nn : nn * nn * nn;
    if (dtype == FLA_F32X2)   // the a array, the b array, the tail of component maxima
        return nodes * node_stride(mesh->dim) * 8 + kNodesX2TailBytes;
    return nodes * node_stride(mesh->dim) * (dtype == FLA_F32 ? 4 : 8);
}

int fla_carrier_sample(fla_ctx* ctx, const fla_carrier_desc* c, const fla_mesh* mesh, double t, int32_t dtype,
                       void* nodes_dev, fla_stream_t stream)
{
    if (!ctx || !c || !mesh_ok(mesh) || !nodes_dev || !aligned(nodes_dev, 16)) return FLA_ERR_ARG;
    if (!dtype_ok(dtype)) return FLA_ERR_ARG;
    if (c->dim != mesh->dim || c->kind < FLA_CARRIER_UNIFORM || c->kind > FLA_CARRIER_ABCJET3) return FLA_ERR_ARG;
    if ((c->kind == FLA_CARRIER_TG2 || c->kind == FLA_CARRIER_JETVORT2) && c->dim != 2) return FLA_ERR_ARG;
    if (c->kind == FLA_CARRIER_ABCJET3 && c->dim != 3) return FLA_ERR_ARG;
    if (c->n_vortex < 0 || c->n_vortex > FLA_MAX_VORTICES || !isfinite(t)) return FLA_ERR_ARG;
    if (c->kind == FLA_CARRIER_JETVORT2) {
        if (!(c->jet_width > 0)) return FLA_ERR_ARG;
        for (int k = 0; k < c->n_vortex; ++k)
            if (!(c->vortex[k][3] > 0)) return FLA_ERR_ARG;
    }
    if (c->kind == FLA_CARRIER_ABCJET3 && !(c->jet_radius > 0)) return FLA_ERR_ARG;
    PhaseScope ps(ctx, FLA_PHASE_CARRIER, (cudaStream_t)stream, 1);
    return cuda_status(launch_carrier_sample(*c, *mesh, t, dtype, nodes_dev, (cudaStream_t)stream));
}

int fla_batch_deadline(double St0, double delta, double dt, int32_t step_start, int32_t* step_dead)
{
    if (!step_dead || !(St0 > 0) || !(dt > 0) || !isfinite(delta)) return FLA_ERR_ARG;
    if (!(delta < 0.0)) {
        *step_dead = FLA_NO_DEADLINE;
        return FLA_OK;
    }
    const double thr = fmax(0.01, 4.0 * dt / St0);
    const double est = (1.0 - thr) / (-delta) / dt;
    if (est > 2.0e9) {
        *step_dead = FLA_NO_DEADLINE;
        return FLA_OK;
    }
    long long s = (long long)step_start + (long long)floor(est) - 2;
    if (s < step_start) s = step_start;
    while (!(1.0 + delta * (double)(s - step_start) * dt < thr)) ++s;
    *step_dead = s > 2147483646LL ? FLA_NO_DEADLINE : (int32_t)s;
    return FLA_OK;
}

int fla_advance(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const void* nodes_dev, int32_t step0,
                int32_t nsteps, double dt, uint32_t flags, fla_stream_t stream)
{
    return fla_advance_ordered(ctx, cloud, mesh, nodes_dev, nullptr, step0, nsteps, dt, flags, stream);
}

int fla_advance_ordered(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const void* nodes_dev,
                        const uint32_t* order_dev, int32_t step0, int32_t nsteps, double dt, uint32_t flags,
                        fla_stream_t stream)
{
    if (!ctx) return FLA_ERR_ARG;
    if (order_dev && !aligned(order_dev, 4)) return FLA_ERR_ARG;
    int st = cloud_ok(cloud, mesh);
    if (st != FLA_OK) return st;
    if (nsteps < 0 || step0 < 0 || (int64_t)step0 + nsteps > 2147483647LL || !(dt > 0) || !isfinite(dt))
        return FLA_ERR_ARG;
    if (flags & ~FLA_ADVANCE_RESET_ACC) return FLA_ERR_ARG;
    if (cloud->n == 0 || nsteps == 0) return FLA_OK;
    if (!nodes_dev || !aligned(nodes_dev, 16)) return FLA_ERR_ARG;
    const bool guarded = cloud->fold_dev != nullptr;   // screening + guarded passes
    PhaseScope ps(ctx, FLA_PHASE_ADVANCE, (cudaStream_t)stream, guarded ? 2 : 1);
    return cuda_status(launch_advance(*cloud, *mesh, nodes_dev, step0, nsteps, dt,
                                      (flags & FLA_ADVANCE_RESET_ACC) != 0, (DevStatus*)ctx->status_dev,
                                      ctx->num_sms, (cudaStream_t)stream, order_dev));
}

int fla_workspace_order(const fla_mesh* mesh, int64_t n_droplets, size_t* offset)
{
    if (!offset || !mesh_ok(mesh) || n_droplets < 1 || n_droplets >= 2147483647LL) return FLA_ERR_ARG;
    // keys and values lead the layout and depend on n alone
    *offset = layout(*mesh, FLA_F32, FLA_KERNEL_ISO, n_droplets).vals[sorted_buffer(*mesh, n_droplets)];
    return FLA_OK;
}

size_t fla_fold_bytes(int32_t dim, int64_t n)
{
    if ((dim != 2 && dim != 3) || n < 0) return 0;
    return fold_layout(dim, n).total;
}

int fla_workspace_size(const fla_mesh* mesh, int32_t dtype, int32_t kernel, int64_t n_droplets, size_t* bytes)
{
    if (!bytes || !mesh_ok(mesh) || !dtype_ok(dtype)) return FLA_ERR_ARG;
    if ((kernel != FLA_KERNEL_ISO && kernel != FLA_KERNEL_ANISO) || n_droplets < 0 || n_droplets >= 2147483647LL)
        return FLA_ERR_ARG;
    *bytes = layout(*mesh, dtype, kernel, n_droplets).total;
    return FLA_OK;
}

int fla_cell_bins(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, uint32_t* keys_sorted_dev,
                  uint32_t* perm_dev, uint32_t* bin_start_dev, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    if (!ctx) return FLA_ERR_ARG;
    int st = cloud_ok(cloud, mesh);
    if (st != FLA_OK) return st;
    if (!bin_start_dev || (cloud->n > 0 && (!keys_sorted_dev || !perm_dev))) return FLA_ERR_ARG;
    const WsLayout L = layout(*mesh, cloud->dtype, FLA_KERNEL_ISO, cloud->n);
    st = ws_ok(ws, ws_bytes, L.rec);
    if (st != FLA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nc = cells_of(*mesh);
    if (cloud->n == 0) {
        return cuda_status(cudaMemsetAsync(bin_start_dev, 0, (size_t)(nc + 1) * 4, s));
    }
    int cur = 0;
    st = bin_cloud(ctx, *cloud, *mesh, ws, L, bin_start_dev, s, &cur);
    if (st != FLA_OK) return st;
    const uint32_t* ks = at<uint32_t>(ws, L.keys[cur]);
    const uint32_t* vs = at<uint32_t>(ws, L.vals[cur]);
    if (cudaMemcpyAsync(keys_sorted_dev, ks, (size_t)cloud->n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return FLA_ERR_CUDA;
    return cuda_status(cudaMemcpyAsync(perm_dev, vs, (size_t)cloud->n * 4, cudaMemcpyDeviceToDevice, s));
}

namespace {

// The kernel-regression deposit; aux (learned correction only) receives per
// sorted record g(f) and whether h moves with it.
int deposit_impl(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const fla_deposit_cfg* cfg,
                 const fla_sources* out, void* ws, size_t ws_bytes, fla_stream_t stream, float* aux)
{
    if (!ctx || !cfg || !out) return FLA_ERR_ARG;
    int st = cloud_ok(cloud, mesh);
    if (st != FLA_OK) return st;
    if (cloud->kind != FLA_CLOUD_FLA) return FLA_ERR_ARG;
    if (cfg->kernel != FLA_KERNEL_ISO && cfg->kernel != FLA_KERNEL_ANISO) return FLA_ERR_ARG;
    if (!(cfg->h_min > 0) || !(cfg->h_max >= cfg->h_min) || !isfinite(cfg->h_max)) return FLA_ERR_ARG;
    if (!(cfg->window_dt > 0) || !isfinite(cfg->window_dt) || !(cfg->p > 0) || !isfinite(cfg->p)) return FLA_ERR_ARG;
    if (cfg->kernel == FLA_KERNEL_ANISO && !(cfg->h_max * cfg->h_max > mesh->dim * cfg->h_min * cfg->h_min))
        return FLA_ERR_ARG;
    if (cfg->precision != FLA_PREC_MIXED && cfg->precision != FLA_PREC_PLAIN) return FLA_ERR_ARG;
    if (cfg->mlp_dev) {   // learned correction: single precision
        if (!aligned(cfg->mlp_dev, 16) || (cfg->mlp_out_dev && !aligned(cfg->mlp_out_dev, 4))) return FLA_ERR_ARG;
        if (cloud->dtype != FLA_F32) return FLA_ERR_UNSUPPORTED;
    }
    if (cfg->h_max * mesh->n > 64.0) return FLA_ERR_UNSUPPORTED;   // support wider than 192 cells
    if (!out->s_mass_dev || !out->s_mom_dev) return FLA_ERR_ARG;
    const size_t T = cloud->dtype == FLA_F64 ? 8 : 4;
    if (!aligned(out->s_mass_dev, T) || !aligned(out->s_mom_dev, T) || (out->dsum_dev && !aligned(out->dsum_dev, T)))
        return FLA_ERR_ARG;
    const WsLayout L = layout(*mesh, cloud->dtype, cfg->kernel, cloud->n);
    st = ws_ok(ws, ws_bytes, L.total);
    if (st != FLA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nc = cells_of(*mesh);
    uint32_t* bins = at<uint32_t>(ws, L.bin_start);
    // misc words 0-7: ext_max, the 2D gather's counters (1, 2), the tile
    // gather's counters (4, 5) and candidate total (6, 7); all start at zero
    unsigned int* ext = at<unsigned int>(ws, L.misc);
    if (cloud->n == 0) {
        if (cudaMemsetAsync(ext, 0, 32, s) != cudaSuccess) return FLA_ERR_CUDA;
        if (cudaMemsetAsync(bins, 0, (size_t)(nc + 1) * 4, s) != cudaSuccess) return FLA_ERR_CUDA;
    } else {
        int cur = 0;
        st = bin_cloud(ctx, *cloud, *mesh, ws, L, bins, s, &cur, ext, 8);   // the keys kernel clears misc
        if (st != FLA_OK) return st;
        {
            PhaseScope ps(ctx, FLA_PHASE_RECORDS, s, 1);
            if (launch_records(*cloud, *mesh, *cfg, at<uint32_t>(ws, L.vals[cur]), bins, nc, at<void>(ws, L.rec),
                               ext, (DevStatus*)ctx->status_dev, s, aux) != cudaSuccess)
                return FLA_ERR_CUDA;
        }
    }
    if (use_gather2d(*mesh, cloud->dtype, cfg->kernel)) {
        PhaseScope ps(ctx, FLA_PHASE_GATHER, s, 3);
        const int nt = gather2d_tiles(mesh->n);
        uint32_t* tiles = at<uint32_t>(ws, L.tiles);
        return cuda_status(launch_gather2d(*mesh, *cfg, at<void>(ws, L.rec), bins, ext, tiles, tiles + nt,
                                           ext + 1, at<void>(ws, L.temp), gather2d_item_budget(mesh->n, cloud->n),
                                           *out, (DevStatus*)ctx->status_dev, ctx->num_sms, s));
    }
    PhaseScope ps(ctx, FLA_PHASE_GATHER, s, 3);
    NwWork w{};
    w.tile_cand = at<uint32_t>(ws, L.tiles);
    w.tile_items = w.tile_cand + nw_tiles(mesh->dim, mesh->n);
    w.counter = at<unsigned int>(ws, L.misc + 16);
    w.done = at<unsigned int>(ws, L.misc + 20);
    w.cand_total = at<unsigned long long>(ws, L.misc + 24);
    w.temp = at<void>(ws, L.temp);
    return cuda_status(launch_nw_gather(*cloud, *mesh, *cfg, at<void>(ws, L.rec), bins, ext, w, *out,
                                        (DevStatus*)ctx->status_dev, ctx->num_sms, s));
}

struct LearnLayout {
    size_t q, aux, dldc, partial, scal, total;
};

LearnLayout learn_layout(const fla_mesh& m, int64_t n, int num_sms)
{
    LearnLayout L{};
    const size_t nn = (size_t)(n > 0 ? n : 1);
    size_t o = 0;
    L.q = o; o += up256((size_t)cells_of(m) * (m.dim == 2 ? 4 : 8) * 4);
    L.aux = o; o += up256(nn * 8);
    L.dldc = o; o += up256(nn * 4);
    L.partial = o; o += up256((size_t)(num_sms > 0 ? num_sms : 1) * kMlpParams * 4);
    L.scal = o; o += 256;
    L.total = o;
    return L;
}

int backward_parts(fla_ctx* ctx, int64_t n)
{
    const int64_t tiles = (n + kMlpRows - 1) / kMlpRows;
    const int64_t p = tiles < ctx->num_sms ? tiles : ctx->num_sms;
    return (int)(p > 0 ? p : 1);
}

}  // namespace

int fla_deposit_sources(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const fla_deposit_cfg* cfg,
                        const fla_sources* out, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    return deposit_impl(ctx, cloud, mesh, cfg, out, ws, ws_bytes, stream, nullptr);
}

int fla_learn_workspace_size(fla_ctx* ctx, const fla_mesh* mesh, int64_t n_droplets, size_t* bytes)
{
    if (!ctx || !bytes || !mesh_ok(mesh) || n_droplets < 0 || n_droplets >= 2147483647LL) return FLA_ERR_ARG;
    *bytes = learn_layout(*mesh, n_droplets, ctx->num_sms).total;
    return FLA_OK;
}

int fla_learn_grad(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const fla_deposit_cfg* cfg,
                   const uint32_t* cells_dev, int64_t n_train, const float* targets_dev, const fla_sources* out,
                   float* grad_dev, float* loss_dev, void* ws, size_t ws_bytes, void* lws, size_t lws_bytes,
                   fla_stream_t stream)
{
    if (!ctx || !cfg || !out || !cloud || !mesh) return FLA_ERR_ARG;
    if (!cfg->mlp_dev || !out->dsum_dev || !grad_dev || !loss_dev) return FLA_ERR_ARG;
    if (cloud->dtype != FLA_F32) return FLA_ERR_UNSUPPORTED;
    if (n_train < 1 || n_train > 2147483647LL || !cells_dev || !targets_dev) return FLA_ERR_ARG;
    const LearnLayout LL = learn_layout(*mesh, cloud->n, ctx->num_sms);
    if (!lws || !aligned(lws, 256) || lws_bytes < LL.total) return FLA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int st = deposit_impl(ctx, cloud, mesh, cfg, out, ws, ws_bytes, stream, at<float>(lws, LL.aux));
    if (st != FLA_OK) return st;
    const WsLayout L = layout(*mesh, cloud->dtype, cfg->kernel, cloud->n);
    const int cur = sorted_buffer(*mesh, cloud->n);
    LearnArgs a{};
    a.dim = mesh->dim;
    a.N = mesh->n;
    a.kernel = cfg->kernel;
    a.hmin2 = (float)(cfg->h_min * cfg->h_min);
    a.n_cells = cells_of(*mesh);
    a.s_mass = (const float*)out->s_mass_dev;
    a.s_mom = (const float*)out->s_mom_dev;
    a.dsum = (const float*)out->dsum_dev;
    a.cells = cells_dev;
    a.n_train = n_train;
    a.targets = targets_dev;
    a.q = at<float>(lws, LL.q);
    a.q_stride = mesh->dim == 2 ? 4 : 8;
    a.scal = at<float>(lws, LL.scal);
    a.loss = loss_dev;
    a.bin_start = at<uint32_t>(ws, L.bin_start);
    a.rec = at<void>(ws, L.rec);
    a.aux = at<float>(lws, LL.aux);
    a.dldc = at<float>(lws, LL.dldc);
    if (launch_learn_cells(a, s) != cudaSuccess) return FLA_ERR_CUDA;
    if (launch_learn_dc(a, cloud->n, s) != cudaSuccess) return FLA_ERR_CUDA;
    const int parts = backward_parts(ctx, cloud->n);
    if (launch_learn_backward(*cloud, *mesh, *cfg, at<uint32_t>(ws, L.vals[cur]), a.bin_start, a.n_cells, a.dldc,
                              at<float>(lws, LL.partial), parts, (DevStatus*)ctx->status_dev, s) != cudaSuccess)
        return FLA_ERR_CUDA;
    return cuda_status(launch_grad_reduce(at<float>(lws, LL.partial), parts, grad_dev, s));
}

int fla_adam_step(fla_ctx* ctx, float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n,
                  float lr, float beta1, float beta2, float eps, int32_t step, fla_stream_t stream)
{
    if (!ctx || n < 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return FLA_ERR_ARG;
    if (n > 0 && (!params_dev || !grad_dev || !m_dev || !v_dev)) return FLA_ERR_ARG;
    return cuda_status(launch_adam(params_dev, grad_dev, m_dev, v_dev, n, lr, beta1, beta2, eps, step,
                                   (cudaStream_t)stream));
}

namespace {
// The box-count (PSI-CELL) and Cloud-In-Cell deposits share their argument checks and binning.
int parcel_deposit(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, double window_dt, int32_t per_cell,
                   const fla_psicell_out* out, void* ws, size_t ws_bytes, fla_stream_t stream, bool cic)
{
    if (!ctx || !out) return FLA_ERR_ARG;
    int st = cloud_ok(cloud, mesh);
    if (st != FLA_OK) return st;
    if (cloud->kind != FLA_CLOUD_LPT) return FLA_ERR_ARG;
    if (!(window_dt > 0) || !isfinite(window_dt) || (per_cell != 0 && per_cell != 1)) return FLA_ERR_ARG;
    if (!out->counts_dev || !out->s_mass_dev || !out->s_mom_dev) return FLA_ERR_ARG;
    const WsLayout L = layout(*mesh, cloud->dtype, FLA_KERNEL_ISO, cloud->n);
    const size_t rec = up256((size_t)(cloud->n > 0 ? cloud->n : 1) * (cic ? 8 : 4) * (cloud->dtype == FLA_F64 ? 8 : 4));
    st = ws_ok(ws, ws_bytes, L.rec + rec);
    if (st != FLA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nc = cells_of(*mesh);
    uint32_t* bins = at<uint32_t>(ws, L.bin_start);
    int cur = 0;
    if (cloud->n == 0) {
        if (cudaMemsetAsync(bins, 0, (size_t)(nc + 1) * 4, s) != cudaSuccess) return FLA_ERR_CUDA;
    } else {
        st = bin_cloud(ctx, *cloud, *mesh, ws, L, bins, s, &cur);
        if (st != FLA_OK) return st;
    }
    PhaseScope ps(ctx, FLA_PHASE_PSICELL, s, cloud->n > 0 ? 2 : 1);
    if (cic)
        return cuda_status(launch_cic(*cloud, *mesh, window_dt, per_cell, at<uint32_t>(ws, L.vals[cur]), bins,
                                      at<void>(ws, L.rec), *out, (DevStatus*)ctx->status_dev, s));
    return cuda_status(launch_psicell(*cloud, *mesh, window_dt, per_cell, at<uint32_t>(ws, L.vals[cur]), bins,
                                      at<void>(ws, L.rec), *out, (DevStatus*)ctx->status_dev, s));
}
}  // namespace

int cic_deposit(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, double window_dt, int32_t per_cell,
                const fla_psicell_out* out, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    return parcel_deposit(ctx, cloud, mesh, window_dt, per_cell, out, ws, ws_bytes, stream, true);
}

int psicell_deposit(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, double window_dt, int32_t per_cell,
                    const fla_psicell_out* out, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    return parcel_deposit(ctx, cloud, mesh, window_dt, per_cell, out, ws, ws_bytes, stream, false);
}

int fla_test_stall(fla_ctx* ctx, uint32_t what)
{
    if (!ctx || (what & ~(FLA_STALL_BINNING | FLA_STALL_BATCH_WINDOW))) return FLA_ERR_ARG;
    ctx->stall |= what;
    return FLA_OK;
}

int fla_sync_status(fla_ctx* ctx, fla_stream_t stream, fla_device_status* out, int reset)
{
    if (!ctx || !out) return FLA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(out, ctx->status_dev, sizeof(fla_device_status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FLA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FLA_ERR_CUDA;
    if (reset && cudaMemsetAsync(ctx->status_dev, 0, 64, s) != cudaSuccess) return FLA_ERR_CUDA;
    if (out->flags & (FLA_STATUS_MLP_TIMEOUT | FLA_STATUS_WAIT_TIMEOUT)) return FLA_ERR_TIMEOUT;
    return out->nonfinite > 0 ? FLA_ERR_NONFINITE : FLA_OK;
}

}  // extern "C"

int fla_mlp_pack(fla_ctx* ctx, const float* params_dev, void* packed_dev, fla_stream_t stream)
{
    if (!ctx || !params_dev || !packed_dev || !aligned(packed_dev, 16) || !aligned(params_dev, 4)) return FLA_ERR_ARG;
    return cuda_status(launch_mlp_pack(params_dev, packed_dev, (cudaStream_t)stream));
}

int fla_mlp_forward(fla_ctx* ctx, const void* packed_dev, const float* features_dev, int64_t n, float* out_dev,
                    fla_stream_t stream)
{
    if (!ctx || n < 0 || n >= 2147483647LL) return FLA_ERR_ARG;
    if (n == 0) return FLA_OK;
    if (!packed_dev || !aligned(packed_dev, 16) || !features_dev || !out_dev) return FLA_ERR_ARG;
    return cuda_status(launch_mlp_forward(packed_dev, features_dev, n, out_dev, (DevStatus*)ctx->status_dev,
                                          (cudaStream_t)stream));
}
