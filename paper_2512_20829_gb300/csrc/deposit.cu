// Kernel-regression gather (Eqs. 13 and 16) and PSI-CELL box counting (Eqs. 10-11).
//
// Gather: one CTA per tile of cells (16x16 in 2D, 8x8x4 in 3D), one cell per
// thread, each warp owning a 32-cell sub-tile.  Droplet records are sorted by
// cell key, so the records of the cells in one mesh row of the tile's
// neighbourhood are contiguous.  The CTA walks those rows, each thread loads
// one record, records whose support cannot reach the tile are culled, and the
// survivors are compacted (order kept) into shared memory.  Each warp then
// tests 32 staged records at a time against its own sub-tile with one ballot
// and evaluates only the records that can reach it: truncation test (as a
// predicate), Gaussian weight 2^(c r^2 + log2(1/h)) with one MUFU ex2 in single
// precision, FMA accumulation.  Each staged chunk is summed plainly and chunk
// sums are added with Neumaier compensation.  Every cell sums its records in
// staging order and no atomics touch the outputs, so results are deterministic.
#include "batch.cuh"

namespace fla {
namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Neumaier-compensated add of a chunk sum v into (s, c).
template <typename T>
__device__ __forceinline__ void neumaier(T& s, T& c, T v)
{
    const T t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

struct GatherArgs {
    const void* rec;
    int64_t rec_base;             // sorted position of rec[0]
    const uint32_t* bin_start;
    const unsigned int* ext_max;
    int N;
    int per_cell;
    void* s_mass;
    void* s_mom;
    void* dsum;
    DevStatus* status;
};

// CTA tile of cells and the per-warp sub-tile (32 cells, one per lane).
template <int D> struct Tile;
template <> struct Tile<2> {
    static constexpr int X = 16, Y = 16, Z = 1;      // 8 warps of 8 x 4 cells
    static constexpr int SX = 8, SY = 4, SZ = 1;
};
template <> struct Tile<3> {
    static constexpr int X = 8, Y = 8, Z = 4;        // 8 warps of 4 x 4 x 2 cells
    static constexpr int SX = 4, SY = 4, SZ = 2;
};

constexpr int GT = 256;            // threads per CTA = cells per tile
constexpr int CAP = 2 * GT;        // staged records

// position of the squared support radius inside a record
template <int D, int KER> struct ExtSlot { static constexpr int v = (KER == FLA_KERNEL_ISO) ? (D == 2 ? 7 : 3) : (D == 2 ? 3 : 10); };

// Weight of one record at this lane's cell centre; inside = truncation test.
template <typename T, int D, int KER>
__device__ __forceinline__ T weight_of(const T* r, const float* xcf, const T* xc, bool& inside)
{
    if (sizeof(T) == 4) {
        const float* rf = reinterpret_cast<const float*>(r);
        float df[3];
#pragma unroll
        for (int i = 0; i < D; ++i) df[i] = __fsub_rn(xcf[i], rf[i]);
        if (KER == FLA_KERNEL_ISO) {
            // single-precision decision in a fixed operation order
            float r2 = __fmul_rn(df[0], df[0]);
            r2 = __fmaf_rn(df[1], df[1], r2);
            if (D == 3) r2 = __fmaf_rn(df[2], df[2], r2);
            const float r2max = D == 2 ? rf[7] : rf[3];
            const float c = D == 2 ? rf[2] : rf[4];
            const float lih = D == 2 ? rf[3] : rf[5];
            inside = r2 <= r2max;
            const float w = ex2_approx(fmaf(r2, c, lih));
            return T(inside ? w : 0.0f);
        } else {
            float P[9];
            float lpref;
            if (D == 2) {
                P[0] = rf[4]; P[1] = rf[5]; P[2] = rf[5]; P[3] = rf[6];
                lpref = rf[2];
            } else {
                P[0] = rf[4]; P[1] = rf[5]; P[2] = rf[6];
                P[3] = rf[5]; P[4] = rf[7]; P[5] = rf[8];
                P[6] = rf[6]; P[7] = rf[8]; P[8] = rf[9];
                lpref = rf[3];
            }
            float pd[3];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float acc = __fmul_rn(P[i * D], df[0]);
#pragma unroll
                for (int k = 1; k < D; ++k) acc = __fmaf_rn(P[i * D + k], df[k], acc);
                pd[i] = acc;
            }
            float q = __fmul_rn(pd[0], df[0]);
#pragma unroll
            for (int i = 1; i < D; ++i) q = __fmaf_rn(pd[i], df[i], q);
            inside = q <= 9.0f;
            const float w = ex2_approx(fmaf(q, -0.72134752044448170368f, lpref));
            return T(inside ? w : 0.0f);
        }
    } else {
        T df[3];
#pragma unroll
        for (int i = 0; i < D; ++i) df[i] = xc[i] - r[i];
        if (KER == FLA_KERNEL_ISO) {
            T r2 = df[0] * df[0] + df[1] * df[1];
            if (D == 3) r2 += df[2] * df[2];
            const T c = D == 2 ? r[2] : r[4];
            const T ih = D == 2 ? r[3] : r[5];
            const T e = r2 * c;                       // = -q/2
            inside = e >= T(-4.5);
            return inside ? ih * exp(e) : T(0);
        } else {
            T P[9];
            T pref;
            if (D == 2) {
                P[0] = r[4]; P[1] = r[5]; P[2] = r[5]; P[3] = r[6];
                pref = r[2];
            } else {
                P[0] = r[4]; P[1] = r[5]; P[2] = r[6];
                P[3] = r[5]; P[4] = r[7]; P[5] = r[8];
                P[6] = r[6]; P[7] = r[8]; P[8] = r[9];
                pref = r[3];
            }
            T q = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) q += df[i] * P[i * D + k] * df[k];
            inside = q <= T(9);
            return inside ? pref * exp(T(-0.5) * q) : T(0);
        }
    }
}

// One CTA tile of cells with origin (tx0, ty0, tz0).
template <typename T, int D, int KER>
__device__ __forceinline__ void gather_tile(const GatherArgs& a, int tx0, int ty0, int tz0)
{
    constexpr int RV = record_values(D, KER);
    constexpr int R4 = RV / 4;
    constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
    constexpr int SX = Tile<D>::SX, SY = Tile<D>::SY, SZ = Tile<D>::SZ;
    constexpr int EXT = ExtSlot<D, KER>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* srec = reinterpret_cast<T*>(smem_raw);
    __shared__ int s_wcount[GT / 32];
    __shared__ int s_count;

    const int N = a.N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0[3] = {tx0, ty0, tz0};
    // warp sub-tile origin and this lane's cell
    int w0[3], cc[3];
    if (D == 2) {
        w0[0] = t0[0] + (warp & 1) * SX; w0[1] = t0[1] + (warp >> 1) * SY; w0[2] = 0;
        cc[0] = w0[0] + (lane & 7); cc[1] = w0[1] + (lane >> 3); cc[2] = 0;
    } else {
        w0[0] = t0[0] + (warp & 1) * SX; w0[1] = t0[1] + ((warp >> 1) & 1) * SY; w0[2] = t0[2] + (warp >> 2) * SZ;
        cc[0] = w0[0] + (lane & 3); cc[1] = w0[1] + ((lane >> 2) & 3); cc[2] = w0[2] + (lane >> 4);
    }
    bool in_mesh = cc[0] < N && cc[1] < N && (D == 2 || cc[2] < N);
    bool warp_live = w0[0] < N && w0[1] < N && (D == 2 || w0[2] < N);
    // cell centres (i + 1/2)/N in the kernel's precision: single-precision tiles
    // need no double-precision division (slow on this GPU)
    auto centre = [&](int i) -> T {
        if (sizeof(T) == 4) return T(((float)i + 0.5f) / (float)N);
        return T(((double)i + 0.5) / (double)N);
    };
    T xc[3];
    float xcf[3];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        xc[q] = centre(cc[q]);
        xcf[q] = sizeof(T) == 4 ? ((float)cc[q] + 0.5f) / (float)N : (float)xc[q];
    }
    // boxes of cell centres: the CTA tile (staging cull) and the warp sub-tile (flush cull)
    T lo[3], hi[3], wlo[3], whi[3];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const int tq = q == 0 ? TX : (q == 1 ? TY : TZ);
        const int sq = q == 0 ? SX : (q == 1 ? SY : SZ);
        const int last = (t0[q] + tq < N ? t0[q] + tq : N) - 1;
        const int wlast = (w0[q] + sq < N ? w0[q] + sq : N) - 1;
        lo[q] = centre(t0[q]);
        hi[q] = centre(last);
        wlo[q] = centre(w0[q]);
        whi[q] = centre(wlast);
    }
    const float ext2max = __uint_as_float(__ldg(a.ext_max));
    const int R = (int)floorf(sqrtf(ext2max) * (float)N + 0.5f) + 1;

    T sD = T(0), cD = T(0);
    T sN[4] = {T(0), T(0), T(0), T(0)}, cN[4] = {T(0), T(0), T(0), T(0)};
    int npairs = 0;
    if (tid == 0) s_count = 0;

    const int xlo = t0[0] - R < 0 ? 0 : t0[0] - R;
    const int xhi = t0[0] + TX - 1 + R > N - 1 ? N - 1 : t0[0] + TX - 1 + R;
    const int ylo = t0[1] - R < 0 ? 0 : t0[1] - R;
    const int yhi = t0[1] + TY - 1 + R > N - 1 ? N - 1 : t0[1] + TY - 1 + R;
    int zlo = 0, zhi = 0;
    if (D == 3) {
        zlo = t0[2] - R < 0 ? 0 : t0[2] - R;
        zhi = t0[2] + TZ - 1 + R > N - 1 ? N - 1 : t0[2] + TZ - 1 + R;
    }
    __syncthreads();

    // Evaluate the staged records for this warp's cells in staging order: 32 records
    // at a time are tested against the warp's sub-tile (one per lane, one ballot),
    // and only those that can reach it are evaluated by every lane.
    auto flush = [&](int count) {
        if (!warp_live) return;
        T pD = T(0), pN[4] = {T(0), T(0), T(0), T(0)};
        for (int k0 = 0; k0 < count; k0 += 32) {
            const int k = k0 + lane;
            bool ov = false;
            if (k < count) {
                const T* r = srec + k * RV;
                T d2 = T(0);
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    const T dl = wlo[q] - r[q], dh = r[q] - whi[q];
                    const T dd = dl > T(0) ? dl : (dh > T(0) ? dh : T(0));
                    d2 += dd * dd;
                }
                ov = d2 <= r[EXT] * T(1.0009765625);
            }
            unsigned m = __ballot_sync(0xffffffffu, ov);
            while (m) {
                const int j1 = __ffs(m) - 1;
                m &= m - 1;
                bool in1;
                const T w1 = weight_of<T, D, KER>(srec + (k0 + j1) * RV, xcf, xc, in1);
                const T* am1 = srec + (k0 + j1) * RV + (RV - 4);
                if (m) {
                    const int j2 = __ffs(m) - 1;
                    m &= m - 1;
                    bool in2;
                    const T w2 = weight_of<T, D, KER>(srec + (k0 + j2) * RV, xcf, xc, in2);
                    const T* am2 = srec + (k0 + j2) * RV + (RV - 4);
                    pD += w1;
#pragma unroll
                    for (int q2 = 0; q2 <= D; ++q2) pN[q2] = fma(w1, am1[q2], pN[q2]);
                    pD += w2;
#pragma unroll
                    for (int q2 = 0; q2 <= D; ++q2) pN[q2] = fma(w2, am2[q2], pN[q2]);
                    npairs += (int)in1 + (int)in2;
                } else {
                    pD += w1;
#pragma unroll
                    for (int q2 = 0; q2 <= D; ++q2) pN[q2] = fma(w1, am1[q2], pN[q2]);
                    npairs += (int)in1;
                }
            }
        }
        neumaier(sD, cD, pD);
#pragma unroll
        for (int q2 = 0; q2 <= D; ++q2) neumaier(sN[q2], cN[q2], pN[q2]);
    };

    // walk the neighbourhood rows; each row's records are contiguous
    for (int z = zlo; z <= zhi; ++z) {
        for (int y = ylo; y <= yhi; ++y) {
            const int64_t rowbase = ((int64_t)z * N + y) * N;
            const uint32_t beg = __ldg(a.bin_start + rowbase + xlo);
            const uint32_t end = __ldg(a.bin_start + rowbase + xhi + 1);
            for (uint32_t j0 = beg; j0 < end; j0 += GT) {
                const uint32_t j = j0 + tid;
                T rv[16];
                bool keep = false;
                if (j < end) {
#pragma unroll
                    for (int v = 0; v < R4; ++v)
                        load4<T>((const T*)a.rec, ((int64_t)j - a.rec_base) * R4 + v, rv + 4 * v);
                    T d2 = T(0);
#pragma unroll
                    for (int q = 0; q < D; ++q) {
                        const T dl = lo[q] - rv[q], dh = rv[q] - hi[q];
                        const T dd = dl > T(0) ? dl : (dh > T(0) ? dh : T(0));
                        d2 += dd * dd;
                    }
                    keep = d2 <= rv[EXT] * T(1.0009765625);   // small margin over rounding of the test
                }
                const unsigned ballot = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) s_wcount[warp] = __popc(ballot);
                __syncthreads();
                int off = s_count;
                for (int w2 = 0; w2 < warp; ++w2) off += s_wcount[w2];
                int total = s_count;
                for (int w2 = 0; w2 < GT / 32; ++w2) total += s_wcount[w2];
                if (keep) {
                    const int pos = off + __popc(ballot & ((1u << lane) - 1u));
#pragma unroll
                    for (int v = 0; v < R4; ++v) store4<T>(srec, (int64_t)pos * R4 + v, rv + 4 * v);
                }
                __syncthreads();
                if (total > CAP - GT) {
                    flush(total);
                    total = 0;
                }
                __syncthreads();
                if (tid == 0) s_count = total;
                __syncthreads();
            }
        }
    }
    const int rem = s_count;
    if (rem > 0) flush(rem);

    // pairs inside the truncation (cells of the mesh only): one atomic per CTA
    {
        const int w = __reduce_add_sync(0xffffffffu, in_mesh ? npairs : 0);
        __syncthreads();
        if (lane == 0) s_wcount[warp] = w;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int q = 0; q < GT / 32; ++q) t += s_wcount[q];
            if (t) atomicAdd(&a.status->pairs, (unsigned long long)t);
        }
    }

    if (in_mesh) {
        const int64_t cell = cc[0] + (int64_t)N * (cc[1] + (D == 3 ? (int64_t)N * cc[2] : 0));
        const int64_t nc = D == 2 ? (int64_t)N * N : (int64_t)N * N * N;
        const T Dt = sD + cD;
        T scale = T(1);
        if (a.per_cell) {
            const double dx = 1.0 / N;
            scale = T(D == 2 ? dx * dx : dx * dx * dx);
        }
        const bool cov = Dt > T(0);
        ((T*)a.s_mass)[cell] = cov ? -(sN[0] + cN[0]) / Dt * scale : T(0);
#pragma unroll
        for (int q = 0; q < D; ++q) ((T*)a.s_mom)[q * nc + cell] = cov ? -(sN[1 + q] + cN[1 + q]) / Dt * scale : T(0);
        if (a.dsum) ((T*)a.dsum)[cell] = Dt;
    }
}

template <typename T, int D, int KER>
__global__ void __launch_bounds__(GT) k_nw_gather(GatherArgs a)
{
    gather_tile<T, D, KER>(a, (int)blockIdx.x * Tile<D>::X, (int)blockIdx.y * Tile<D>::Y, (int)blockIdx.z * Tile<D>::Z);
}

// Batched clouds of one group: persistent CTAs take tiles from the group's
// tile table in order through an atomic counter; each tile is computed as by
// k_nw_gather, so the result does not depend on which CTA takes it.
template <int D, int KER>
__global__ void __launch_bounds__(GT) k_batch_gather(BatchDev b, int group, DevStatus* st)
{
    __shared__ int s_tile;
    const BatchTile* tiles = b.tiles[group];
    const int nt = b.n_tiles[group];
    const int64_t rec_base = b.bin_start[b.group_cells[group]];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&b.tile_counter[group], 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= nt) break;
        const BatchTile bt = tiles[t];
        const BatchCloud& c = b.clouds[bt.cloud];
        GatherArgs a{};
        a.rec = b.rec[group];
        a.rec_base = rec_base;
        a.bin_start = b.bin_start + c.cell_off;
        a.ext_max = b.ext_max + bt.cloud;
        a.N = c.N;
        a.per_cell = c.per_cell;
        a.s_mass = c.s_mass;
        a.s_mom = c.s_mom;
        a.dsum = c.dsum;
        a.status = st;
        gather_tile<float, D, KER>(a, bt.x0, bt.y0, bt.z0);
    }
}

template <typename T, int D, int KER>
cudaError_t launch_gather_t(const GatherArgs& a, cudaStream_t s)
{
    constexpr int RV = record_values(D, KER);
    const size_t smem = (size_t)CAP * RV * sizeof(T);
    auto fn = k_nw_gather<T, D, KER>;   // tiles of one mesh
    static bool attr_set = false;   // set once, before any stream capture that uses it
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int N = a.N;
    dim3 grid((N + Tile<D>::X - 1) / Tile<D>::X, (N + Tile<D>::Y - 1) / Tile<D>::Y,
              D == 3 ? (N + Tile<D>::Z - 1) / Tile<D>::Z : 1);
    fn<<<grid, GT, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- PSI-CELL

struct PsiArgs {
    const void* state;
    const uint32_t* meta;
    const fla_batch* batches;
    const uint32_t* perm;
    const uint32_t* bin_start;
    int64_t n, n_cells;
    double inv_window;
    void* rec;
    DevStatus* status;
};

// Gather w * acc / T_window of each binned parcel into sorted order (4 values).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_psi_records(PsiArgs a)
{
    constexpr int OA = acc_offset(FLA_CLOUD_LPT, D);
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    if (j >= nvalid) return;
    const uint32_t i = a.perm[j];
    const double w = __ldg(&a.batches[a.meta[i] & FLA_META_BATCH_MASK].n0);
    T v0[4], v1[4], out[4];
    load4<T>((const T*)a.state, (OA / 4) * a.n + i, v0);
    if (OA % 4 + D + 1 > 4) load4<T>((const T*)a.state, (OA / 4 + 1) * a.n + i, v1);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = T(0);
#pragma unroll
    for (int q = 0; q <= D; ++q) {
        const int o = OA % 4 + q;
        const T v = o < 4 ? v0[o] : v1[o - 4];
        // single precision stays single: double arithmetic runs on the slow FP64 pipe
        out[q] = sizeof(T) == 4 ? T((float)w * (float)v * (float)a.inv_window) : T(w * (double)v * a.inv_window);
    }
    store4<T>((T*)a.rec, j, out);
}

// One warp per cell: fixed lane assignment and a butterfly reduction.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_psi_cells(const T* __restrict__ rec, const uint32_t* __restrict__ bin_start,
                                                   int64_t n_cells, T scale, uint32_t* __restrict__ counts,
                                                   T* __restrict__ s_mass, T* __restrict__ s_mom)
{
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n_cells) return;
    const uint32_t beg = bin_start[c], end = bin_start[c + 1];
    T s[4] = {T(0), T(0), T(0), T(0)};
    for (uint32_t j = beg + lane; j < end; j += 32) {
        T v[4];
        load4<T>(rec, j, v);
#pragma unroll
        for (int q = 0; q <= D; ++q) s[q] += v[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q <= D; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) {
        counts[c] = end - beg;
        s_mass[c] = -scale * s[0];
#pragma unroll
        for (int q = 0; q < D; ++q) s_mom[q * n_cells + c] = -scale * s[1 + q];
    }
}

}  // namespace

cudaError_t launch_nw_gather(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg, const void* rec,
                             const uint32_t* bin_start, const unsigned int* ext_max, const fla_sources& out,
                             DevStatus* st, cudaStream_t s)
{
    GatherArgs a{};
    a.status = st;
    a.rec = rec;
    a.bin_start = bin_start;
    a.ext_max = ext_max;
    a.N = m.n;
    a.per_cell = cfg.per_cell;
    a.s_mass = out.s_mass_dev;
    a.s_mom = out.s_mom_dev;
    a.dsum = out.dsum_dev;
    const bool iso = cfg.kernel == FLA_KERNEL_ISO;
    if (cl.dtype == FLA_F32) {
        if (m.dim == 2) return iso ? launch_gather_t<float, 2, 0>(a, s) : launch_gather_t<float, 2, 1>(a, s);
        return iso ? launch_gather_t<float, 3, 0>(a, s) : launch_gather_t<float, 3, 1>(a, s);
    }
    if (m.dim == 2) return iso ? launch_gather_t<double, 2, 0>(a, s) : launch_gather_t<double, 2, 1>(a, s);
    return iso ? launch_gather_t<double, 3, 0>(a, s) : launch_gather_t<double, 3, 1>(a, s);
}

cudaError_t launch_psicell(const fla_cloud& cl, const fla_mesh& m, double window_dt, int per_cell,
                           const uint32_t* perm, const uint32_t* bin_start, void* rec, const fla_psicell_out& out,
                           DevStatus* st, cudaStream_t s)
{
    const int64_t nc = m.dim == 2 ? (int64_t)m.n * m.n : (int64_t)m.n * m.n * m.n;
    PsiArgs a{};
    a.state = cl.state_dev;
    a.meta = cl.meta_dev;
    a.batches = cl.batches_dev;
    a.perm = perm;
    a.bin_start = bin_start;
    a.n = cl.n;
    a.n_cells = nc;
    a.inv_window = 1.0 / window_dt;
    a.rec = rec;
    a.status = st;
    const double dx = 1.0 / m.n;
    const double V = m.dim == 2 ? dx * dx : dx * dx * dx;
    const double scale = per_cell ? 1.0 : 1.0 / V;
    const unsigned rb = (unsigned)((cl.n + 255) / 256);
    const unsigned cb = (unsigned)((nc * 32 + 255) / 256);
    if (cl.dtype == FLA_F32) {
        if (cl.n > 0) {
            if (m.dim == 2) k_psi_records<float, 2><<<rb, 256, 0, s>>>(a);
            else k_psi_records<float, 3><<<rb, 256, 0, s>>>(a);
        }
        if (m.dim == 2)
            k_psi_cells<float, 2><<<cb, 256, 0, s>>>((const float*)rec, bin_start, nc, (float)scale, out.counts_dev,
                                                     (float*)out.s_mass_dev, (float*)out.s_mom_dev);
        else
            k_psi_cells<float, 3><<<cb, 256, 0, s>>>((const float*)rec, bin_start, nc, (float)scale, out.counts_dev,
                                                     (float*)out.s_mass_dev, (float*)out.s_mom_dev);
    } else {
        if (cl.n > 0) {
            if (m.dim == 2) k_psi_records<double, 2><<<rb, 256, 0, s>>>(a);
            else k_psi_records<double, 3><<<rb, 256, 0, s>>>(a);
        }
        if (m.dim == 2)
            k_psi_cells<double, 2><<<cb, 256, 0, s>>>((const double*)rec, bin_start, nc, scale, out.counts_dev,
                                                      (double*)out.s_mass_dev, (double*)out.s_mom_dev);
        else
            k_psi_cells<double, 3><<<cb, 256, 0, s>>>((const double*)rec, bin_start, nc, scale, out.counts_dev,
                                                      (double*)out.s_mass_dev, (double*)out.s_mom_dev);
    }
    return cudaGetLastError();
}

namespace {
template <int D, int KER>
cudaError_t launch_batch_gather_t(const BatchDev& b, int group, int ctas, DevStatus* st, cudaStream_t s)
{
    constexpr int RV = record_values(D, KER);
    const size_t smem = (size_t)CAP * RV * sizeof(float);
    auto fn = k_batch_gather<D, KER>;   // shared-memory attribute set by batch_prepare_gathers
    cudaError_t e = cudaMemsetAsync(b.tile_counter + group, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    fn<<<ctas, GT, smem, s>>>(b, group, st);
    return cudaGetLastError();
}
}  // namespace

template <int D, int KER>
cudaError_t prepare_gather_t()
{
    constexpr int RV = record_values(D, KER);
    return cudaFuncSetAttribute(k_batch_gather<D, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)CAP * RV * sizeof(float)));
}

// Shared-memory limits of the batched gathers (and their modules loaded), set
// once when a plan is created, before any launch or capture.
cudaError_t batch_prepare_gathers()
{
    cudaError_t e = prepare_gather_t<2, FLA_KERNEL_ISO>();
    if (e == cudaSuccess) e = prepare_gather_t<2, FLA_KERNEL_ANISO>();
    if (e == cudaSuccess) e = prepare_gather_t<3, FLA_KERNEL_ISO>();
    if (e == cudaSuccess) e = prepare_gather_t<3, FLA_KERNEL_ANISO>();
    return e;
}

cudaError_t launch_batch_gather(const BatchDev& b, int group, int ctas, DevStatus* st, cudaStream_t s)
{
    if (b.n_tiles[group] == 0) return cudaSuccess;
    if (ctas > b.n_tiles[group]) ctas = b.n_tiles[group];
    switch (group) {
    case 0: return launch_batch_gather_t<2, FLA_KERNEL_ISO>(b, group, ctas, st, s);
    case 1: return launch_batch_gather_t<2, FLA_KERNEL_ANISO>(b, group, ctas, st, s);
    case 2: return launch_batch_gather_t<3, FLA_KERNEL_ISO>(b, group, ctas, st, s);
    default: return launch_batch_gather_t<3, FLA_KERNEL_ANISO>(b, group, ctas, st, s);
    }
}

}  // namespace fla
