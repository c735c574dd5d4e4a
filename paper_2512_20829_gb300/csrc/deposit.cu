// Kernel-regression gather (Eqs. 13 and 16) and PSI-CELL box counting (Eqs. 10-11).
//
// Gather: tiles of cells (16x16 in 2D, 8x8x4 in 3D), one cell per thread of
// a CTA, each warp owning a 32-cell sub-tile.  Droplet records are sorted by
// cell key, so the records of the cells in one mesh row of the tile's
// neighbourhood are contiguous; a tile's candidates are those rows' records
// in row order, cut into work items (below) that persistent CTAs take.  A CTA
// walks its item's candidates, each thread loads one record, records whose
// support cannot reach the tile are culled, and the survivors are compacted
// (order kept) into shared memory with a mask of the warp sub-tiles each can
// reach (support sphere, and for the J-scaled kernel the support's bounding
// box).  Each warp then selects, 32 staged records at a time with one ballot
// over their masks, the records that reach its own sub-tile and evaluates
// only those: truncation test (as a predicate), Gaussian weight
// 2^(c r^2 + log2(1/h)) with one MUFU ex2 in single precision, FMA
// accumulation.  Each staged chunk (up to 1,024 records) is summed plainly and
// chunk sums are added with Neumaier compensation.  Every cell sums its records
// in staging order and no atomics touch the outputs, so results are
// deterministic.
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

// CTA tile of cells and the per-warp sub-tile (32 cells, one per lane).  A
// tile's candidates arrive in mesh-row order (x rows, y inner, z outer), so a
// staged chunk holds records of a few neighbouring rows: it spans the tile in
// x but only part of it in y and z.  The sub-tiles therefore split the tile
// four ways in x, two in y and not in z (3D: 2 x 4 x 4 cells), so that every
// warp finds records of its own in most chunks; with 4 x 4 x 2 sub-tiles
// (two per axis) the warps whose z half the chunk missed idled at the chunk's
// barrier.  A support reaches as many sub-tiles either way.
template <int D> struct Tile;
template <> struct Tile<2> {
    static constexpr int X = 16, Y = 16, Z = 1;      // 8 warps of 4 x 8 cells
    static constexpr int SX = 4, SY = 8, SZ = 1;
    static constexpr int NSX = 4, NSY = 2, NSZ = 1;
};
template <> struct Tile<3> {
    static constexpr int X = 8, Y = 8, Z = 4;        // 8 warps of 2 x 4 x 4 cells
    static constexpr int SX = 2, SY = 4, SZ = 4;
    static constexpr int NSX = 4, NSY = 2, NSZ = 1;
};

constexpr int GT = 256;            // threads per CTA = cells per tile
constexpr int CAP = 4 * GT;        // staged records (1,024: 4-5 % faster than 512 on the ABC cone)

// The x cells of mesh row (y, z) whose records can reach the tile with origin
// t0: a record in a cell dq cells away from the tile's cells along axis q lies
// at least (dq - 1/2) cells from the box of their centres (0 for dq = 0), and
// a record reaches the tile only within its support radius of that box (the
// staging test: d^2 <= ext (1 + 2^-10)).  rr2 = (largest such radius in cells)^2
// with that margin.  Returns false for a row no record of which can reach it.
// The plan and the gather both call this and must agree on every row to the
// bit, so each operation is rounded explicitly (no contraction that could
// differ between the two call sites).
template <int D>
__device__ __forceinline__ bool row_xrange(int N, const int t0[3], int y, int z, float rr2, int& xlo, int& xhi)
{
    constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
    const int dy = max(max(t0[1] - y, y - (t0[1] + TY - 1)), 0);
    const int dz = D == 3 ? max(max(t0[2] - z, z - (t0[2] + TZ - 1)), 0) : 0;
    const float ey = dy > 0 ? (float)dy - 0.5f : 0.0f, ez = dz > 0 ? (float)dz - 0.5f : 0.0f;
    const float rem = __fsub_rn(__fsub_rn(rr2, __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    if (!(rem >= 0.0f)) return false;
    // dx - 1/2 <= sqrt(rem), with a little slack over the float rounding
    const int xr = (int)floorf(__fadd_rn(__fmul_rn(__fsqrt_rn(rem), 1.0001f), 0.501f));
    xlo = max(t0[0] - xr, 0);
    xhi = min(t0[0] + TX - 1 + xr, N - 1);
    return xlo <= xhi;
}

// (largest support radius in cells)^2 with the staging test's margin, from the
// cloud's largest squared support radius ext2max
__device__ __forceinline__ float row_radius2(float ext2max, int N)
{
    const float n = (float)N;
    return __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(ext2max, 1.0009765625f), n), n), 1.0001f);
}

// Rows of a tile's neighbourhood on each side: the largest support radius in
// cells, rounded up with a cell to spare (rounded explicitly, as row_xrange).
__device__ __forceinline__ int support_rows(float ext2max, int N)
{
    return (int)floorf(__fadd_rn(__fmul_rn(__fsqrt_rn(ext2max), (float)N), 0.5f)) + 1;
}

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

// Bounds of a J-scaled record's truncated support {d : d' P d <= 9} (P = Sigma^-1):
//  * W2: squared half-widths per axis of the axis-aligned box that holds it,
//    9 Sigma_qq = 9 C_qq / det P (C the cofactors of P);
//  * a separating axis against a box: with b the offset from the record to the
//    box's nearest point, every point p of the box has (p - x).b >= |b|^2 (the
//    box is convex), while the support reaches 3 sqrt(b' Sigma b) / |b| along b
//    at most; so it misses the box when |b|^4 > 9 b' Sigma b = grow' b' C b.
//    The support's longest axis is often a third of the sphere of radius
//    3 sqrt(tr Sigma) that bounds it, which this test cuts down to the
//    ellipsoid's own extent towards the box.
// The margin in grow covers the rounding of the single- or double-precision
// evaluation and of these bounds; it grows with a bound on the condition
// number of Sigma, kappa <= tr(Sigma)^D det(P).  Where that bound is large or
// P is not positive definite, neither bound is used (valid = false) and the
// sphere test alone decides.  The spherical kernel needs neither: its sphere
// test is exact.
template <typename T>
struct SupportBounds {
    T W2[3];
    T C[6];        // cofactors c00, c11, c22, c01, c02, c12 (2D: c00, c11, c01 in slots 0, 1, 3)
    T grow;        // 9 (1 + margin) / det P
    bool valid;
};

template <typename T, int D, int KER>
__device__ __forceinline__ SupportBounds<T> support_bounds(const T* r)
{
    SupportBounds<T> s;
    s.W2[0] = s.W2[1] = s.W2[2] = T(INFINITY);
    s.valid = false;
    if (KER == FLA_KERNEL_ISO) return s;
    const T eps = sizeof(T) == 4 ? T(5.9604644775390625e-8) : T(1.1102230246251565e-16);
    T det;
    if (D == 2) {
        const T a = r[4], b = r[5], c = r[6];
        det = a * c - b * b;
        s.C[0] = c;
        s.C[1] = a;
        s.C[2] = T(0);
        s.C[3] = -b;
        s.C[4] = s.C[5] = T(0);
    } else {
        const T p00 = r[4], p01 = r[5], p02 = r[6], p11 = r[7], p12 = r[8], p22 = r[9];
        const T c00 = p11 * p22 - p12 * p12, c11 = p00 * p22 - p02 * p02, c22 = p00 * p11 - p01 * p01;
        const T c01 = p12 * p02 - p01 * p22, c02 = p01 * p12 - p11 * p02, c12 = p01 * p02 - p00 * p12;
        det = p00 * c00 + p01 * c01 + p02 * c02;
        s.C[0] = c00;
        s.C[1] = c11;
        s.C[2] = c22;
        s.C[3] = c01;
        s.C[4] = c02;
        s.C[5] = c12;
    }
    const T tr = r[ExtSlot<D, KER>::v] * T(1.0 / 9.0);
    const T kb = (D == 2 ? tr * tr : tr * tr * tr) * det;
    if (!(det > T(0)) || !(kb <= T(1e4))) return s;
    s.grow = T(9) * (T(1) + T(0.0009765625) + T(64) * kb * eps) / det;
    if (!(s.grow < T(INFINITY))) return s;
    s.valid = true;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const T w2 = s.C[q] * s.grow;
        if (w2 >= T(0) && w2 < T(INFINITY)) s.W2[q] = w2;
    }
    return s;
}

// The warp sub-tiles of a tile that a staged record can reach: bit w set when
// the record's support sphere (radius^2 in slot EXT, with the 2^-10 margin of
// the tile test) reaches sub-tile w's box of cell centres and, for the J-scaled
// kernel, its support box overlaps that box and no separating axis (above)
// splits them.  slab[q][s] = {lo, hi} of the s-th slab of sub-tiles along
// axis q (Tile<D>::NSX, NSY, NSZ of them).
template <typename T, int D, int KER>
__device__ __forceinline__ unsigned subtile_mask(const T* rv, const T (*slab)[4][2])
{
    constexpr int NSX = Tile<D>::NSX, NSY = Tile<D>::NSY, NSZ = Tile<D>::NSZ;
    const SupportBounds<T> sb = support_bounds<T, D, KER>(rv);
    const T e2m = rv[ExtSlot<D, KER>::v] * T(1.0009765625);
    T ba_[NSX], bb_[NSY], bc_[NSZ];   // signed offsets to the nearest point of each slab
    auto off = [&](int q, int sl) {
        const T dl = slab[q][sl][0] - rv[q], dh = rv[q] - slab[q][sl][1];
        return dl > T(0) ? dl : (dh > T(0) ? -dh : T(0));
    };
#pragma unroll
    for (int sl = 0; sl < NSX; ++sl) ba_[sl] = off(0, sl);
#pragma unroll
    for (int sl = 0; sl < NSY; ++sl) bb_[sl] = off(1, sl);
#pragma unroll
    for (int sl = 0; sl < NSZ; ++sl) bc_[sl] = D == 3 ? off(2, sl) : T(0);
    unsigned m = 0;
#pragma unroll
    for (int w = 0; w < GT / 32; ++w) {
        const int sx = w % NSX, sy = (w / NSX) % NSY, sz = w / (NSX * NSY);
        const T bx = ba_[sx], by = bb_[sy], bz = bc_[sz];
        const T xx = bx * bx, yy = by * by, zz = bz * bz;
        const T d2 = D == 3 ? xx + yy + zz : xx + yy;
        bool hit = d2 <= e2m;
        if (KER != FLA_KERNEL_ISO && sb.valid) {
            hit = hit && xx <= sb.W2[0] && yy <= sb.W2[1] && (D == 2 || zz <= sb.W2[2]);
            T qf = sb.C[0] * xx + sb.C[1] * yy + T(2) * sb.C[3] * (bx * by);
            if (D == 3) qf += sb.C[2] * zz + T(2) * (sb.C[4] * (bx * bz) + sb.C[5] * (by * bz));
            hit = hit && d2 * d2 <= sb.grow * qf;
        }
        if (hit) m |= 1u << w;
    }
    return m;
}

// Cell of thread tid in the tile with origin t0: warp = sub-tile, lane = cell.
template <int D>
__device__ __forceinline__ void tile_cell(int tid, const int t0[3], int w0[3], int cc[3])
{
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int SX = Tile<D>::SX, SY = Tile<D>::SY, SZ = Tile<D>::SZ;
    constexpr int NSX = Tile<D>::NSX, NSY = Tile<D>::NSY;
    static_assert(SX * SY * SZ == 32 && Tile<D>::NSX * Tile<D>::NSY * Tile<D>::NSZ == GT / 32, "sub-tiles");
    static_assert(NSX <= 4 && NSY <= 4 && Tile<D>::NSZ <= 4, "at most 4 slabs per axis");
    w0[0] = t0[0] + (warp % NSX) * SX;
    w0[1] = t0[1] + ((warp / NSX) % NSY) * SY;
    w0[2] = D == 3 ? t0[2] + (warp / (NSX * NSY)) * SZ : 0;
    cc[0] = w0[0] + lane % SX;
    cc[1] = w0[1] + (lane / SX) % SY;
    cc[2] = D == 3 ? w0[2] + lane / (SX * SY) : 0;
}

// Source terms of one cell from its weight sum Dt and weighted sums Nq (Eq. 13).
template <typename T, int D>
__device__ __forceinline__ void write_cell(const GatherArgs& a, const int cc[3], T Dt, const T Nq[4])
{
    const int N = a.N;
    const int64_t cell = cc[0] + (int64_t)N * (cc[1] + (D == 3 ? (int64_t)N * cc[2] : 0));
    const int64_t nc = D == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    T scale = T(1);
    if (a.per_cell) {
        const double dx = 1.0 / N;
        scale = T(D == 2 ? dx * dx : dx * dx * dx);
    }
    const bool cov = Dt > T(0);
    ((T*)a.s_mass)[cell] = cov ? -Nq[0] / Dt * scale : T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) ((T*)a.s_mom)[q * nc + cell] = cov ? -Nq[1 + q] / Dt * scale : T(0);
    if (a.dsum) ((T*)a.dsum)[cell] = Dt;
}

// The candidates [c0, c1) of one CTA tile of cells with origin (tx0, ty0, tz0).
// The candidates of a tile are the records of the mesh rows within R of it
// (R from the largest support in the cloud), concatenated in row order (z
// outer, y inner).  part == nullptr: the tile is one work item and the source
// terms are written; otherwise the item's D + 2 sums per cell go to part
// (value-major, GT cells each).
template <typename T, int D, int KER>
__device__ __forceinline__ void gather_tile(const GatherArgs& a, int tx0, int ty0, int tz0, uint32_t c0, uint32_t c1,
                                            T* part)
{
    constexpr int RV = record_values(D, KER);
    constexpr int R4 = RV / 4;
    constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
    constexpr int SX = Tile<D>::SX, SY = Tile<D>::SY, SZ = Tile<D>::SZ;
    constexpr int EXT = ExtSlot<D, KER>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* srec = reinterpret_cast<T*>(smem_raw);
    __shared__ int s_wcount[2][GT / 32];          // kept records per warp, double-buffered by chunk
    __shared__ uint32_t s_rbeg[GT], s_rexc[GT];   // a batch of rows: segment start, candidates before it
    __shared__ uint32_t s_wsum[GT / 32];
    __shared__ uint8_t s_mask[CAP];               // per staged record: the warp sub-tiles it reaches
    __shared__ T s_slab[3][4][2];                 // sub-tile slabs of cell centres per axis

    const int N = a.N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0[3] = {tx0, ty0, tz0};
    int w0[3], cc[3];
    tile_cell<D>(tid, t0, w0, cc);
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
    // box of cell centres of the CTA tile (staging cull) and the sub-tile slabs (flush masks)
    T lo[3], hi[3];
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const int tq = q == 0 ? TX : (q == 1 ? TY : TZ);
        const int last = (t0[q] + tq < N ? t0[q] + tq : N) - 1;
        lo[q] = centre(t0[q]);
        hi[q] = centre(last);
    }
    if (tid < 3 * 4 * 2) {
        const int q = tid >> 3, sl = (tid >> 1) & 3, end = tid & 1;
        const int sq = q == 0 ? SX : (q == 1 ? SY : SZ);
        const int first = (q == 0 ? tx0 : (q == 1 ? ty0 : tz0)) + sl * sq;
        const int last = (first + sq < N ? first + sq : N) - 1;
        s_slab[q][sl][end] = centre(end ? last : first);
    }
    const float ext2max = __uint_as_float(ldro(a.ext_max));
    const int R = support_rows(ext2max, N);
    const float rr2 = row_radius2(ext2max, N);

    T sD = T(0), cD = T(0);
    T sN[4] = {T(0), T(0), T(0), T(0)}, cN[4] = {T(0), T(0), T(0), T(0)};
    int npairs = 0;
    int count = 0;      // staged records (the same in every thread)
    int wbuf = 0;       // s_wcount buffer of the current chunk

    const int ylo = t0[1] - R < 0 ? 0 : t0[1] - R;
    const int yhi = t0[1] + TY - 1 + R > N - 1 ? N - 1 : t0[1] + TY - 1 + R;
    int zlo = 0, zhi = 0;
    if (D == 3) {
        zlo = t0[2] - R < 0 ? 0 : t0[2] - R;
        zhi = t0[2] + TZ - 1 + R > N - 1 ? N - 1 : t0[2] + TZ - 1 + R;
    }
    const int ny = yhi - ylo + 1;
    const int nrows = ny * (zhi - zlo + 1);
    __syncthreads();

    // Evaluate the staged records for this warp's cells in staging order: for 32
    // records at a time each lane reads one record's sub-tile mask (set when it was
    // staged), one ballot selects those that reach this warp's sub-tile, and
    // every lane evaluates only those.
    auto flush = [&](int count) {
        if (!warp_live) return;
        T pD = T(0), pN[4] = {T(0), T(0), T(0), T(0)};
        for (int k0 = 0; k0 < count; k0 += 32) {
            const int k = k0 + lane;
            const bool ov = k < count && ((s_mask[k] >> warp) & 1u);
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

    // Walk the candidates [c0, c1) a batch of GT rows at a time: each thread reads
    // one row's segment, a CTA scan gives the candidates before each row, and then
    // GT consecutive candidates at a time are loaded (thread j finds the row of
    // candidate j by binary search), culled against the tile and staged in order.
    uint32_t off = 0;   // candidates before the current batch of rows
    for (int rb = 0; rb < nrows && off < c1; rb += GT) {
        const int r = rb + tid;
        uint32_t beg = 0, len = 0;
        int rxlo, rxhi;
        if (r < nrows && row_xrange<D>(N, t0, ylo + r % ny, zlo + r / ny, rr2, rxlo, rxhi)) {
            const int y = ylo + r % ny, z = zlo + r / ny;
            const int64_t rowbase = ((int64_t)z * N + y) * N;
            beg = ldro(a.bin_start + rowbase + rxlo);
            len = ldro(a.bin_start + rowbase + rxhi + 1) - beg;
        }
        uint32_t x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += v;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0, btotal = 0;
#pragma unroll
        for (int w2 = 0; w2 < GT / 32; ++w2) {
            const uint32_t v = s_wsum[w2];
            wpre += w2 < warp ? v : 0u;
            btotal += v;
        }
        s_rbeg[tid] = beg;
        s_rexc[tid] = wpre + x - len;
        __syncthreads();
        const uint32_t jlo = c0 > off ? c0 - off : 0u;
        const uint32_t jhi = c1 - off < btotal ? c1 - off : btotal;
        for (uint32_t j0 = jlo; j0 < jhi; j0 += GT) {
            const uint32_t j = j0 + tid;
            T rv[16];
            bool keep = false;
            unsigned msk = 0u;
            if (j < jhi) {
                int rl = 0, rh = GT - 1;   // last row with s_rexc <= j
                while (rl < rh) {
                    const int mid = (rl + rh + 1) >> 1;
                    if (s_rexc[mid] <= j) rl = mid;
                    else rh = mid - 1;
                }
                const int64_t pos = (int64_t)(s_rbeg[rl] + (j - s_rexc[rl])) - a.rec_base;
#pragma unroll
                for (int v = 0; v < R4; ++v) load4<T>((const T*)a.rec, pos * R4 + v, rv + 4 * v);
                T d2 = T(0);
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    const T dl = lo[q] - rv[q], dh = rv[q] - hi[q];
                    const T dd = dl > T(0) ? dl : (dh > T(0) ? dh : T(0));
                    d2 += dd * dd;
                }
                keep = d2 <= rv[EXT] * T(1.0009765625);   // small margin over rounding of the test
                if (keep) {
                    msk = subtile_mask<T, D, KER>(rv, s_slab);
                    keep = msk != 0u;
                }
            }
            const unsigned ballot = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_wcount[wbuf][warp] = __popc(ballot);
            __syncthreads();
            // Records are appended after the staged ones, which nothing reads until a
            // flush, and the counts alternate between two buffers (a warp can reach
            // this chunk's buffer again only after every warp has passed the next
            // chunk's barrier): one barrier per chunk unless the stage is flushed.
            int pos0 = count, total = count;
#pragma unroll
            for (int w2 = 0; w2 < GT / 32; ++w2) {
                const int c = s_wcount[wbuf][w2];
                pos0 += w2 < warp ? c : 0;
                total += c;
            }
            wbuf ^= 1;
            if (keep) {
                const int pos = pos0 + __popc(ballot & ((1u << lane) - 1u));
#pragma unroll
                for (int v = 0; v < R4; ++v) store4<T>(srec, (int64_t)pos * R4 + v, rv + 4 * v);
                s_mask[pos] = (uint8_t)msk;
            }
            if (total > CAP - GT) {
                __syncthreads();   // the staged records are complete
                flush(total);
                __syncthreads();   // every warp has read them before they are overwritten
                total = 0;
            }
            count = total;
        }
        off += btotal;
        __syncthreads();   // the row batch's tables are rewritten next
    }
    __syncthreads();
    if (count > 0) flush(count);

    // pairs inside the truncation (cells of the mesh only): one atomic per CTA
    {
        const int w = __reduce_add_sync(0xffffffffu, in_mesh ? npairs : 0);
        __syncthreads();
        if (lane == 0) s_wcount[0][warp] = w;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int q = 0; q < GT / 32; ++q) t += s_wcount[0][q];
            if (t) atomicAdd(&a.status->pairs, (unsigned long long)t);
        }
    }

    if (in_mesh) {
        if (part) {
            part[tid] = sD + cD;
#pragma unroll
            for (int q = 0; q <= D; ++q) part[(1 + q) * GT + tid] = sN[q] + cN[q];
        } else {
            T Nq[4];
#pragma unroll
            for (int q = 0; q <= D; ++q) Nq[q] = sN[q] + cN[q];
            write_cell<T, D>(a, cc, sD + cD, Nq);
        }
    }
}

// ------------------------------------------------------------ work items
//
// A tile whose candidate list is long (a dense cluster of droplets, or a wide
// support) would hold one CTA for as long as the rest of the mesh takes.  A
// plan kernel therefore counts each tile's candidates and cuts the list into
// work items of about `chunk` candidates; persistent CTAs take items from
// a counter, and the items of a tile leave per-cell partial sums that a
// combine kernel adds in item order (Neumaier-compensated) before dividing.
// A tile of one item writes its cells directly.  The item budget of a cloud
// is its tiles plus min(ceil(16 n / chunk) + 1, 65,536); when the candidates
// need more, the cloud's chunk grows so that its items fit.  Item boundaries
// depend only on the candidate counts, so the result is deterministic and the
// same for a cloud gathered alone or in a batch.

struct NwItems {
    // tile source: a batch tile table (clouds != nullptr) or the tile grid of one mesh
    const BatchTile* tiles;
    const BatchCloud* clouds;
    const uint32_t* bin_start;        // batch: bin starts of all clouds (cloud k from cell_off)
    const unsigned int* ext_max;      // per cloud
    int N, per_cell, tiles_x, tiles_y;
    int64_t n_drops;                  // one mesh: droplets (item budget)
    void* s_mass;
    void* s_mom;
    void* dsum;
    // records
    const void* rec;
    const uint32_t* rec_base_at;      // batch: sorted position of rec[0] (device); else 0
    // plan and items
    int n_tiles, cloud_lo, cloud_hi;  // tiles; clouds whose totals the plan resets
    uint32_t* tile_cand;              // n_tiles
    uint32_t* tile_items;             // n_tiles + 1 (exclusive prefix)
    unsigned long long* cloud_cand;   // per cloud: candidates of all its tiles (zero between plans)
    unsigned int* done;               // plan CTAs finished (reset by the last)
    unsigned int* counter;            // items taken (zeroed by the plan)
    void* temp;                       // item partials
    DevStatus* status;
    uint32_t chunk;                   // candidates per work item (nw_chunk)
};

struct TileRef {
    GatherArgs g;
    int o[3];
    int cloud;
    int64_t n;        // droplets of the cloud
};

template <int D>
__device__ __forceinline__ TileRef tile_ref(const NwItems& a, int t)
{
    TileRef r;
    r.g.rec = a.rec;
    r.g.rec_base = a.rec_base_at ? (int64_t)ldro(a.rec_base_at) : 0;
    r.g.status = a.status;
    if (a.clouds) {
        const BatchTile bt = a.tiles[t];
        const BatchCloud& c = a.clouds[bt.cloud];
        r.g.bin_start = a.bin_start + c.cell_off;
        r.g.ext_max = a.ext_max + bt.cloud;
        r.g.N = c.N;
        r.g.per_cell = c.per_cell;
        r.g.s_mass = c.s_mass;
        r.g.s_mom = c.s_mom;
        r.g.dsum = c.dsum;
        r.o[0] = bt.x0; r.o[1] = bt.y0; r.o[2] = bt.z0;
        r.cloud = bt.cloud;
        r.n = c.n;
    } else {
        r.g.bin_start = a.bin_start;
        r.g.ext_max = a.ext_max;
        r.g.N = a.N;
        r.g.per_cell = a.per_cell;
        r.g.s_mass = a.s_mass;
        r.g.s_mom = a.s_mom;
        r.g.dsum = a.dsum;
        r.o[0] = (t % a.tiles_x) * Tile<D>::X;
        r.o[1] = ((t / a.tiles_x) % a.tiles_y) * Tile<D>::Y;
        r.o[2] = (t / (a.tiles_x * a.tiles_y)) * Tile<D>::Z;
        r.cloud = 0;
        r.n = a.n_drops;
    }
    return r;
}

// Items beyond one per tile that a cloud may use: ceil(16 n / chunk) + 1, at
// most 65,536 (the partials of a 3D double-precision item are 10 KB); a cloud
// whose candidates need more widens its chunk instead.
__host__ __device__ inline int64_t nw_extra_items(int64_t n, uint32_t chunk)
{
    const int64_t e = (16 * (n > 0 ? n : 1) + chunk - 1) / chunk + 1;
    return e < 65536 ? e : 65536;
}

// Candidates of tile t (one warp; lanes over the neighbourhood rows).
template <int D>
__device__ __forceinline__ void nw_tile_cand(const NwItems& a, int t, int lane)
{
    const TileRef tr = tile_ref<D>(a, t);
    const int N = tr.g.N;
    const float ext2max = __uint_as_float(ldro(tr.g.ext_max));
    const int R = support_rows(ext2max, N);
    const float rr2 = row_radius2(ext2max, N);
    const int t0[3] = {tr.o[0], tr.o[1], tr.o[2]};
    const int ylo = max(tr.o[1] - R, 0), yhi = min(tr.o[1] + Tile<D>::Y - 1 + R, N - 1);
    const int zlo = D == 3 ? max(tr.o[2] - R, 0) : 0;
    const int zhi = D == 3 ? min(tr.o[2] + Tile<D>::Z - 1 + R, N - 1) : 0;
    const int ny = yhi - ylo + 1, nrows = ny * (zhi - zlo + 1);
    uint32_t cand = 0;
    for (int r = lane; r < nrows; r += 32) {
        int xlo, xhi;
        if (!row_xrange<D>(N, t0, ylo + r % ny, zlo + r / ny, rr2, xlo, xhi)) continue;
        const int64_t rb = ((int64_t)(zlo + r / ny) * N + ylo + r % ny) * N;
        cand += ldro(tr.g.bin_start + rb + xhi + 1) - ldro(tr.g.bin_start + rb + xlo);
    }
    cand = __reduce_add_sync(0xffffffffu, cand);
    if (lane == 0) {
        a.tile_cand[t] = cand;
        if (cand) atomicAdd(a.cloud_cand + tr.cloud, (unsigned long long)cand);
    }
}

// Item counts of every tile, max(1, ceil(cand / chunk)) with chunk =
// max(a.chunk, ceil(cloud candidates / extra items)), and their exclusive
// scan over the tiles (one CTA); the clouds' candidate totals are reset.
__device__ __forceinline__ void nw_item_scan(const NwItems& a)
{
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    uint32_t running = 0;
    for (int base = 0; base < a.n_tiles; base += blockDim.x) {
        const int tt = base + tid;
        uint32_t v = 0;
        if (tt < a.n_tiles) {
            const int k = a.clouds ? a.tiles[tt].cloud : 0;
            const int64_t nk = a.clouds ? a.clouds[k].n : a.n_drops;
            const unsigned long long tot = __ldcg(a.cloud_cand + k);
            const unsigned long long extra = (unsigned long long)nw_extra_items(nk, a.chunk);
            unsigned long long chunk = (tot + extra - 1) / extra;
            if (chunk < a.chunk) chunk = a.chunk;
            const unsigned long long cand = __ldcg(a.tile_cand + tt);
            v = cand ? (uint32_t)((cand + chunk - 1) / chunk) : 1u;
        }
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
        if (tt < a.n_tiles) a.tile_items[tt] = running + (w > 0 ? s_warp[w - 1] : 0) + x - v;
        running += s_warp[nw - 1];
        __syncthreads();
    }
    if (tid == 0) {
        a.tile_items[a.n_tiles] = running;
        *a.done = 0u;
    }
    for (int k = a.cloud_lo + tid; k < a.cloud_hi; k += blockDim.x) a.cloud_cand[k] = 0ull;
}

// Candidates of each tile; the last CTA to finish turns them into item counts
// and offsets.
template <int D>
__global__ void __launch_bounds__(256) k_nw_plan(NwItems a)
{
    pdl_entry();
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.counter = 0u;   // the items kernel's counter
    const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (t < a.n_tiles) nw_tile_cand<D>(a, t, threadIdx.x & 31);
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    nw_item_scan(a);
}

// Persistent CTAs: one work item at a time from the counter.
template <typename T, int D, int KER>
__device__ __forceinline__ void nw_items_loop(const NwItems& a)
{
    __shared__ uint32_t s_item;
    const uint32_t total = __ldcg(a.tile_items + a.n_tiles);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = a.n_tiles - 1;   // last tile with tile_items <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldcg(a.tile_items + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const int t = lo;
        const uint32_t i0 = __ldcg(a.tile_items + t), ni = __ldcg(a.tile_items + t + 1) - i0;
        const uint32_t cand = __ldcg(a.tile_cand + t);
        const uint32_t csize = (cand + ni - 1) / ni;
        const uint32_t c0 = (item - i0) * csize, c1 = min(c0 + csize, cand);
        const TileRef tr = tile_ref<D>(a, t);
        T* part = ni > 1 ? (T*)a.temp + (int64_t)item * (D + 2) * GT : nullptr;
        gather_tile<T, D, KER>(tr.g, tr.o[0], tr.o[1], tr.o[2], c0, c1, part);
    }
    __syncthreads();   // s_item is read by every thread before the CTA moves on
}

template <typename T, int D, int KER>
__global__ void __launch_bounds__(GT, sizeof(T) == 8 ? 1 : (D == 2 ? 3 : 2)) k_nw_items(NwItems a)
{
    pdl_entry();
    nw_items_loop<T, D, KER>(a);
}

// Tiles of several items: the items' partials of each cell in item order.
template <typename T, int D>
__device__ __forceinline__ void nw_combine_loop(const NwItems& a)
{
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const uint32_t i0 = __ldcg(a.tile_items + t), i1 = __ldcg(a.tile_items + t + 1);
        if (i1 - i0 <= 1) continue;
        const TileRef tr = tile_ref<D>(a, t);
        int w0[3], cc[3];
        tile_cell<D>(tid, tr.o, w0, cc);
        const int N = tr.g.N;
        if (!(cc[0] < N && cc[1] < N && (D == 2 || cc[2] < N))) continue;
        T s[D + 2], c[D + 2];
#pragma unroll
        for (int q = 0; q < D + 2; ++q) s[q] = c[q] = T(0);
        for (uint32_t it = i0; it < i1; ++it) {
            const T* p = (const T*)a.temp + (int64_t)it * (D + 2) * GT + tid;
#pragma unroll
            for (int q = 0; q < D + 2; ++q) neumaier(s[q], c[q], __ldcg(p + q * GT));
        }
        T Nq[4];
#pragma unroll
        for (int q = 0; q <= D; ++q) Nq[q] = s[1 + q] + c[1 + q];
        write_cell<T, D>(tr.g, cc, s[0] + c[0], Nq);
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(GT) k_nw_combine(NwItems a)
{
    pdl_entry();
    nw_combine_loop<T, D>(a);
}

template <typename T, int D, int KER>
size_t items_smem() { return (size_t)CAP * record_values(D, KER) * sizeof(T); }

// Shared-memory limit of the items kernel (set once, before any capture) and
// its resident CTAs per SM.
template <typename T, int D, int KER>
int items_prepare()
{
    static int per_sm = -1;
    if (per_sm < 0) {
        auto fn = k_nw_items<T, D, KER>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)items_smem<T, D, KER>()) !=
            cudaSuccess)
            return -1;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, GT, items_smem<T, D, KER>()) != cudaSuccess)
            return -1;
        per_sm = b > 0 ? b : 1;
    }
    return per_sm;
}

// Plan, items and combine of one tile set (one mesh, or one batch group).
template <typename T, int D, int KER>
cudaError_t launch_items_t(const NwItems& a, int ctas, int num_sms, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    const cudaError_t e = launch_pdl(k_nw_plan<D>, dim3((unsigned)(((int64_t)a.n_tiles * 32 + 255) / 256)), dim3(256), 0, s, a);
    if (e != cudaSuccess) return e;
    launch_pdl(k_nw_items<T, D, KER>, dim3(ctas), dim3(GT), items_smem<T, D, KER>(), s, a);
    const int cb = a.n_tiles < 8 * num_sms ? a.n_tiles : 8 * num_sms;
    launch_pdl(k_nw_combine<T, D>, dim3(cb), dim3(GT), 0, s, a);
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
    pdl_entry();
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
    pdl_entry();
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


// Cloud-In-Cell (CIC): each parcel's w * acc / T_window is spread over the
// cell centres around it with the tent weights prod_a (1 - |x_a - xc_a| N)^+,
// the overlap of a cell-sized cloud around the parcel with each cell.  The
// records pass writes, per sorted parcel, its position and w * acc / T (two
// vectors of 4); the cells pass takes one warp per cell over the parcels of
// the 3^D cells around it (the tent vanishes one cell away), in a fixed lane
// assignment with a butterfly reduction: deterministic, no float atomics.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_cic_records(PsiArgs a)
{
    pdl_entry();
    constexpr int OA = acc_offset(FLA_CLOUD_LPT, D);
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    if (j >= nvalid) return;
    const uint32_t i = a.perm[j];
    const double w = __ldg(&a.batches[a.meta[i] & FLA_META_BATCH_MASK].n0);
    T x[4], v0[4], v1[4], out[4];
    load4<T>((const T*)a.state, i, x);
    load4<T>((const T*)a.state, (OA / 4) * a.n + i, v0);
    if (OA % 4 + D + 1 > 4) load4<T>((const T*)a.state, (OA / 4 + 1) * a.n + i, v1);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = T(0);
#pragma unroll
    for (int q = 0; q <= D; ++q) {
        const int o = OA % 4 + q;
        const T v = o < 4 ? v0[o] : v1[o - 4];
        out[q] = sizeof(T) == 4 ? T((float)w * (float)v * (float)a.inv_window) : T(w * (double)v * a.inv_window);
    }
    if (D == 2) x[2] = T(0);
    x[3] = T(0);
    store4<T>((T*)a.rec, 2 * j, x);
    store4<T>((T*)a.rec, 2 * j + 1, out);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_cic_cells(const T* __restrict__ rec, const uint32_t* __restrict__ bin_start,
                                                   int N, T scale, uint32_t* __restrict__ counts,
                                                   T* __restrict__ s_mass, T* __restrict__ s_mom)
{
    pdl_entry();
    const int64_t nc = D == 2 ? (int64_t)N * N : (int64_t)N * N * N;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= nc) return;
    int ci[3] = {(int)(c % N), (int)((c / N) % N), D == 3 ? (int)(c / ((int64_t)N * N)) : 0};
    T xc[3];
#pragma unroll
    for (int q = 0; q < D; ++q) xc[q] = (T(ci[q]) + T(0.5)) / T(N);
    const T fN = T(N);
    T s[4] = {T(0), T(0), T(0), T(0)};
    const int zlo = D == 3 ? (ci[2] > 0 ? ci[2] - 1 : 0) : 0, zhi = D == 3 ? (ci[2] < N - 1 ? ci[2] + 1 : N - 1) : 0;
    const int ylo = ci[1] > 0 ? ci[1] - 1 : 0, yhi = ci[1] < N - 1 ? ci[1] + 1 : N - 1;
    const int xlo = ci[0] > 0 ? ci[0] - 1 : 0, xhi = ci[0] < N - 1 ? ci[0] + 1 : N - 1;
    for (int kz = zlo; kz <= zhi; ++kz)
        for (int ky = ylo; ky <= yhi; ++ky) {
            // the cells xlo..xhi of one row are contiguous in the sorted order
            const int64_t rb = ((int64_t)kz * N + ky) * N;
            const uint32_t beg = bin_start[rb + xlo], end = bin_start[rb + xhi + 1];
            for (uint32_t j = beg + lane; j < end; j += 32) {
                T p[4], v[4];
                load4<T>(rec, 2 * (int64_t)j, p);
                load4<T>(rec, 2 * (int64_t)j + 1, v);
                T W = T(1);
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    const T t = T(1) - fabs(p[q] - xc[q]) * fN;
                    W = t > T(0) ? W * t : T(0);
                }
#pragma unroll
                for (int q = 0; q <= D; ++q) s[q] = fma(W, v[q], s[q]);
            }
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q <= D; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) {
        counts[c] = bin_start[c + 1] - bin_start[c];
        s_mass[c] = -scale * s[0];
#pragma unroll
        for (int q = 0; q < D; ++q) s_mom[q * nc + c] = -scale * s[1 + q];
    }
}

template <typename T, int D, int KER>
cudaError_t launch_nw_t(const NwItems& a, int num_sms, cudaStream_t s)
{
    const int per_sm = items_prepare<T, D, KER>();
    if (per_sm < 0) return cudaErrorInvalidValue;
    return launch_items_t<T, D, KER>(a, per_sm * num_sms, num_sms, s);
}

}  // namespace

int nw_tiles(int dim, int N)
{
    if (dim == 2) return ((N + 15) / 16) * ((N + 15) / 16);
    return ((N + 7) / 8) * ((N + 7) / 8) * ((N + 3) / 4);
}

int64_t nw_item_budget(int dim, int N, int64_t n, size_t elem)
{
    return nw_tiles(dim, N) + nw_extra_items(n, nw_chunk(elem));
}

size_t nw_temp_bytes(int dim, int N, int64_t n, size_t elem)
{
    return (size_t)nw_item_budget(dim, N, n, elem) * (size_t)(dim + 2) * GT * elem;
}

cudaError_t launch_nw_gather(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg, const void* rec,
                             const uint32_t* bin_start, const unsigned int* ext_max, const NwWork& w,
                             const fla_sources& out, DevStatus* st, int num_sms, cudaStream_t s)
{
    NwItems a{};
    a.bin_start = bin_start;
    a.ext_max = ext_max;
    a.N = m.n;
    a.per_cell = cfg.per_cell;
    a.tiles_x = m.dim == 2 ? (m.n + 15) / 16 : (m.n + 7) / 8;
    a.tiles_y = a.tiles_x;
    a.n_drops = cl.n;
    a.s_mass = out.s_mass_dev;
    a.s_mom = out.s_mom_dev;
    a.dsum = out.dsum_dev;
    a.rec = rec;
    a.n_tiles = nw_tiles(m.dim, m.n);
    a.cloud_lo = 0;
    a.cloud_hi = 1;
    a.tile_cand = w.tile_cand;
    a.tile_items = w.tile_items;
    a.cloud_cand = w.cand_total;
    a.done = w.done;
    a.counter = w.counter;
    a.temp = w.temp;
    a.status = st;
    a.chunk = nw_chunk(cl.dtype == FLA_F64 ? 8 : 4);
    const bool iso = cfg.kernel == FLA_KERNEL_ISO;
    if (cl.dtype != FLA_F64) {
        if (m.dim == 2) return iso ? launch_nw_t<float, 2, 0>(a, num_sms, s) : launch_nw_t<float, 2, 1>(a, num_sms, s);
        return iso ? launch_nw_t<float, 3, 0>(a, num_sms, s) : launch_nw_t<float, 3, 1>(a, num_sms, s);
    }
    if (m.dim == 2) return iso ? launch_nw_t<double, 2, 0>(a, num_sms, s) : launch_nw_t<double, 2, 1>(a, num_sms, s);
    return iso ? launch_nw_t<double, 3, 0>(a, num_sms, s) : launch_nw_t<double, 3, 1>(a, num_sms, s);
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
    if (cl.dtype != FLA_F64) {
        if (cl.n > 0) {
            if (m.dim == 2) launch_pdl(k_psi_records<float, 2>, dim3(rb), dim3(256), 0, s, a);
            else launch_pdl(k_psi_records<float, 3>, dim3(rb), dim3(256), 0, s, a);
        }
        if (m.dim == 2)
            launch_pdl(k_psi_cells<float, 2>, dim3(cb), dim3(256), 0, s, (const float*)rec, bin_start, nc, (float)scale, out.counts_dev,
                                                     (float*)out.s_mass_dev, (float*)out.s_mom_dev);
        else
            launch_pdl(k_psi_cells<float, 3>, dim3(cb), dim3(256), 0, s, (const float*)rec, bin_start, nc, (float)scale, out.counts_dev,
                                                     (float*)out.s_mass_dev, (float*)out.s_mom_dev);
    } else {
        if (cl.n > 0) {
            if (m.dim == 2) launch_pdl(k_psi_records<double, 2>, dim3(rb), dim3(256), 0, s, a);
            else launch_pdl(k_psi_records<double, 3>, dim3(rb), dim3(256), 0, s, a);
        }
        if (m.dim == 2)
            launch_pdl(k_psi_cells<double, 2>, dim3(cb), dim3(256), 0, s, (const double*)rec, bin_start, nc, scale, out.counts_dev,
                                                      (double*)out.s_mass_dev, (double*)out.s_mom_dev);
        else
            launch_pdl(k_psi_cells<double, 3>, dim3(cb), dim3(256), 0, s, (const double*)rec, bin_start, nc, scale, out.counts_dev,
                                                      (double*)out.s_mass_dev, (double*)out.s_mom_dev);
    }
    return cudaGetLastError();
}

cudaError_t launch_cic(const fla_cloud& cl, const fla_mesh& m, double window_dt, int per_cell, const uint32_t* perm,
                       const uint32_t* bin_start, void* rec, const fla_psicell_out& out, DevStatus* st, cudaStream_t s)
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
    if (cl.dtype != FLA_F64) {
        if (cl.n > 0) {
            if (m.dim == 2) launch_pdl(k_cic_records<float, 2>, dim3(rb), dim3(256), 0, s, a);
            else launch_pdl(k_cic_records<float, 3>, dim3(rb), dim3(256), 0, s, a);
        }
        if (m.dim == 2)
            launch_pdl(k_cic_cells<float, 2>, dim3(cb), dim3(256), 0, s, (const float*)rec, bin_start, m.n,
                       (float)scale, out.counts_dev, (float*)out.s_mass_dev, (float*)out.s_mom_dev);
        else
            launch_pdl(k_cic_cells<float, 3>, dim3(cb), dim3(256), 0, s, (const float*)rec, bin_start, m.n,
                       (float)scale, out.counts_dev, (float*)out.s_mass_dev, (float*)out.s_mom_dev);
    } else {
        if (cl.n > 0) {
            if (m.dim == 2) launch_pdl(k_cic_records<double, 2>, dim3(rb), dim3(256), 0, s, a);
            else launch_pdl(k_cic_records<double, 3>, dim3(rb), dim3(256), 0, s, a);
        }
        if (m.dim == 2)
            launch_pdl(k_cic_cells<double, 2>, dim3(cb), dim3(256), 0, s, (const double*)rec, bin_start, m.n, scale,
                       out.counts_dev, (double*)out.s_mass_dev, (double*)out.s_mom_dev);
        else
            launch_pdl(k_cic_cells<double, 3>, dim3(cb), dim3(256), 0, s, (const double*)rec, bin_start, m.n, scale,
                       out.counts_dev, (double*)out.s_mass_dev, (double*)out.s_mom_dev);
    }
    return cudaGetLastError();
}

namespace {
template <int D, int KER>
cudaError_t launch_batch_gather_t(const BatchDev& b, int group, int ctas, DevStatus* st, int num_sms, cudaStream_t s)
{
    NwItems a{};
    a.tiles = b.tiles[group];
    a.clouds = b.clouds;
    a.bin_start = b.bin_start;
    a.ext_max = b.ext_max;
    a.rec = b.rec[group];
    a.rec_base_at = b.bin_start + b.group_cells[group];
    a.n_tiles = b.n_tiles[group];
    a.cloud_lo = b.group_first[group];
    a.cloud_hi = b.group_first[group + 1];
    a.tile_cand = b.tile_cand[group];
    a.tile_items = b.tile_items[group];
    a.cloud_cand = b.cloud_cand;
    a.done = b.plan_done + group;
    a.counter = b.tile_counter + group;
    a.temp = b.item_temp[group];
    a.status = st;
    a.chunk = nw_chunk(4);
    return launch_items_t<float, D, KER>(a, ctas, num_sms, s);
}
}  // namespace

// Shared-memory limits of the batched gathers (and their modules loaded), set
// once when a plan is created, before any launch or capture.
cudaError_t batch_prepare_gathers()
{
    const bool ok = items_prepare<float, 2, FLA_KERNEL_ISO>() > 0 && items_prepare<float, 2, FLA_KERNEL_ANISO>() > 0 &&
                    items_prepare<float, 3, FLA_KERNEL_ISO>() > 0 && items_prepare<float, 3, FLA_KERNEL_ANISO>() > 0;
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_batch_gather(const BatchDev& b, int group, int ctas, DevStatus* st, int num_sms, cudaStream_t s)
{
    if (b.n_tiles[group] == 0) return cudaSuccess;
    switch (group) {
    case 0: return launch_batch_gather_t<2, FLA_KERNEL_ISO>(b, group, ctas, st, num_sms, s);
    case 1: return launch_batch_gather_t<2, FLA_KERNEL_ANISO>(b, group, ctas, st, num_sms, s);
    case 2: return launch_batch_gather_t<3, FLA_KERNEL_ISO>(b, group, ctas, st, num_sms, s);
    default: return launch_batch_gather_t<3, FLA_KERNEL_ANISO>(b, group, ctas, st, num_sms, s);
    }
}

}  // namespace fla

#ifdef FLA_WINDOW_PHASES
// Gather phases of the persistent window kernel (window.cuh): the work-item
// tile gather of one batch group, as launch_batch_gather runs it.
#include <string.h>
#include "window.cuh"
namespace fla {

static_assert(sizeof(NwItems) <= sizeof(WindowBlob), "gather arguments fit the window's blob");

size_t window_gather_blob(WindowBlob* out, const BatchDev& b, int group, DevStatus* st, uint32_t chunk)
{
    NwItems a{};
    a.tiles = b.tiles[group];
    a.clouds = b.clouds;
    a.bin_start = b.bin_start;
    a.ext_max = b.ext_max;
    a.rec = b.rec[group];
    a.rec_base_at = b.bin_start + b.group_cells[group];
    a.n_tiles = b.n_tiles[group];
    a.cloud_lo = b.group_first[group];
    a.cloud_hi = b.group_first[group + 1];
    a.tile_cand = b.tile_cand[group];
    a.tile_items = b.tile_items[group];
    a.cloud_cand = b.cloud_cand;
    a.done = b.plan_done + group;
    a.counter = b.tile_counter + group;
    a.temp = b.item_temp[group];
    a.status = st;
    a.chunk = chunk;
    memset(out, 0, sizeof(*out));
    memcpy(out->b, &a, sizeof(a));
    return sizeof(a);
}

size_t window_items_smem()
{
    size_t m = items_smem<float, 2, FLA_KERNEL_ISO>();
    m = items_smem<float, 2, FLA_KERNEL_ANISO>() > m ? items_smem<float, 2, FLA_KERNEL_ANISO>() : m;
    m = items_smem<float, 3, FLA_KERNEL_ISO>() > m ? items_smem<float, 3, FLA_KERNEL_ISO>() : m;
    m = items_smem<float, 3, FLA_KERNEL_ANISO>() > m ? items_smem<float, 3, FLA_KERNEL_ANISO>() : m;
    return m;
}

__device__ void window_gather_cand(const WindowBlob& nw, int dim)
{
    const NwItems& a = *reinterpret_cast<const NwItems*>(nw.b);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.counter = 0u;   // the items phase's counter
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < a.n_tiles; t += warps) {
        if (dim == 2) nw_tile_cand<2>(a, (int)t, lane);
        else nw_tile_cand<3>(a, (int)t, lane);
    }
}

__device__ void window_gather_plan(const WindowBlob& nw, int)
{
    nw_item_scan(*reinterpret_cast<const NwItems*>(nw.b));
}

__device__ void window_gather_items(const WindowBlob& nw, int dim, int kernel, unsigned char*)
{
    const NwItems& a = *reinterpret_cast<const NwItems*>(nw.b);
    if (dim == 2) {
        if (kernel == FLA_KERNEL_ISO) nw_items_loop<float, 2, FLA_KERNEL_ISO>(a);
        else nw_items_loop<float, 2, FLA_KERNEL_ANISO>(a);
    } else {
        if (kernel == FLA_KERNEL_ISO) nw_items_loop<float, 3, FLA_KERNEL_ISO>(a);
        else nw_items_loop<float, 3, FLA_KERNEL_ANISO>(a);
    }
}

__device__ void window_gather_combine(const WindowBlob& nw, int dim)
{
    const NwItems& a = *reinterpret_cast<const NwItems*>(nw.b);
    if (dim == 2) nw_combine_loop<float, 2>(a);
    else nw_combine_loop<float, 3>(a);
}

}  // namespace fla
#endif
