// FLA / LPT advance: k fused RK4 steps per launch, one thread per droplet.
//
// Per droplet and step (Eqs. 3-5 and 8; App. B parcel level a-b):
//   x' = v,  v' = (u(x) - v)/St(t),  J' = W,  W' = (grad u(x) . J - W)/St(t),
//   St(t) = St0 (1 + delta (t - t0))  (d^2 law with r0 = 1),
// with window sums of mdot = 1.5 delta r and F + mdot v = m (u - v)/St + mdot v
// taken at the first RK stage.  The state stays in registers across the fused
// steps, so HBM is touched once per launch; the carrier node array (a few MB
// in 2D) is read through the L1/L2 caches by the interpolation gathers.
//
// Fold guard (single-precision FLA clouds with a fold array): near a fold
// caustic det J nearly vanishes (Eq. 6), so a droplet whose |det J| falls
// below tau integrates the J, W part of its RK4 step in double precision from
// the stage values of grad u and 1/St, keeping J, W in the fold array; it
// returns to single precision once |det J| exceeds 4 tau.  Two launches keep
// the common case at full speed: a screening pass integrates every droplet in
// single precision and tests det J at each step start; a droplet that is in
// the guard, or would enter it during the launch, is left untouched and
// appended to a list, and a second pass integrates the listed droplets from
// the same starting state with the guard logic.  The result equals one pass
// that applies the guard at every step.
//
// Compensated clouds (FLA_F32X2): every state value is a double-float
// hi + lo (two single-precision planes), the carrier nodes are double-float
// too, and the whole step -- cell fraction, interpolation weights and sums,
// 1/St, the right-hand side and the RK4 combinations -- runs in double-float
// arithmetic on the single-precision pipe.  Near a fold caustic n = n0/|det J|
// is ill-conditioned: single-precision rounding anywhere in the step (of the
// seed position, of the interpolated carrier, of the small differences u - v
// and grad u . J - W) moves det J by far more than its own size there, so the
// step as a whole has to carry more than single precision for n to match the
// double-precision method.  The window sums (a smooth average) stay single.
#include "batch.cuh"
#include "df32.cuh"

namespace fla {
namespace {

struct AdvArgs {
    void* state;
    uint32_t* meta;
    const fla_batch* batches;
    const void* nodes;
    int64_t n;
    int N;
    int step0, nsteps;
    double dt, delta;
    int reset;
    DevStatus* status;
    double* fold;        // fold-guard planes (FP64), or null
    uint32_t* fold_list; // droplets handed from the screening pass to the guarded pass
    unsigned int* fold_count;
    float tau_fold;
    const uint32_t* order; // thread t advances droplet order[t] (null: droplet t)
};

enum { kPlain = 0, kScreen = 1, kGuarded = 2 };

// The droplet of thread t: order[t] when an order is given (a permutation of
// [0, n), e.g. the cell-sorted one of the last binning, so that the droplets
// of a warp share carrier nodes), else t.  Entries out of range map to n (no
// droplet): a wrong order leaves droplets unadvanced but never reads or writes
// outside the cloud.
__device__ __forceinline__ int64_t droplet_of(const uint32_t* order, int64_t t, int64_t n)
{
    if (t >= n) return n;
    if (!order) return t;
    const int64_t i = (int64_t)__ldg(order + t);
    return i < n ? i : n;
}

// Double-precision J, W of one droplet in the fold guard, and its RK4 stage
// accumulators.
template <int D>
struct FoldState {
    double y[2 * D * D];    // J then W
    double ks[2 * D * D];
    double ys[2 * D * D];
};

template <int D>
struct StageG {
    float g[D * D];
};

template <int D>
__device__ __forceinline__ StageG<D> stage_g(const float* G)
{
    StageG<D> r;
#pragma unroll
    for (int q = 0; q < D * D; ++q) r.g[q] = G[q];
    return r;
}

// One RK4 stage of J' = W, W' = (G J - W)/St in double precision (Eq. 8).
// stage 0..3; hs = the stage's step (dt/2, dt/2, dt, and dt for the final combination).
template <int D>
__device__ __forceinline__ void fold_stage(FoldState<D>& f, StageG<D> G, float invSt, double hs, int stage)
{
    constexpr int Q = D * D;
    const double iS = (double)invSt;
    const double* src = stage == 0 ? f.y : f.ys;
    double k[2 * Q];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            double gj = 0.0;
#pragma unroll
            for (int j = 0; j < D; ++j) gj = fma((double)G.g[i * D + j], src[j * D + c], gj);
            k[i * D + c] = src[Q + i * D + c];
            k[Q + i * D + c] = (gj - src[Q + i * D + c]) * iS;
        }
    if (stage == 0) {
#pragma unroll
        for (int q = 0; q < 2 * Q; ++q) { f.ks[q] = k[q]; f.ys[q] = fma(hs, k[q], f.y[q]); }
    } else if (stage < 3) {
#pragma unroll
        for (int q = 0; q < 2 * Q; ++q) { f.ks[q] = fma(2.0, k[q], f.ks[q]); f.ys[q] = fma(hs, k[q], f.y[q]); }
    } else {
        const double sixth = hs / 6.0;
#pragma unroll
        for (int q = 0; q < 2 * Q; ++q) f.y[q] = fma(sixth, f.ks[q] + k[q], f.y[q]);
    }
}

template <int D>
__device__ __forceinline__ float det_f32(const float* J)
{
    if (D == 2) return J[0] * J[3] - J[1] * J[2];
    return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
           J[2] * (J[3] * J[7] - J[4] * J[6]);
}

template <int D>
__device__ __forceinline__ double fold_det(const FoldState<D>& f)
{
    const double* J = f.y;
    if (D == 2) return J[0] * J[3] - J[1] * J[2];
    return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
           J[2] * (J[3] * J[7] - J[4] * J[6]);
}

template <int D>
__device__ __forceinline__ void fold_load(FoldState<D>& f, const double* fold, int64_t n, int64_t i)
{
    constexpr int NQ = 2 * D * D;
#pragma unroll
    for (int p = 0; p < fold_planes(D); ++p) {
        const double2 a = *reinterpret_cast<const double2*>(fold + (p * n + i) * 4);
        const double2 b = *reinterpret_cast<const double2*>(fold + (p * n + i) * 4 + 2);
        const double v[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * p + c < NQ) f.y[4 * p + c] = v[c];
    }
}

template <int D>
__device__ __forceinline__ void fold_store(const FoldState<D>& f, double* fold, int64_t n, int64_t i)
{
    constexpr int NQ = 2 * D * D;
#pragma unroll
    for (int p = 0; p < fold_planes(D); ++p) {
        double v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (4 * p + c < NQ) ? f.y[4 * p + c] : 0.0;
        *reinterpret_cast<double2*>(fold + (p * n + i) * 4) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(fold + (p * n + i) * 4 + 2) = make_double2(v[2], v[3]);
    }
}

// Cell index of coordinate s = x N: floor clamped to [0, N-1]; positions past
// the edge are extrapolated from the edge cell (RK stages may step outside).
template <typename T>
__device__ __forceinline__ int cell_of(T s, int N, T& frac)
{
    int i;
    if (s >= T(N - 1)) i = N - 1;
    else if (s > T(0)) i = (int)s;
    else i = 0;
    frac = s - T(i);
    return i;
}

// Bi/trilinear interpolation of the node values (u then grad u) at x.
template <typename T, int D>
__device__ __forceinline__ void interp(const T* __restrict__ nodes, int N, T fN, const T* x, T* u, T* G)
{
    constexpr int S4 = node_stride(D) / 4;
    T f[D];
    int ic[D];
#pragma unroll
    for (int a = 0; a < D; ++a) ic[a] = cell_of<T>(x[a] * fN, N, f[a]);
    const int64_t nn = N + 1;
    int64_t base = ic[0];
    if (D == 2) base += nn * ic[1];
    else base += nn * (ic[1] + nn * (int64_t)ic[2]);
    T acc[D + D * D];
#pragma unroll
    for (int q = 0; q < D + D * D; ++q) acc[q] = T(0);
#pragma unroll
    for (int cnr = 0; cnr < (1 << D); ++cnr) {
        T w = T(1);
        int64_t idx = base;
        int64_t mul = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int bit = (cnr >> a) & 1;
            w *= bit ? f[a] : T(1) - f[a];
            idx += bit * mul;
            mul *= nn;
        }
        T v[node_stride(D)];
#pragma unroll
        for (int c = 0; c < S4; ++c) load4<T>(nodes, idx * S4 + c, v + 4 * c);
#pragma unroll
        for (int q = 0; q < D + D * D; ++q) acc[q] = fma(w, v[q], acc[q]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = acc[a];
#pragma unroll
    for (int q = 0; q < D * D; ++q) G[q] = acc[D + q];
}

// Right-hand side of the droplet system given u, G at the stage position.
template <typename T, int D, bool FLA>
__device__ __forceinline__ void rhs(const T* y, const T* u, const T* G, T invSt, T* f)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        f[a] = y[D + a];
        f[D + a] = (u[a] - y[D + a]) * invSt;
    }
    if (FLA) {
        const T* J = y + 2 * D;
        const T* W = y + 2 * D + D * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                T gj = T(0);
#pragma unroll
                for (int j = 0; j < D; ++j) gj = fma(G[i * D + j], J[j * D + k], gj);
                f[2 * D + i * D + k] = W[i * D + k];
                f[2 * D + D * D + i * D + k] = (gj - W[i * D + k]) * invSt;
            }
    }
}

template <typename T, int D, bool FLA, int MODE>
__device__ __forceinline__ int advance_one(const AdvArgs& a, int64_t i, int& fold_steps)
{
    constexpr bool FOLD = MODE == kGuarded;
    constexpr int kind = FLA ? FLA_CLOUD_FLA : FLA_CLOUD_LPT;
    constexpr int NP = state_planes(kind, D);
    constexpr int NY = FLA ? 2 * D + 2 * D * D : 2 * D;
    constexpr int OA = acc_offset(kind, D);
    uint32_t meta = a.meta[i];
    if (meta & FLA_META_DEAD) return 0;
    if (MODE == kScreen && (meta & FLA_META_FOLD)) {   // in the guard: the guarded pass takes it
        a.fold_list[atomicAdd(a.fold_count, 1u)] = (uint32_t)i;
        return 0;
    }
    const fla_batch* B = a.batches + (meta & FLA_META_BATCH_MASK);
    const int ss = __ldg(&B->step_start);
    const int sd = __ldg(&B->step_dead);
    bool active = (meta & FLA_META_ACTIVE) != 0;
    if (!active && (ss < a.step0 || ss >= a.step0 + a.nsteps)) return 0;

    T* state = (T*)a.state;
    const T* nodes = (const T*)a.nodes;
    T sv[NP * 4];
#pragma unroll
    for (int p = 0; p < NP; ++p) load4<T>(state, p * a.n + i, sv + 4 * p);
    T y[NY], acc[1 + D];
#pragma unroll
    for (int q = 0; q < NY; ++q) y[q] = sv[q];
#pragma unroll
    for (int q = 0; q <= D; ++q) acc[q] = a.reset ? T(0) : sv[OA + q];

    const T St0 = T(__ldg(&B->St0));
    const T delta = T(a.delta);
    const T h = T(a.dt);
    const T half = T(0.5) * h;
    const T sixth = h / T(6);
    const T fN = T(a.N);
    T u[D], G[D * D];
    int integrated = 0;
    FoldState<D> fs;
    bool fold = false;
    if (FOLD && (meta & FLA_META_FOLD)) {
        fold = true;
        fold_load<D>(fs, a.fold, a.n, i);
    }

    for (int s = a.step0; s < a.step0 + a.nsteps; ++s) {
        if (!active) {
            if (s != ss) continue;
            // release: v0 = u(x0); J = I, W = dv0/dx0 = grad u(x0) (initial data of Eq. 8)
            interp<T, D>(nodes, a.N, fN, y, u, G);
#pragma unroll
            for (int q = 0; q < D; ++q) y[D + q] = u[q];
            if (FLA) {
#pragma unroll
                for (int q = 0; q < D * D; ++q) {
                    y[2 * D + q] = (q % (D + 1) == 0) ? T(1) : T(0);
                    y[2 * D + D * D + q] = G[q];
                }
            }
#pragma unroll
            for (int q = 0; q <= D; ++q) acc[q] = T(0);
            active = true;
            meta |= FLA_META_ACTIVE;
            if (FOLD) {
                fold = false;
                meta &= ~FLA_META_FOLD;
            }
        }
        if (s >= sd) {   // evaporated (deadline decided on the host in double precision)
            active = false;
            meta = (meta & ~FLA_META_ACTIVE) | FLA_META_DEAD;
            break;
        }
        if (MODE == kScreen && fabsf(det_f32<D>((const float*)y + 2 * D)) < a.tau_fold) {
            // would enter the guard: leave the state as it was and hand the droplet over
            a.fold_list[atomicAdd(a.fold_count, 1u)] = (uint32_t)i;
            return 0;
        }
        ++integrated;
        if (FOLD) {   // enter or leave the fold guard (hysteresis tau .. 4 tau)
            if (!fold) {
                if (fabsf(det_f32<D>((const float*)y + 2 * D)) < a.tau_fold) {
                    fold = true;
                    meta |= FLA_META_FOLD;
#pragma unroll
                    for (int q = 0; q < 2 * D * D; ++q) fs.y[q] = (double)y[2 * D + q];
                }
            } else if (fabs(fold_det<D>(fs)) > 4.0 * (double)a.tau_fold) {
                fold = false;
                meta &= ~FLA_META_FOLD;
            }
            fold_steps += fold ? 1 : 0;
        }
        const T tau = T(s - ss) * h;                       // t - t0
        const T r2a = T(1) + delta * tau;                  // (r/r0)^2, Eq. 4
        const T r2b = T(1) + delta * (tau + half);
        const T r2c = T(1) + delta * (tau + h);
        const T iSa = T(1) / (St0 * r2a), iSb = T(1) / (St0 * r2b), iSc = T(1) / (St0 * r2c);

        T k[NY], ks[NY], ys[NY];
        // stage 1; the window sums use its u and v (left rectangle over substeps)
        interp<T, D>(nodes, a.N, fN, y, u, G);
        {
            const T r = sqrt(r2a);
            const T m = r2a * r;                 // m = r^3
            const T mdot = T(1.5) * delta * r;   // dm/dt with r r' = delta/2
            acc[0] = fma(h, mdot, acc[0]);
#pragma unroll
            for (int q = 0; q < D; ++q)
                acc[1 + q] = fma(h, m * (u[q] - y[D + q]) * iSa + mdot * y[D + q], acc[1 + q]);
        }
        rhs<T, D, FLA>(y, u, G, iSa, k);
        if (FOLD && fold) fold_stage<D>(fs, stage_g<D>((const float*)G), (float)iSa, 0.5 * a.dt, 0);
#pragma unroll
        for (int q = 0; q < NY; ++q) {
            ks[q] = k[q];
            ys[q] = fma(half, k[q], y[q]);
        }
        // stage 2
        interp<T, D>(nodes, a.N, fN, ys, u, G);
        rhs<T, D, FLA>(ys, u, G, iSb, k);
        if (FOLD && fold) fold_stage<D>(fs, stage_g<D>((const float*)G), (float)iSb, 0.5 * a.dt, 1);
#pragma unroll
        for (int q = 0; q < NY; ++q) {
            ks[q] = fma(T(2), k[q], ks[q]);
            ys[q] = fma(half, k[q], y[q]);
        }
        // stage 3
        interp<T, D>(nodes, a.N, fN, ys, u, G);
        rhs<T, D, FLA>(ys, u, G, iSb, k);
        if (FOLD && fold) fold_stage<D>(fs, stage_g<D>((const float*)G), (float)iSb, a.dt, 2);
#pragma unroll
        for (int q = 0; q < NY; ++q) {
            ks[q] = fma(T(2), k[q], ks[q]);
            ys[q] = fma(h, k[q], y[q]);
        }
        // stage 4
        interp<T, D>(nodes, a.N, fN, ys, u, G);
        rhs<T, D, FLA>(ys, u, G, iSc, k);
#pragma unroll
        for (int q = 0; q < NY; ++q) y[q] = fma(sixth, ks[q] + k[q], y[q]);
        if (FOLD && fold) {   // double-precision J, W replace the single-precision update
            fold_stage<D>(fs, stage_g<D>((const float*)G), (float)iSc, a.dt, 3);
#pragma unroll
            for (int q = 0; q < 2 * D * D; ++q) y[2 * D + q] = (T)fs.y[q];
        }
        // outflow: leaving [0,1]^dim ends the trajectory
        bool out = false;
#pragma unroll
        for (int q = 0; q < D; ++q) out |= !(y[q] >= T(0) && y[q] <= T(1));
        if (out) {
            active = false;
            meta = (meta & ~FLA_META_ACTIVE) | FLA_META_DEAD;
            break;
        }
    }
#pragma unroll
    for (int q = 0; q < NY; ++q) sv[q] = y[q];
#pragma unroll
    for (int q = 0; q <= D; ++q) sv[OA + q] = acc[q];
#pragma unroll
    for (int p = 0; p < NP; ++p) store4<T>(state, p * a.n + i, sv + 4 * p);
    if (FOLD && fold) fold_store<D>(fs, a.fold, a.n, i);
    a.meta[i] = meta;
    return integrated;
}

template <typename T, int D, bool FLA, int MODE>
__global__ void __launch_bounds__(128) k_advance(AdvArgs a)
{
    pdl_entry();
    constexpr bool FOLD = MODE == kGuarded;
    int nf = 0, n = 0;
    if (MODE != kGuarded) {
        const int64_t i = droplet_of(a.order, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, a.n);
        n = i < a.n ? advance_one<T, D, FLA, MODE>(a, i, nf) : 0;
    } else {   // the listed droplets, grid-stride
        const unsigned cnt = *a.fold_count;
        for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x)
            n += advance_one<T, D, FLA, MODE>(a, a.fold_list[k], nf);
    }
    // integrated droplet steps (and those in the fold guard): one atomic per block
    __shared__ int s_sum[2][4];
    const int w = __reduce_add_sync(0xffffffffu, n);
    const int wf = FOLD ? __reduce_add_sync(0xffffffffu, nf) : 0;
    if ((threadIdx.x & 31) == 0) {
        s_sum[0][threadIdx.x >> 5] = w;
        s_sum[1][threadIdx.x >> 5] = wf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t = (long long)s_sum[0][0] + s_sum[0][1] + s_sum[0][2] + s_sum[0][3];
        if (t) atomicAdd(&a.status->droplet_steps, (unsigned long long)t);
        if (FOLD) {
            const long long tf = (long long)s_sum[1][0] + s_sum[1][1] + s_sum[1][2] + s_sum[1][3];
            if (tf) atomicAdd(&a.status->fold_steps, (unsigned long long)tf);
        }
    }
}

// ---------------------------------------------------------------- compensated (FLA_F32X2)

struct AdvX2Args {
    float* state;          // hi planes, then lo planes
    uint32_t* meta;
    const fla_batch* batches;
    const float* nodes;    // a node array, then b node array (k_carrier_split_x2)
    int64_t n, n_nodes;
    int N;
    int step0, nsteps;
    df dt, half, sixth, delta;
    int reset;
    DevStatus* status;
    const uint32_t* order; // as AdvArgs::order
};

// Bi/trilinear interpolation of the double-float node values at the
// double-float position x.  The cell index is floor(x N) clamped to
// [0, N - 1] and the fraction x N - i is exact in double-float; the corner
// weights w are double-float products of the fractions.  Each node value is
// stored as a + b, a on its component's grid Q (at most 12 significant bits,
// |a| <= 2^11 Q) and b the rest (|b| <= Q/2).  With w = w1 + w2, w1 on the
// grid 2^-10 (|w1| < 8 2^10 units while the fractions lie in (-1/2, 3/2)):
//   sum w v = sum w1 a  (exact: products below 2^22 units of 2^-10 Q, sums
//                        below 2^24 units)
//           + sum (w2 a + w b)   (terms of size 2^-11 of the component's
//                                 scale, plain single precision)
// so the result carries about 2^-30 of the component's largest magnitude, at
// three single-precision operations per corner and value.
template <int D>
__device__ __forceinline__ void interp_x2(const AdvX2Args& a, const df* x, df* u, df* G)
{
    constexpr int S = node_stride(D);
    constexpr int NV = D + D * D;
    df f[D];
    int64_t base = 0, mul = 1;
    const int64_t nn = a.N + 1;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const df s = x[q] * (float)a.N;
        int i = df_floor(s);
        i = i < 0 ? 0 : (i > a.N - 1 ? a.N - 1 : i);
        f[q] = two_sum(__fsub_rn(s.hi, (float)i), s.lo);   // s.hi - i is exact
        base += (int64_t)i * mul;
        mul *= nn;
    }
    df g[D];   // 1 - f
#pragma unroll
    for (int q = 0; q < D; ++q) g[q] = df_of(1.0f) - f[q];
    float sa[NV], sb[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sa[q] = sb[q] = 0.0f;
    // Corner weights w = prod_q (f_q or g_q), corners in the order of their
    // bits (x, then y, then z): the factors of the lower axes once per stage,
    // then one product with the last axis's factor per corner.  The products
    // are left unrenormalised (hi + lo, |lo| a few ulp(hi) at most): they only
    // feed the split w = w1 + w2, which needs w to about 2^-36.
    constexpr int NC = 1 << (D - 1);
    df wl[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        wl[c] = (c & 1) ? f[0] : g[0];
        if (D == 3) wl[c] = mul_unnorm(wl[c], ((c >> 1) & 1) ? f[1] : g[1]);
    }
    // four corners per iteration (3D cone, advance ms per run: 236.5 four at a
    // time, 250.1 two at a time, 251.8 fully unrolled, where the node loads of
    // all corners compete for the registers)
#pragma unroll 4
    for (int cnr = 0; cnr < (1 << D); ++cnr) {
        const int c = cnr & (NC - 1);
        df wlo;   // selected, not indexed: an indexed wl would live in local memory
        if (D == 3) {
            const bool hy = (c >> 1) & 1;
            wlo = (c & 1) ? (hy ? wl[NC - 1] : wl[1]) : (hy ? wl[NC - 2] : wl[0]);
        } else {
            wlo = (c & 1) ? wl[NC - 1] : wl[0];
        }
        const df w = mul_unnorm(wlo, (cnr >> (D - 1)) ? f[D - 1] : g[D - 1]);
        int64_t idx = base + (cnr & 1), m2 = nn;
#pragma unroll
        for (int q = 1; q < D; ++q) {
            idx += ((cnr >> q) & 1) * m2;
            m2 *= nn;
        }
        const float w1 = __fmul_rn(rintf(__fmul_rn(w.hi, 1024.0f)), 1.0f / 1024.0f);
        const float w2 = __fadd_rn(__fsub_rn(w.hi, w1), w.lo);   // w.hi - w1 is exact
        float va[S], vb[S];
#pragma unroll
        for (int k = 0; k < S / 4; ++k) {
            load4<float>(a.nodes, idx * (S / 4) + k, va + 4 * k);
            load4<float>(a.nodes + a.n_nodes * S, idx * (S / 4) + k, vb + 4 * k);
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            sa[q] = __fmaf_rn(w1, va[q], sa[q]);
            sb[q] = __fmaf_rn(w.hi, vb[q], __fmaf_rn(w2, va[q], sb[q]));
        }
    }
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = two_sum(sa[q], sb[q]);
#pragma unroll
    for (int q = 0; q < D * D; ++q) G[q] = two_sum(sa[D + q], sb[D + q]);
}

// Right-hand side of Eqs. 3 and 8 in double-float.  The slopes are left
// unrenormalised (hi + lo with |lo| a few ulp(hi)): they only enter the
// stage states and the slope sum, whose operations take any such pair.
template <int D, bool FLA>
__device__ __forceinline__ void rhs_x2(const df* y, const df* u, const df* G, df invSt, df* f)
{
#pragma unroll
    for (int q = 0; q < D; ++q) {
        f[q] = y[D + q];
        f[D + q] = mul_unnorm(add_unnorm(u[q], -y[D + q]), invSt);
    }
    if (FLA) {
        const df* J = y + 2 * D;
        const df* W = y + 2 * D + D * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                // grad u . J - W as one compensated sum
                DotAcc gj = dot_first(G[i * D], J[k]);
#pragma unroll
                for (int j = 1; j < D; ++j) gj = dot_add(gj, G[i * D + j], J[j * D + k]);
                gj = dot_add(gj, -W[i * D + k]);
                f[2 * D + i * D + k] = W[i * D + k];
                f[2 * D + D * D + i * D + k] = mul_unnorm(dot_unnorm(gj), invSt);
            }
    }
}

// The step-start state and the slope sum of one droplet (registers).  Keeping
// them in shared memory instead, to fit more warps per SM, was slower on the 3D
// cone (512 ms per run with 3 blocks per SM, 605 ms with 4 and spills, against
// 448 ms in registers at 8 warps per SM).
template <int NY>
struct RegVec {
    df v[NY];
    __device__ __forceinline__ df get(int q) const { return v[q]; }
    __device__ __forceinline__ void set(int q, df x) { v[q] = x; }
};

template <int D, bool FLA, class VecY, class VecK>
__device__ __forceinline__ int advance_x2_one(const AdvX2Args& a, int64_t i, VecY& y, VecK& ks)
{
    constexpr int kind = FLA ? FLA_CLOUD_FLA : FLA_CLOUD_LPT;
    constexpr int NP = state_planes(kind, D);
    constexpr int NY = FLA ? 2 * D + 2 * D * D : 2 * D;
    constexpr int OA = acc_offset(kind, D);
    uint32_t meta = a.meta[i];
    if (meta & FLA_META_DEAD) return 0;
    const fla_batch* B = a.batches + (meta & FLA_META_BATCH_MASK);
    const int ss = __ldg(&B->step_start);
    const int sd = __ldg(&B->step_dead);
    bool active = (meta & FLA_META_ACTIVE) != 0;
    if (!active && (ss < a.step0 || ss >= a.step0 + a.nsteps)) return 0;

    float acc[1 + D];
    {
        float sh[NP * 4], sl[NP * 4];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            load4<float>(a.state, p * a.n + i, sh + 4 * p);
            load4<float>(a.state, (NP + p) * a.n + i, sl + 4 * p);
        }
#pragma unroll
        for (int q = 0; q < NY; ++q) y.set(q, df{sh[q], sl[q]});
#pragma unroll
        for (int q = 0; q <= D; ++q) acc[q] = a.reset ? 0.0f : sh[OA + q];
    }

    const df St0 = df_of(__ldg(&B->St0));
    const float h32 = a.dt.hi, delta32 = a.delta.hi;
    df u[D], G[D * D];
    int integrated = 0;
    for (int s = a.step0; s < a.step0 + a.nsteps; ++s) {
        if (!active) {
            if (s != ss) continue;
            // release: v0 = u(x0); J = I, W = dv0/dx0 = grad u(x0) (initial data of Eq. 8)
            df x0[D];
#pragma unroll
            for (int q = 0; q < D; ++q) x0[q] = y.get(q);
            interp_x2<D>(a, x0, u, G);
#pragma unroll
            for (int q = 0; q < D; ++q) y.set(D + q, u[q]);
            if (FLA) {
#pragma unroll
                for (int q = 0; q < D * D; ++q) {
                    y.set(2 * D + q, df_of((q % (D + 1) == 0) ? 1.0f : 0.0f));
                    y.set(2 * D + D * D + q, G[q]);
                }
            }
#pragma unroll
            for (int q = 0; q <= D; ++q) acc[q] = 0.0f;
            active = true;
            meta |= FLA_META_ACTIVE;
        }
        if (s >= sd) {   // evaporated (deadline decided on the host in double precision)
            active = false;
            meta = (meta & ~FLA_META_ACTIVE) | FLA_META_DEAD;
            break;
        }
        ++integrated;
        // St(t) = St0 (1 + delta (t - t0)) at the stage times t, t + dt/2, t + dt (Eqs. 4-5)
        const df tau = a.dt * (float)(s - ss);
        const df r2a = a.delta * tau + 1.0f;
        const df r2b = a.delta * (tau + a.half) + 1.0f;
        const df r2c = a.delta * (tau + a.dt) + 1.0f;
        const df iSa = df_rcp(St0 * r2a), iSb = df_rcp(St0 * r2b), iSc = df_rcp(St0 * r2c);

        // The four RK4 stages run as a loop (not unrolled): the double-float
        // interpolation and right-hand side are long, and four inlined copies
        // overflow the instruction cache.
        df k[NY], ys[NY];
#pragma unroll
        for (int q = 0; q < NY; ++q) ys[q] = y.get(q);
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
            interp_x2<D>(a, ys, u, G);
            if (stage == 0) {   // window sums at the first stage (left rectangle over substeps)
                const float r2 = r2a.hi;
                const float r = sqrtf(r2);
                const float m = r2 * r;                   // m = r^3
                const float mdot = 1.5f * delta32 * r;    // dm/dt with r r' = delta/2
                const float iS = iSa.hi;
                acc[0] = fmaf(h32, mdot, acc[0]);
#pragma unroll
                for (int q = 0; q < D; ++q)
                    acc[1 + q] = fmaf(h32, m * (u[q] - ys[D + q]).hi * iS + mdot * ys[D + q].hi, acc[1 + q]);
            }
            rhs_x2<D, FLA>(ys, u, G, stage == 0 ? iSa : (stage == 3 ? iSc : iSb), k);
            // k1 + 2 k2 + 2 k3 + k4 (the factor 2 is exact), and the next stage's
            // state y + c k (c = dt/2, dt/2, dt)
            const float wk = (stage == 1 || stage == 2) ? 2.0f : 1.0f;
            const df c = stage == 2 ? a.dt : a.half;
            // the running slope sum and the stage states stay unrenormalised; the
            // step's final axpy renormalises the new state
#pragma unroll
            for (int q = 0; q < NY; ++q)
                ks.set(q, stage == 0 ? k[q] : add_unnorm(ks.get(q), df{k[q].hi * wk, k[q].lo * wk}));
            if (stage < 3) {
#pragma unroll
                for (int q = 0; q < NY; ++q) ys[q] = axpy_unnorm(c, k[q], y.get(q));
            }
        }
#pragma unroll
        for (int q = 0; q < NY; ++q) y.set(q, df_axpy(a.sixth, ks.get(q), y.get(q)));
        // outflow: leaving [0,1]^dim ends the trajectory
        bool out = false;
#pragma unroll
        for (int q = 0; q < D; ++q) out |= df_lt(y.get(q), 0.0f) || df_gt(y.get(q), 1.0f);
        if (out) {
            active = false;
            meta = (meta & ~FLA_META_ACTIVE) | FLA_META_DEAD;
            break;
        }
    }
    {
        float sh[NP * 4], sl[NP * 4];
#pragma unroll
        for (int q = 0; q < NP * 4; ++q) sh[q] = sl[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < NY; ++q) {
            const df v = y.get(q);
            sh[q] = v.hi;
            sl[q] = v.lo;
        }
#pragma unroll
        for (int q = 0; q <= D; ++q) sh[OA + q] = acc[q];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            store4<float>(a.state, p * a.n + i, sh + 4 * p);
            store4<float>(a.state, (NP + p) * a.n + i, sl + 4 * p);
        }
    }
    a.meta[i] = meta;
    return integrated;
}

constexpr int kAdvX2Threads = 128;

// The 2D step runs 3 blocks per SM in 168 registers (13.8 ms per jet run,
// against 14.5 ms at 4 blocks in 128 registers with spills; uncapped it takes
// 187); the 3D step keeps its 255.
template <int D, bool FLA>
constexpr int x2_min_blocks() { return D == 2 && FLA ? 3 : 1; }

template <int D, bool FLA>
__global__ void __launch_bounds__(kAdvX2Threads, x2_min_blocks<D, FLA>()) k_advance_x2(AdvX2Args a)
{
    pdl_entry();
    constexpr int NY = FLA ? 2 * D + 2 * D * D : 2 * D;
    const int64_t i = droplet_of(a.order, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, a.n);
    int n = 0;
    if (i < a.n) {
        RegVec<NY> y, ks;
        n = advance_x2_one<D, FLA>(a, i, y, ks);
    }
    __shared__ int s_sum[kAdvX2Threads / 32];
    const int w = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
#pragma unroll
        for (int q = 0; q < kAdvX2Threads / 32; ++q) t += s_sum[q];
        if (t) atomicAdd(&a.status->droplet_steps, (unsigned long long)t);
    }
}

template <int D, bool FLA>
cudaError_t launch_x2(const AdvX2Args& b, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((b.n + kAdvX2Threads - 1) / kAdvX2Threads);
    launch_pdl(k_advance_x2<D, FLA>, dim3(blocks), dim3(kAdvX2Threads), 0, s, b);
    return cudaGetLastError();
}

// Batched clouds of one dimension (single precision, FLA): droplet g of the
// group belongs to cloud k with pre[k] <= g < pre[k + 1] of the group's
// prefix; the per-droplet work is that of k_advance.
// skip_active: leave droplets that are active now to the cell-sorted part of
// an ordered launch (below).
template <int D>
__device__ __forceinline__ int batch_advance_droplet(const BatchDev& b, int first, int count, int64_t g, int nsteps,
                                                     double dt, int reset, DevStatus* st, bool skip_active = false)
{
    // droplets of the group's clouds are contiguous in the global droplet order
    const int64_t base = b.drop_pre[first];
    const int k = first + batch_find(b.drop_pre + first, count, base + g);
    const BatchCloud& c = b.clouds[k];
    if (skip_active && (c.meta[base + g - b.drop_pre[k]] & FLA_META_ACTIVE)) return 0;
    AdvArgs a{};
    a.state = c.state;
    a.meta = c.meta;
    a.batches = c.batches;
    a.nodes = c.nodes;
    a.n = c.n;
    a.N = c.N;
    a.step0 = *b.step;
    a.nsteps = nsteps;
    a.dt = dt;
    a.delta = c.delta;
    a.reset = reset;
    a.status = st;
    int nf = 0;
    return advance_one<float, D, true, kPlain>(a, base + g - b.drop_pre[k], nf);
}

// The launch covers 2 n_dim threads.  Once a window of this run has binned
// the clouds (step[1] set), the droplets that were active then -- the sorted
// positions [s0, s1) of this dimension's cells, s1 - s0 = A of them -- are
// taken in that cell-sorted order by threads [0, A), so that the droplets of a
// warp read the same carrier nodes; threads [A, A + n_dim) then run through
// the dimension's droplets in seed order and take those that are not active
// (pending releases; dead ones return at once).  The two sets are disjoint:
// between the binning and this launch no kernel changes a meta word, and a
// droplet that the sorted part ends stays out of the second set.  Each
// droplet's arithmetic is the same whichever thread runs it.
template <int D>
__global__ void __launch_bounds__(256) k_batch_advance(BatchDev b, int first, int count, int64_t n_dim,
                                                       int nsteps, double dt, int reset, DevStatus* st)
{
    pdl_entry();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int n = 0;
    if (b.step[1] == 0) {
        if (t < n_dim) n = batch_advance_droplet<D>(b, first, count, t, nsteps, dt, reset, st);
    } else {
        const int g0 = batch_group(D, 0);
        const uint32_t s0 = __ldg(b.bin_start + b.group_cells[g0]);
        const uint32_t s1 = __ldg(b.bin_start + b.group_cells[g0 + 2]);
        const int64_t A = s1 > s0 ? (int64_t)(s1 - s0) : 0;
        if (t < A) {
            const int64_t g = (int64_t)__ldg(b.perm + s0 + t) - b.drop_pre[first];
            if (g >= 0 && g < n_dim) n = batch_advance_droplet<D>(b, first, count, g, nsteps, dt, reset, st);
        } else if (t - A < n_dim) {
            n = batch_advance_droplet<D>(b, first, count, t - A, nsteps, dt, reset, st, true);
        }
    }
    __shared__ int s_sum[8];
    const int w = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_sum[q];
        if (t) atomicAdd(&st->droplet_steps, (unsigned long long)t);
    }
}

template <typename T, int D, bool FLA, int MODE = kPlain>
cudaError_t launch_t(const AdvArgs& a, cudaStream_t s, int guarded_blocks = 0)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
    launch_pdl(k_advance<T, D, FLA, MODE>, dim3(blocks), dim3(threads), 0, s, a);
    if constexpr (MODE == kScreen) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const unsigned gb = (unsigned)(guarded_blocks < (int)blocks ? guarded_blocks : (int)blocks);
        launch_pdl(k_advance<T, D, FLA, kGuarded>, dim3(gb), dim3(threads), 0, s, a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_advance(const fla_cloud& cl, const fla_mesh& m, const void* nodes, int step0, int nsteps,
                           double dt, bool reset, DevStatus* st, int num_sms, cudaStream_t s, const uint32_t* order)
{
    AdvArgs a{};
    a.order = order;
    a.status = st;
    a.state = cl.state_dev;
    a.meta = cl.meta_dev;
    a.batches = cl.batches_dev;
    a.nodes = nodes;
    a.n = cl.n;
    a.N = m.n;
    a.step0 = step0;
    a.nsteps = nsteps;
    a.dt = dt;
    a.delta = cl.delta;
    a.reset = reset ? 1 : 0;
    a.fold = (double*)cl.fold_dev;
    a.tau_fold = (float)cl.tau_fold;
    if (a.n == 0) return cudaSuccess;
    const bool fla = cl.kind == FLA_CLOUD_FLA;
    if (cl.dtype == FLA_F32X2) {
        AdvX2Args b{};
        b.state = (float*)cl.state_dev;
        b.meta = cl.meta_dev;
        b.batches = cl.batches_dev;
        b.nodes = (const float*)nodes;
        b.n = cl.n;
        const int64_t nn = m.n + 1;
        b.n_nodes = m.dim == 2 ? nn * nn : nn * nn * nn;
        b.N = m.n;
        b.step0 = step0;
        b.nsteps = nsteps;
        b.dt = df_host(dt);
        b.half = df_host(0.5 * dt);
        b.sixth = df_host(dt / 6.0);
        b.delta = df_host(cl.delta);
        b.reset = reset ? 1 : 0;
        b.status = st;
        b.order = order;
        if (cl.dim == 2) return fla ? launch_x2<2, true>(b, s) : launch_x2<2, false>(b, s);
        return fla ? launch_x2<3, true>(b, s) : launch_x2<3, false>(b, s);
    }
    if (cl.dtype == FLA_F32 && fla && a.fold) {
        FoldLayout L = fold_layout(cl.dim, cl.n);
        a.fold_list = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(cl.fold_dev) + L.list);
        a.fold_count = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(cl.fold_dev) + L.count);
        const cudaError_t e = cudaMemsetAsync(a.fold_count, 0, 4, s);
        if (e != cudaSuccess) return e;
        const int gb = 4 * (num_sms > 0 ? num_sms : 1);
        if (cl.dim == 2) return launch_t<float, 2, true, kScreen>(a, s, gb);
        return launch_t<float, 3, true, kScreen>(a, s, gb);
    }
    if (cl.dtype == FLA_F32) {
        if (cl.dim == 2) return fla ? launch_t<float, 2, true>(a, s) : launch_t<float, 2, false>(a, s);
        return fla ? launch_t<float, 3, true>(a, s) : launch_t<float, 3, false>(a, s);
    }
    if (cl.dim == 2) return fla ? launch_t<double, 2, true>(a, s) : launch_t<double, 2, false>(a, s);
    return fla ? launch_t<double, 3, true>(a, s) : launch_t<double, 3, false>(a, s);
}

// Loads the batched advance kernels' module before the autotuner times them.
cudaError_t batch_prepare_advance()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_batch_advance<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_batch_advance<3>);
    return e;
}

cudaError_t launch_batch_advance(const BatchDev& b, int dim, int64_t n_dim, int nsteps, double dt, bool reset,
                                 int threads, DevStatus* st, cudaStream_t s)
{
    if (n_dim == 0 || nsteps == 0) return cudaSuccess;
    const int g0 = batch_group(dim, 0);
    const int first = b.group_first[g0], count = b.group_first[g0 + 2] - first;
    const unsigned blocks = (unsigned)((2 * n_dim + threads - 1) / threads);   // see k_batch_advance
    if (dim == 2) launch_pdl(k_batch_advance<2>, dim3(blocks), dim3(threads), 0, s, b, first, count, n_dim, nsteps, dt, reset ? 1 : 0, st);
    else launch_pdl(k_batch_advance<3>, dim3(blocks), dim3(threads), 0, s, b, first, count, n_dim, nsteps, dt, reset ? 1 : 0, st);
    return cudaGetLastError();
}

}  // namespace fla

#ifdef FLA_WINDOW_PHASES
// Phase of the persistent window kernel (window.cuh): the droplets of one
// dimension's clouds, window sums reset.
#include "window.cuh"
namespace fla {

__device__ int window_advance(const BatchDev& b, int dim, int64_t n_dim, int nsteps, double dt, DevStatus* st)
{
    if (n_dim == 0 || nsteps == 0) return 0;
    const int g0 = batch_group(dim, 0);
    const int first = b.group_first[g0], count = b.group_first[g0 + 2] - first;
    int n = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_dim; g += (int64_t)gridDim.x * blockDim.x)
        n += dim == 2 ? batch_advance_droplet<2>(b, first, count, g, nsteps, dt, 1, st)
                      : batch_advance_droplet<3>(b, first, count, g, nsteps, dt, 1, st);
    return n;
}

}  // namespace fla
#endif
