// Droplet records for the kernel-regression gather, written in sorted order.
//
// Per binned droplet (Eq. 6, Eq. 15, Eq. 14 and App. B parcel level c):
//   n = n0 / max(|det J|, 1e-12),  a = n * acc / T_window,
//   ISO:   h = clamp(h0 |det J|^p, h_min, h_max), weight (1/h) exp(-r^2/(2 h^2)),
//   ANISO: Sigma = f h0^2 J J^T + h_min^2 I, f = min(1, (h_max^2 - d h_min^2)/tr(h0^2 J J^T)),
//          weight det(Sigma)^-1/2 exp(-d^T Sigma^-1 d / 2).
//
// Precision (single-precision path, mixed mode): det J is formed in double
// where it can cancel -- always in 2D (the products of single-precision
// entries are exact in double), and in 3D when the single-precision cofactor
// expansion is below 1e-2 of the product of the rows' L1 norms (near a fold
// caustic, where det J nearly vanishes).  A droplet held in the advance's fold
// guard takes det J from its double-precision J and n = n0/|det J| in double.
// Everything else is single precision; double-precision division and square
// root, which are slow on this GPU, are used for those droplets only.  Plain
// mode forms det J and n in single precision for every droplet.
// The values that decide the truncation test (h and 9 h^2; Sigma^-1) are
// formed one rounding per operation in a fixed order: this file is compiled
// without FMA contraction so that the decision is reproducible.
#include "mlp_tc.cuh"
#include "batch.cuh"

namespace fla {
namespace {

struct RecArgs {
    const void* state;
    const uint32_t* meta;
    const fla_batch* batches;
    const uint32_t* perm;
    const uint32_t* bin_start;
    int64_t n;
    int64_t n_cells;
    double h_min, h_max, p, window_dt;
    float inv_window;           // 1 / window_dt
    float room;                 // (float)(h_max^2 - d h_min^2)
    float hmin2;                // (float)(h_min^2)
    void* rec;
    unsigned int* ext_max;      // max over droplets of the squared support radius (float bits)
    DevStatus* status;
    const double* fold;         // fold-guard planes (double J first), or null
    int plain;                  // 1: det J and n in single precision
    const unsigned char* mlp;   // packed learned correction, or null
    float* mlp_out;             // g(f) per droplet index, or null
    double dx;                  // cell size (network feature f4)
    float* aux;                 // per sorted record: g(f) and 1 if h moves with it, or null
    int x2;                     // 1: compensated cloud (FLA_F32X2), lo planes after the hi planes
};

template <typename T, int D>
__device__ __forceinline__ double det_double(const T* J)
{
    if (D == 2) return (double)J[0] * (double)J[3] - (double)J[1] * (double)J[2];
    const double j0 = J[0], j1 = J[1], j2 = J[2], j3 = J[3], j4 = J[4], j5 = J[5], j6 = J[6], j7 = J[7], j8 = J[8];
    return j0 * (j4 * j8 - j5 * j7) - j1 * (j3 * j8 - j5 * j6) + j2 * (j3 * j7 - j4 * j6);
}

// det J for the single-precision path: double where it can cancel.
template <int D>
__device__ __forceinline__ double det_mixed(const float* j)
{
    if (D == 2) return det_double<float, 2>(j);
    const float detf = j[0] * (j[4] * j[8] - j[5] * j[7]) - j[1] * (j[3] * j[8] - j[5] * j[6]) +
                       j[2] * (j[3] * j[7] - j[4] * j[6]);
    const float H = (fabsf(j[0]) + fabsf(j[1]) + fabsf(j[2])) * (fabsf(j[3]) + fabsf(j[4]) + fabsf(j[5])) *
                    (fabsf(j[6]) + fabsf(j[7]) + fabsf(j[8]));
    if (fabsf(detf) < 0.01f * H) return det_double<float, 3>(j);   // near a fold: FP64
    return (double)detf;
}

template <int D>
__device__ __forceinline__ float det_f32(const float* j)
{
    if (D == 2) return j[0] * j[3] - j[1] * j[2];
    return j[0] * (j[4] * j[8] - j[5] * j[7]) - j[1] * (j[3] * j[8] - j[5] * j[6]) +
           j[2] * (j[3] * j[7] - j[4] * j[6]);
}

// |det J| and n = n0/max(|det J|, 1e-12) of a single-precision droplet in the
// selected precision (see file header).
template <int D>
__device__ __forceinline__ void det_and_n(const RecArgs& a, const float* J, uint32_t meta, int64_t i, double n0,
                                          double& adet, float& n)
{
    if (a.x2) {   // compensated cloud: J = hi + lo, det J and n in double precision
        constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
        constexpr int P0 = (2 * D) / 4, P1 = (2 * D + D * D - 1) / 4;
        float lo[(P1 - P0 + 1) * 4];
#pragma unroll
        for (int p = P0; p <= P1; ++p) load4<float>((const float*)a.state, (NP + p) * a.n + i, lo + 4 * (p - P0));
        double jd[D * D];
#pragma unroll
        for (int q = 0; q < D * D; ++q) jd[q] = (double)J[q] + (double)lo[2 * D + q - 4 * P0];
        adet = fabs(det_double<double, D>(jd));
        n = (float)(n0 / (adet > 1e-12 ? adet : 1e-12));
        return;
    }
    if (a.plain) {
        const float d = fabsf(det_f32<D>(J));
        adet = (double)d;
        n = (float)n0 / fmaxf(d, 1e-12f);
        return;
    }
    if (a.fold && (meta & FLA_META_FOLD)) {
        double jd[D * D];
#pragma unroll
        for (int q = 0; q < D * D; ++q) jd[q] = a.fold[((int64_t)(q >> 2) * a.n + i) * 4 + (q & 3)];
        adet = fabs(det_double<double, D>(jd));
        n = (float)(n0 / (adet > 1e-12 ? adet : 1e-12));
        return;
    }
    adet = fabs(det_mixed<D>(J));
    n = (float)n0 / fmaxf((float)adet, 1e-12f);
}

// Sigma and its inverse in single precision, in a fixed order (see file header).
template <int D>
__device__ __forceinline__ void sigma_inverse_f32(const float* j, float h0f, float room, float hmin2, float* P,
                                                  float& dS, float& tr, bool* capped = nullptr)
{
    float S[D * D];
    const float h02 = h0f * h0f;
    float tr0 = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float sum = 0.0f;
#pragma unroll
            for (int q = 0; q < D; ++q) sum = sum + j[i * D + q] * j[k * D + q];
            S[i * D + k] = h02 * sum;
            if (i == k) tr0 = tr0 + S[i * D + k];
        }
    if (tr0 > room) {
        const float f = room / tr0;
#pragma unroll
        for (int q = 0; q < D * D; ++q) S[q] = S[q] * f;
    }
    if (capped) *capped = tr0 > room;
#pragma unroll
    for (int i = 0; i < D; ++i) S[i * D + i] = S[i * D + i] + hmin2;
    tr = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) tr = tr + S[i * D + i];
    if (D == 2) {
        dS = S[0] * S[3] - S[1] * S[2];
        const float inv = 1.0f / dS;
        P[0] = S[3] * inv; P[3] = S[0] * inv; P[1] = -S[1] * inv; P[2] = P[1];
    } else {
        const float c00 = S[4] * S[8] - S[5] * S[7];
        const float c01 = S[5] * S[6] - S[3] * S[8];
        const float c02 = S[3] * S[7] - S[4] * S[6];
        const float c11 = S[0] * S[8] - S[2] * S[6];
        const float c12 = S[2] * S[3] - S[0] * S[5];
        const float c22 = S[0] * S[4] - S[1] * S[3];
        dS = S[0] * c00 + S[1] * c01 + S[2] * c02;
        const float inv = 1.0f / dS;
        P[0] = c00 * inv; P[1] = c01 * inv; P[2] = c02 * inv;
        P[3] = P[1];      P[4] = c11 * inv; P[5] = c12 * inv;
        P[6] = P[2];      P[7] = P[5];      P[8] = c22 * inv;
    }
}

// Single-precision record.  Layouts: see fla_internal.cuh (c = -log2(e)/(2 h^2),
// lih = log2(1/h), lpref = log2(det(Sigma)^-1/2): the weight is 2^(c r^2 + lih)).
template <int D, int KER>
__device__ __forceinline__ void record_f32(const RecArgs& a, const float* sv, double adet, float n, double h0,
                                           double corr, float* r, float& ext2, bool& bad, bool* h_free = nullptr)
{
    constexpr int OA = acc_offset(FLA_CLOUD_FLA, D);
    const float* J = sv + 2 * D;
    float am[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q <= D; ++q) am[q] = n * sv[OA + q] * a.inv_window;
    if (KER == FLA_KERNEL_ISO) {
        double h = (a.p == 1.0) ? h0 * adet : h0 * pow(adet, a.p);
        h *= corr;   // learned correction (1 without the network)
        if (h_free) *h_free = h > a.h_min && h < a.h_max;
        h = h < a.h_min ? a.h_min : h;
        h = h > a.h_max ? a.h_max : h;
        const float hf = (float)h;
        const float r2max = (float)(9.0 * (double)hf * (double)hf);
        const float c = -0.72134752044448170368f / (hf * hf);
        const float lih = -log2f(hf);
        if (D == 2) {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = c; r[3] = lih;
            r[4] = am[0]; r[5] = am[1]; r[6] = am[2]; r[7] = r2max;
        } else {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = r2max;
            r[4] = c; r[5] = lih;
            r[8] = am[0]; r[9] = am[1]; r[10] = am[2]; r[11] = am[3];
        }
        ext2 = r2max;
        bad = !isfinite(n) || !isfinite(hf);
    } else {
        // learned correction: the Lagrangian bandwidth h0 scaled (corr = 1 without the network)
        float P[9], dS, tr;
        bool capped = false;
        sigma_inverse_f32<D>(J, (float)(h0 * corr), a.room, a.hmin2, P, dS, tr, &capped);
        if (h_free) *h_free = !capped;   // Sigma moves with c only below the trace cap
        const float lpref = -0.5f * log2f(dS);
        const float e2 = 9.0f * tr;
        if (D == 2) {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = lpref; r[3] = e2;
            r[4] = P[0]; r[5] = P[1]; r[6] = P[3];
            r[8] = am[0]; r[9] = am[1]; r[10] = am[2];
        } else {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = lpref;
            r[4] = P[0]; r[5] = P[1]; r[6] = P[2]; r[7] = P[4];
            r[8] = P[5]; r[9] = P[8]; r[10] = e2;
            r[12] = am[0]; r[13] = am[1]; r[14] = am[2]; r[15] = am[3];
        }
        ext2 = e2;
        bad = !isfinite(n) || !(dS > 0.0f) || !isfinite(dS);
    }
#pragma unroll
    for (int q = 0; q <= D; ++q) bad |= !isfinite(am[q]);
}

// Double-precision record (the FP64 path): c = -1/(2 h^2), ih = 1/h, pref = det(Sigma)^-1/2.
template <int D, int KER>
__device__ __forceinline__ void record_f64(const RecArgs& a, const double* sv, double n0, double h0, double* r,
                                           float& ext2, bool& bad)
{
    constexpr int OA = acc_offset(FLA_CLOUD_FLA, D);
    const double* J = sv + 2 * D;
    const double adet = fabs(det_double<double, D>(J));
    const double nd = n0 / (adet > 1e-12 ? adet : 1e-12);
    double am[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q <= D; ++q) am[q] = nd * sv[OA + q] / a.window_dt;
    if (KER == FLA_KERNEL_ISO) {
        double h = (a.p == 1.0) ? h0 * adet : h0 * pow(adet, a.p);
        h = h < a.h_min ? a.h_min : h;
        h = h > a.h_max ? a.h_max : h;
        const double r2max = 9.0 * h * h;
        const double c = -0.5 / (h * h);
        const double ih = 1.0 / h;
        if (D == 2) {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = c; r[3] = ih;
            r[4] = am[0]; r[5] = am[1]; r[6] = am[2]; r[7] = r2max;
        } else {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = r2max;
            r[4] = c; r[5] = ih;
            r[8] = am[0]; r[9] = am[1]; r[10] = am[2]; r[11] = am[3];
        }
        ext2 = (float)r2max;
        bad = !isfinite(nd) || !isfinite(h);
    } else {
        double Sg[9];
        double tr0 = 0.0;
#pragma unroll
        for (int ii = 0; ii < D; ++ii)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double s = 0.0;
#pragma unroll
                for (int jj = 0; jj < D; ++jj) s += J[ii * D + jj] * J[k * D + jj];
                Sg[ii * D + k] = h0 * h0 * s;
                if (ii == k) tr0 += Sg[ii * D + k];
            }
        const double room = a.h_max * a.h_max - (double)D * a.h_min * a.h_min;
        if (tr0 > room) {
            const double f = room / tr0;
#pragma unroll
            for (int q = 0; q < D * D; ++q) Sg[q] *= f;
        }
#pragma unroll
        for (int ii = 0; ii < D; ++ii) Sg[ii * D + ii] += a.h_min * a.h_min;
        double tr = 0.0;
#pragma unroll
        for (int ii = 0; ii < D; ++ii) tr += Sg[ii * D + ii];
        double P[9], dS;
        if (D == 2) {
            dS = Sg[0] * Sg[3] - Sg[1] * Sg[2];
            P[0] = Sg[3] / dS; P[3] = Sg[0] / dS; P[1] = -Sg[1] / dS;
        } else {
            const double c00 = Sg[4] * Sg[8] - Sg[5] * Sg[7];
            const double c01 = Sg[5] * Sg[6] - Sg[3] * Sg[8];
            const double c02 = Sg[3] * Sg[7] - Sg[4] * Sg[6];
            const double c11 = Sg[0] * Sg[8] - Sg[2] * Sg[6];
            const double c12 = Sg[2] * Sg[3] - Sg[0] * Sg[5];
            const double c22 = Sg[0] * Sg[4] - Sg[1] * Sg[3];
            dS = Sg[0] * c00 + Sg[1] * c01 + Sg[2] * c02;
            P[0] = c00 / dS; P[1] = c01 / dS; P[2] = c02 / dS;
            P[4] = c11 / dS; P[5] = c12 / dS; P[8] = c22 / dS;
        }
        const double pref = 1.0 / sqrt(dS);
        const double e2 = 9.0 * tr;
        if (D == 2) {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = pref; r[3] = e2;
            r[4] = P[0]; r[5] = P[1]; r[6] = P[3];
            r[8] = am[0]; r[9] = am[1]; r[10] = am[2];
        } else {
            r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = pref;
            r[4] = P[0]; r[5] = P[1]; r[6] = P[2]; r[7] = P[4];
            r[8] = P[5]; r[9] = P[8]; r[10] = e2;
            r[12] = am[0]; r[13] = am[1]; r[14] = am[2]; r[15] = am[3];
        }
        ext2 = (float)e2;
        bad = !isfinite(nd) || !(dS > 0.0) || !isfinite(dS);
    }
#pragma unroll
    for (int q = 0; q <= D; ++q) bad |= !isfinite(am[q]);
}

template <typename T, int D, int KER>
__global__ void __launch_bounds__(256) k_records(RecArgs a)
{
    pdl_entry();
    constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
    constexpr int RV = record_values(D, KER);
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    float ext2 = 0.0f;
    bool bad = false;
    if (j < nvalid) {
        const uint32_t i = a.perm[j];
        T sv[NP * 4];
#pragma unroll
        for (int p = 0; p < NP; ++p) load4<T>((const T*)a.state, p * a.n + i, sv + 4 * p);
        const uint32_t meta = a.meta[i];
        const fla_batch* B = a.batches + (meta & FLA_META_BATCH_MASK);
        const double n0 = __ldg(&B->n0), h0 = __ldg(&B->h0);
        T r[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = T(0);
        if (sizeof(T) == 4) {
            double adet;
            float n;
            det_and_n<D>(a, (const float*)sv + 2 * D, meta, i, n0, adet, n);
            record_f32<D, KER>(a, (const float*)sv, adet, n, h0, 1.0, (float*)r, ext2, bad);
        }
        else record_f64<D, KER>(a, (const double*)sv, n0, h0, (double*)r, ext2, bad);
#pragma unroll
        for (int v = 0; v < RV / 4; ++v) store4<T>((T*)a.rec, j * (RV / 4) + v, r + 4 * v);
        if (!(ext2 >= 0.0f) || !isfinite(ext2)) ext2 = 0.0f;
    }
    // block maximum of the support extent and the counters: one atomic each per block
    __shared__ float s_ext[8];
    __shared__ unsigned s_bad[8];
    float e = ext2;
    unsigned b = bad ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s_ext[w] = e; s_bad[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        unsigned nb = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { m = fmaxf(m, s_ext[q]); nb += s_bad[q]; }
        const int64_t lo = blockIdx.x * (int64_t)blockDim.x;
        const int64_t cnt = nvalid > lo ? ((nvalid - lo) < (int64_t)blockDim.x ? (nvalid - lo) : (int64_t)blockDim.x) : 0;
        if (m > 0.0f) atomicMax(a.ext_max, __float_as_uint(m));
        if (nb) atomicAdd(&a.status->nonfinite, (unsigned long long)nb);
        if (cnt) atomicAdd(&a.status->deposited, (unsigned long long)cnt);
    }
}

// |det J| below which the learned correction is not applied (see fla.h).
constexpr double kLearnFoldTau = 1e-2;

// Network features of a droplet (see fla.h), single precision.
template <int D>
__device__ __forceinline__ void mlp_features(const float* J, double adet, float n, double h0, double dx, float* f)
{
    float I1 = 0.0f;
#pragma unroll
    for (int q = 0; q < D * D; ++q) I1 = I1 + J[q] * J[q];
    float I2;
    if (D == 2) {
        I2 = (float)(adet * adet);
    } else {
        I2 = 0.0f;
#pragma unroll
        for (int r0 = 0; r0 < 3; ++r0)
#pragma unroll
            for (int r1 = r0 + 1; r1 < 3; ++r1)
#pragma unroll
                for (int c0 = 0; c0 < 3; ++c0)
#pragma unroll
                    for (int c1 = c0 + 1; c1 < 3; ++c1) {
                        const float mnr = J[r0 * 3 + c0] * J[r1 * 3 + c1] - J[r0 * 3 + c1] * J[r1 * 3 + c0];
                        I2 = I2 + mnr * mnr;
                    }
    }
    const float ad = (float)adet;
    const float root = D == 2 ? sqrtf(ad) : cbrtf(ad);
    f[0] = logf(fmaxf(I1, 1e-30f)) * 0.125f;
    f[1] = logf(fmaxf(I2, 1e-30f)) * 0.125f;
    f[2] = logf(fmaxf(ad, 1e-30f)) * 0.125f;
    f[3] = logf(fmaxf(n, 1e-30f)) * 0.125f;
    f[4] = logf(fmaxf((float)(h0 / dx) * root, 1e-30f)) * 0.25f;
    f[5] = fminf(ad, 4.0f) * 0.25f;
}

// Records with the learned correction (single precision; the spherical
// kernel's h or the J-scaled kernel's Lagrangian bandwidth h0 scaled by
// exp(clip(g(f), -2, 2))): persistent CTAs take tiles of 128 sorted positions
// (the packed weights are copied and the TMEM columns allocated once per CTA),
// the network on the tensor cores.
template <int D, int KER>
__global__ void __launch_bounds__(kMlpRows) k_records_mlp(RecArgs a)
{
    pdl_entry();
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
    constexpr int RV = record_values(D, KER);
    const int64_t nvalid = a.bin_start[a.n_cells];
    const int64_t tiles = (nvalid + kMlpRows - 1) / kMlpRows;
    // the grid is sized for every droplet of the cloud; a CTA without a tile of
    // binned records leaves before copying the weights and allocating TMEM
    // (it would contribute nothing to the counters below)
    if ((int64_t)blockIdx.x >= tiles) return;
    MlpCta m = mlp_cta_layout(smem);
    mlp_cta_begin(m, a.mlp);
    float ext_max = 0.0f;
    unsigned n_bad = 0, n_dep = 0;
    bool all_ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t j = tile * kMlpRows + threadIdx.x;
        const bool valid = j < nvalid;
        float sv[NP * 4];
        float f[kMlpIn] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        uint32_t i = 0;
        double adet = 1.0, h0 = 0.0;
        float n = 0.0f;
        if (valid) {
            i = a.perm[j];
#pragma unroll
            for (int p = 0; p < NP; ++p) load4<float>((const float*)a.state, p * a.n + i, sv + 4 * p);
            const uint32_t meta = a.meta[i];
            const fla_batch* B = a.batches + (meta & FLA_META_BATCH_MASK);
            const double n0 = __ldg(&B->n0);
            h0 = __ldg(&B->h0);
            det_and_n<D>(a, sv + 2 * D, meta, i, n0, adet, n);
            mlp_features<D>(sv + 2 * D, adet, n, h0, a.dx, f);
        }
        bool ok = true;
        const float c = mlp_cta_forward(m, f, &ok);
        all_ok &= ok;
        if (valid) {
            // near a fold caustic (|det J| < 1e-2) the plain kernel is the fallback: n is
            // singular there and no bandwidth learned away from it transfers
            const bool fold = adet < kLearnFoldTau;
            const float ct = fold ? 0.0f : fminf(fmaxf(c, -2.0f), 2.0f);
            float r[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) r[q] = 0.0f;
            bool h_free = false, bad = false;
            float ext2 = 0.0f;
            record_f32<D, KER>(a, sv, adet, n, h0, exp((double)ct), r, ext2, bad, &h_free);
#pragma unroll
            for (int v = 0; v < RV / 4; ++v) store4<float>((float*)a.rec, j * (RV / 4) + v, r + 4 * v);
            if (ext2 >= 0.0f && isfinite(ext2)) ext_max = fmaxf(ext_max, ext2);
            n_bad += bad ? 1u : 0u;
            n_dep += 1u;
            if (a.mlp_out) a.mlp_out[i] = c;
            if (a.aux) {
                a.aux[2 * j] = c;
                a.aux[2 * j + 1] = (!fold && h_free && c > -2.0f && c < 2.0f) ? 1.0f : 0.0f;
            }
        }
    }
    if (!all_ok && threadIdx.x == 0) atomicOr(&a.status->flags, kFlagMlpTimeout);
    __shared__ float s_ext[4];
    __shared__ unsigned s_bad[4], s_dep[4];
    float e = ext_max;
    unsigned b = n_bad, dcount = n_dep;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
        b += __shfl_xor_sync(0xffffffffu, b, o);
        dcount += __shfl_xor_sync(0xffffffffu, dcount, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_ext[threadIdx.x >> 5] = e;
        s_bad[threadIdx.x >> 5] = b;
        s_dep[threadIdx.x >> 5] = dcount;
    }
    mlp_cta_end(m);   // synchronises the CTA
    if (threadIdx.x == 0) {
        const float mx = fmaxf(fmaxf(s_ext[0], s_ext[1]), fmaxf(s_ext[2], s_ext[3]));
        const unsigned nb = s_bad[0] + s_bad[1] + s_bad[2] + s_bad[3];
        const unsigned nd = s_dep[0] + s_dep[1] + s_dep[2] + s_dep[3];
        if (mx > 0.0f) atomicMax(a.ext_max, __float_as_uint(mx));
        if (nb) atomicAdd(&a.status->nonfinite, (unsigned long long)nb);
        if (nd) atomicAdd(&a.status->deposited, (unsigned long long)nd);
    }
}

// Backward of the learned correction over tiles of 128 sorted records
// (persistent CTAs): the tensor-core forward is repeated with its
// activations kept in shared memory, then on the CUDA cores
//   d3 = dL/dc W4 silu'(z3), d2 = silu'(z2) W3^T d3, d1 = silu'(z1) W2^T d2
// (BF16 weights as in the forward) and the parameter gradients
//   dW4 = sum dL/dc a3, dW3 = sum d3 a2^T, dW2 = sum d2 a1^T, dW1 = sum d1 a0^T
// and the bias sums, accumulated per thread over the CTA's tiles and written
// as one partial gradient per CTA.
template <int D>
__global__ void __launch_bounds__(kMlpRows, 1) k_learn_backward(RecArgs a, const float* __restrict__ dldc,
                                                                float* __restrict__ partial)
{
    pdl_entry();
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
    constexpr int RP = kLearnRowPad;
    MlpCta m = mlp_cta_layout(smem);
    float* Z1 = reinterpret_cast<float*>(smem + kMlpSmemBytes);
    float* Z2 = Z1 + kMlpRows * RP;
    float* Z3 = Z2 + kMlpRows * RP;
    float* A1 = Z3 + kMlpRows * RP;
    float* A2 = A1 + kMlpRows * RP;
    float* A0 = A2 + kMlpRows * RP;     // 8 per row
    float* GC = A0 + kMlpRows * 8;      // dL/dc per row
    mlp_cta_begin(m, a.mlp);
    const int t = threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    const int64_t tiles = (nvalid + kMlpRows - 1) / kMlpRows;
    const float* w4 = reinterpret_cast<const float*>(m.img + kPkW4);
    float gW3[32], gW2[32], gW1[3];
#pragma unroll
    for (int q = 0; q < 32; ++q) { gW3[q] = 0.0f; gW2[q] = 0.0f; }
    gW1[0] = gW1[1] = gW1[2] = 0.0f;
    float gb1 = 0.0f, gb2 = 0.0f, gb3 = 0.0f, gW4 = 0.0f, gb4 = 0.0f;
    bool all_ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t j = tile * kMlpRows + t;
        float f[kMlpIn] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float g = 0.0f;
        if (j < nvalid) {
            const uint32_t i = a.perm[j];
            float sv[NP * 4];
#pragma unroll
            for (int p = 0; p < NP; ++p) load4<float>((const float*)a.state, p * a.n + i, sv + 4 * p);
            const uint32_t meta = a.meta[i];
            const fla_batch* B = a.batches + (meta & FLA_META_BATCH_MASK);
            double adet;
            float n;
            det_and_n<D>(a, sv + 2 * D, meta, i, __ldg(&B->n0), adet, n);
            mlp_features<D>(sv + 2 * D, adet, n, __ldg(&B->h0), a.dx, f);
            g = dldc[j];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) A0[t * 8 + k] = k < kMlpIn ? __bfloat162float(__float2bfloat16_rn(f[k])) : 0.0f;
        GC[t] = g;
        bool ok = true;
        mlp_cta_forward_keep(m, f, Z1 + t * RP, Z2 + t * RP, Z3 + t * RP, A1 + t * RP, A2 + t * RP, &ok);
        all_ok &= ok;
        __syncthreads();
        // last layer: dW4_k = sum_r g_r silu(z3_rk), db4 = sum_r g_r
        if (t < kMlpH) {
            float sacc = 0.0f;
            for (int r = 0; r < kMlpRows; ++r) sacc = fmaf(GC[r], silu_f(Z3[r * RP + t]), sacc);
            gW4 += sacc;
        }
        if (t == 0) {
            float sacc = 0.0f;
            for (int r = 0; r < kMlpRows; ++r) sacc += GC[r];
            gb4 += sacc;
        }
        __syncthreads();
        // d3 (own row, in place of z3)
        for (int k = 0; k < kMlpH; ++k) Z3[t * RP + k] = g * w4[k] * silu_grad_f(Z3[t * RP + k]);
        __syncthreads();
        // dW3[k][k'] = sum_r d3_rk a2_rk', db3
        {
            const int kp = t & 63, k0 = t >> 6;
            for (int r = 0; r < kMlpRows; ++r) {
                const float av = A2[r * RP + kp];
#pragma unroll
                for (int q = 0; q < 32; ++q) gW3[q] = fmaf(Z3[r * RP + k0 + 2 * q], av, gW3[q]);
            }
            if (t < kMlpH) {
                float sacc = 0.0f;
                for (int r = 0; r < kMlpRows; ++r) sacc += Z3[r * RP + t];
                gb3 += sacc;
            }
        }
        // d2 (own row, in place of z2): silu'(z2_k') sum_k d3_k W3[k][k']
        for (int kp = 0; kp < kMlpH; ++kp) {
            float sacc = 0.0f;
            for (int k = 0; k < kMlpH; ++k) sacc = fmaf(Z3[t * RP + k], img_weight(m.img, kPkW3, k, kp, kMlpH), sacc);
            Z2[t * RP + kp] = sacc * silu_grad_f(Z2[t * RP + kp]);
        }
        __syncthreads();
        {
            const int kp = t & 63, k0 = t >> 6;
            for (int r = 0; r < kMlpRows; ++r) {
                const float av = A1[r * RP + kp];
#pragma unroll
                for (int q = 0; q < 32; ++q) gW2[q] = fmaf(Z2[r * RP + k0 + 2 * q], av, gW2[q]);
            }
            if (t >= kMlpH) {
                float sacc = 0.0f;
                for (int r = 0; r < kMlpRows; ++r) sacc += Z2[r * RP + t - kMlpH];
                gb2 += sacc;
            }
        }
        // d1 (own row, in place of z1): silu'(z1_k'') sum_k' d2_k' W2[k'][k'']
        for (int kq = 0; kq < kMlpH; ++kq) {
            float sacc = 0.0f;
            for (int k = 0; k < kMlpH; ++k) sacc = fmaf(Z2[t * RP + k], img_weight(m.img, kPkW2, k, kq, kMlpH), sacc);
            Z1[t * RP + kq] = sacc * silu_grad_f(Z1[t * RP + kq]);
        }
        __syncthreads();
        {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int e = t + kMlpRows * q;          // W1 entry (k'', f)
                const int kq = e / kMlpIn, fi = e % kMlpIn;
                float sacc = 0.0f;
                for (int r = 0; r < kMlpRows; ++r) sacc = fmaf(Z1[r * RP + kq], A0[r * 8 + fi], sacc);
                gW1[q] += sacc;
            }
            if (t < kMlpH) {
                float sacc = 0.0f;
                for (int r = 0; r < kMlpRows; ++r) sacc += Z1[r * RP + t];
                gb1 += sacc;
            }
        }
        __syncthreads();   // the next tile's forward overwrites the shared arrays
    }
    float* out = partial + (int64_t)blockIdx.x * kMlpParams;
    {
        const int kp = t & 63, k0 = t >> 6;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            out[kOffW3 + (k0 + 2 * q) * kMlpH + kp] = gW3[q];
            out[kOffW2 + (k0 + 2 * q) * kMlpH + kp] = gW2[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) out[kOffW1 + t + kMlpRows * q] = gW1[q];
    if (t < kMlpH) {
        out[kOffB1 + t] = gb1;
        out[kOffB3 + t] = gb3;
        out[kOffW4 + t] = gW4;
    } else {
        out[kOffB2 + t - kMlpH] = gb2;
    }
    if (t == 0) out[kOffB4] = gb4;
    if (!all_ok && t == 0) atomicOr(&a.status->flags, kFlagMlpTimeout);
    mlp_cta_end(m);
}

// Batched clouds of one group (single precision): the sorted positions of the
// group's cells, each record computed as k_records does for its cloud.
// One block of 256 sorted positions from the group's first, block_base on
// (every thread of the CTA takes part: it ends with a CTA barrier).
template <int D, int KER>
__device__ __forceinline__ void batch_records_block(const BatchDev& b, int group, DevStatus* st, int64_t block_base)
{
    constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
    constexpr int RV = record_values(D, KER);
    const int64_t jb = b.bin_start[b.group_cells[group]], je = b.bin_start[b.group_cells[group + 1]];
    const int64_t j = jb + block_base + threadIdx.x;
    float ext2 = 0.0f;
    bool bad = false;
    int k = -1;
    if (j < je) {
        const uint32_t g = b.perm[j];
        k = batch_find(b.drop_pre, b.n_clouds, g);
        const BatchCloud& c = b.clouds[k];
        const int64_t i = g - b.drop_pre[k];
        RecArgs a{};
        a.h_min = c.h_min;
        a.h_max = c.h_max;
        a.p = c.p;
        a.window_dt = c.window_dt;
        a.inv_window = (float)(1.0 / c.window_dt);
        a.room = (float)(c.h_max * c.h_max - (double)D * c.h_min * c.h_min);
        a.hmin2 = (float)(c.h_min * c.h_min);
        a.plain = c.plain;
        a.n = c.n;
        float sv[NP * 4];
#pragma unroll
        for (int p = 0; p < NP; ++p) load4<float>(c.state, p * c.n + i, sv + 4 * p);
        const uint32_t meta = c.meta[i];
        const fla_batch* B = c.batches + (meta & FLA_META_BATCH_MASK);
        double adet;
        float n;
        det_and_n<D>(a, sv + 2 * D, meta, i, __ldg(&B->n0), adet, n);
        float r[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0.0f;
        record_f32<D, KER>(a, sv, adet, n, __ldg(&B->h0), 1.0, r, ext2, bad);
#pragma unroll
        for (int v = 0; v < RV / 4; ++v) store4<float>((float*)b.rec[group], (j - jb) * (RV / 4) + v, r + 4 * v);
        if (!(ext2 >= 0.0f) || !isfinite(ext2)) ext2 = 0.0f;
    }
    // per-cloud maximum support: one atomic per warp when the warp holds one cloud
    const int k0 = __shfl_sync(0xffffffffu, k, 0);
    if (__all_sync(0xffffffffu, k == k0)) {
        float e = ext2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
        if ((threadIdx.x & 31) == 0 && k0 >= 0 && e > 0.0f) atomicMax(b.ext_max + k0, __float_as_uint(e));
    } else if (k >= 0 && ext2 > 0.0f) {
        atomicMax(b.ext_max + k, __float_as_uint(ext2));
    }
    __shared__ unsigned s_cnt[8], s_bad[8];
    const unsigned nv = __reduce_add_sync(0xffffffffu, k >= 0 ? 1u : 0u);
    const unsigned nb = __reduce_add_sync(0xffffffffu, bad ? 1u : 0u);
    if ((threadIdx.x & 31) == 0) { s_cnt[threadIdx.x >> 5] = nv; s_bad[threadIdx.x >> 5] = nb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0, tb = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { tc += s_cnt[q]; tb += s_bad[q]; }
        if (tc) atomicAdd(&st->deposited, tc);
        if (tb) atomicAdd(&st->nonfinite, tb);
    }
    __syncthreads();   // the counters are reused by the next block
}

template <int D, int KER>
__global__ void __launch_bounds__(256) k_batch_records(BatchDev b, int group, DevStatus* st)
{
    pdl_entry();
    batch_records_block<D, KER>(b, group, st, blockIdx.x * (int64_t)blockDim.x);
}

template <typename T, int D, int KER>
cudaError_t launch_t(const RecArgs& a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((a.n + 255) / 256);
    launch_pdl(k_records<T, D, KER>, dim3(blocks), dim3(256), 0, s, a);
    return cudaGetLastError();
}

}  // namespace

namespace {
RecArgs make_rec_args(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg, const uint32_t* perm,
                      const uint32_t* bin_start, int64_t n_cells, void* rec, unsigned int* ext_max, DevStatus* st)
{
    RecArgs a{};
    a.state = cl.state_dev;
    a.meta = cl.meta_dev;
    a.batches = cl.batches_dev;
    a.perm = perm;
    a.bin_start = bin_start;
    a.n = cl.n;
    a.n_cells = n_cells;
    a.h_min = cfg.h_min;
    a.h_max = cfg.h_max;
    a.p = cfg.p;
    a.window_dt = cfg.window_dt;
    a.inv_window = (float)(1.0 / cfg.window_dt);
    a.room = (float)(cfg.h_max * cfg.h_max - (double)m.dim * cfg.h_min * cfg.h_min);
    a.hmin2 = (float)(cfg.h_min * cfg.h_min);
    a.rec = rec;
    a.ext_max = ext_max;
    a.status = st;
    a.fold = (const double*)cl.fold_dev;
    a.plain = cfg.precision == FLA_PREC_PLAIN ? 1 : 0;
    a.mlp = (const unsigned char*)cfg.mlp_dev;
    a.mlp_out = cfg.mlp_out_dev;
    a.dx = 1.0 / m.n;
    a.x2 = cl.dtype == FLA_F32X2 ? 1 : 0;
    return a;
}
}  // namespace

cudaError_t launch_records(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg,
                           const uint32_t* perm, const uint32_t* bin_start, int64_t n_cells, void* rec,
                           unsigned int* ext_max, DevStatus* st, cudaStream_t s, float* aux)
{
    RecArgs a = make_rec_args(cl, m, cfg, perm, bin_start, n_cells, rec, ext_max, st);
    a.aux = aux;
    if (a.n == 0) return cudaSuccess;
    if (a.mlp) {   // validated by the caller: single precision
        // persistent: as many CTAs as fit at once (shared memory allows 6 per SM), at most one per tile
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles = (a.n + kMlpRows - 1) / kMlpRows;
        const unsigned blocks = (unsigned)(tiles < 6LL * sms ? tiles : 6LL * sms);
        const bool iso = cfg.kernel == FLA_KERNEL_ISO;
        if (m.dim == 2) {
            if (iso) launch_pdl(k_records_mlp<2, FLA_KERNEL_ISO>, dim3(blocks), dim3(kMlpRows), kMlpSmemBytes, s, a);
            else launch_pdl(k_records_mlp<2, FLA_KERNEL_ANISO>, dim3(blocks), dim3(kMlpRows), kMlpSmemBytes, s, a);
        } else {
            if (iso) launch_pdl(k_records_mlp<3, FLA_KERNEL_ISO>, dim3(blocks), dim3(kMlpRows), kMlpSmemBytes, s, a);
            else launch_pdl(k_records_mlp<3, FLA_KERNEL_ANISO>, dim3(blocks), dim3(kMlpRows), kMlpSmemBytes, s, a);
        }
        return cudaGetLastError();
    }
    const bool iso = cfg.kernel == FLA_KERNEL_ISO;
    if (cl.dtype != FLA_F64) {   // FLA_F32 and FLA_F32X2 (records from the hi planes)
        if (m.dim == 2) return iso ? launch_t<float, 2, 0>(a, s) : launch_t<float, 2, 1>(a, s);
        return iso ? launch_t<float, 3, 0>(a, s) : launch_t<float, 3, 1>(a, s);
    }
    if (m.dim == 2) return iso ? launch_t<double, 2, 0>(a, s) : launch_t<double, 2, 1>(a, s);
    return iso ? launch_t<double, 3, 0>(a, s) : launch_t<double, 3, 1>(a, s);
}

}  // namespace fla

namespace fla {

cudaError_t launch_learn_backward(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg,
                                  const uint32_t* perm, const uint32_t* bin_start, int64_t n_cells,
                                  const float* dldc, float* partial, int n_parts, DevStatus* st, cudaStream_t s)
{
    RecArgs a = make_rec_args(cl, m, cfg, perm, bin_start, n_cells, nullptr, nullptr, st);
    cudaError_t e;
    if (m.dim == 2) {
        e = cudaFuncSetAttribute(k_learn_backward<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLearnSmemBytes);
        if (e != cudaSuccess) return e;
        k_learn_backward<2><<<n_parts, kMlpRows, kLearnSmemBytes, s>>>(a, dldc, partial);
    } else {
        e = cudaFuncSetAttribute(k_learn_backward<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLearnSmemBytes);
        if (e != cudaSuccess) return e;
        k_learn_backward<3><<<n_parts, kMlpRows, kLearnSmemBytes, s>>>(a, dldc, partial);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_records(const BatchDev& b, int group, DevStatus* st, cudaStream_t s)
{
    const int64_t n = b.group_drops[group];   // upper bound on the group's binned droplets
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    switch (group) {
    case 0: launch_pdl(k_batch_records<2, FLA_KERNEL_ISO>, dim3(blocks), dim3(256), 0, s, b, group, st); break;
    case 1: launch_pdl(k_batch_records<2, FLA_KERNEL_ANISO>, dim3(blocks), dim3(256), 0, s, b, group, st); break;
    case 2: launch_pdl(k_batch_records<3, FLA_KERNEL_ISO>, dim3(blocks), dim3(256), 0, s, b, group, st); break;
    default: launch_pdl(k_batch_records<3, FLA_KERNEL_ANISO>, dim3(blocks), dim3(256), 0, s, b, group, st); break;
    }
    return cudaGetLastError();
}

}  // namespace fla

#ifdef FLA_WINDOW_PHASES
// Phase of the persistent window kernel (window.cuh): the records of one
// group, blocks of 256 sorted positions in a grid-stride loop.
#include "window.cuh"
namespace fla {

namespace {
template <int D, int KER>
__device__ void window_records_t(const BatchDev& b, int group, DevStatus* st)
{
    const int64_t n = b.group_drops[group];   // upper bound on the group's binned droplets
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x)
        batch_records_block<D, KER>(b, group, st, base);
}
}  // namespace

__device__ void window_records(const BatchDev& b, int group, DevStatus* st)
{
    switch (group) {
    case 0: window_records_t<2, FLA_KERNEL_ISO>(b, group, st); break;
    case 1: window_records_t<2, FLA_KERNEL_ANISO>(b, group, st); break;
    case 2: window_records_t<3, FLA_KERNEL_ISO>(b, group, st); break;
    default: window_records_t<3, FLA_KERNEL_ANISO>(b, group, st); break;
    }
}

}  // namespace fla
#endif
