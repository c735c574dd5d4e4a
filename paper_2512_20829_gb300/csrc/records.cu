// Droplet records for the kernel-regression gather, written in sorted order.
//
// Per binned droplet (Eq. 6, Eq. 15, Eq. 14 and App. B parcel level c):
//   det J in double precision from the stored J,
//   n = n0 / max(|det J|, 1e-12),  a = n * acc / T_window,
//   ISO:   h = clamp(h0 |det J|^p, h_min, h_max), weight (1/h) exp(-r^2/(2 h^2)),
//   ANISO: Sigma = f h0^2 J J^T + h_min^2 I, f = min(1, (h_max^2 - d h_min^2)/tr(h0^2 J J^T)),
//          weight det(Sigma)^-1/2 exp(-d^T Sigma^-1 d / 2).
// This file is compiled without FMA contraction: the double-precision values
// that decide the truncation test (h, Sigma^-1) are formed with one rounding
// per operation in a fixed order, so the decision is reproducible.
#include "fla_internal.cuh"

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
    int kernel;
    double h_min, h_max, p, window_dt;
    void* rec;
    unsigned int* ext_max;      // max over droplets of the squared support radius (float bits)
    DevStatus* status;
};

template <typename T, int D>
__device__ __forceinline__ double det_of(const T* J)
{
    if (D == 2) return (double)J[0] * (double)J[3] - (double)J[1] * (double)J[2];
    const double j0 = J[0], j1 = J[1], j2 = J[2], j3 = J[3], j4 = J[4], j5 = J[5], j6 = J[6], j7 = J[7], j8 = J[8];
    return j0 * (j4 * j8 - j5 * j7) - j1 * (j3 * j8 - j5 * j6) + j2 * (j3 * j7 - j4 * j6);
}

template <typename T, int D, int KER>
__global__ void __launch_bounds__(256) k_records(RecArgs a)
{
    constexpr int NP = state_planes(FLA_CLOUD_FLA, D);
    constexpr int OJ = 2 * D;
    constexpr int OA = acc_offset(FLA_CLOUD_FLA, D);
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
        const fla_batch* B = a.batches + (a.meta[i] & FLA_META_BATCH_MASK);
        const double n0 = __ldg(&B->n0), h0 = __ldg(&B->h0);
        const T* J = sv + OJ;
        const double det = det_of<T, D>(J);
        const double adet = fabs(det);
        const double nd = n0 / (adet > 1e-12 ? adet : 1e-12);
        T r[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = T(0);
        T am[4];
#pragma unroll
        for (int q = 0; q <= D; ++q) am[q] = T(nd * (double)sv[OA + q] / a.window_dt);
        if (KER == FLA_KERNEL_ISO) {
            double h = (a.p == 1.0) ? h0 * adet : h0 * pow(adet, a.p);
            h = h < a.h_min ? a.h_min : h;
            h = h > a.h_max ? a.h_max : h;
            const T hT = T(h);
            const T r2max = T(9.0 * (double)hT * (double)hT);
            const T c = sizeof(T) == 4 ? T(-0.72134752044448170368 / (h * h)) : T(-0.5 / (h * h));
            const T inv_h = T(1.0 / h);
            if (D == 2) {
                r[0] = sv[0]; r[1] = sv[1]; r[2] = c; r[3] = inv_h;
                r[4] = am[0]; r[5] = am[1]; r[6] = am[2]; r[7] = r2max;
            } else {
                r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = r2max;
                r[4] = c; r[5] = inv_h;
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
                    for (int jj = 0; jj < D; ++jj) s += (double)J[ii * D + jj] * (double)J[k * D + jj];
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
            double P[9];
            double dS;
            if (D == 2) {
                dS = Sg[0] * Sg[3] - Sg[1] * Sg[2];
                P[0] = Sg[3] / dS; P[3] = Sg[0] / dS; P[1] = -Sg[1] / dS; P[2] = P[1];
            } else {
                dS = Sg[0] * (Sg[4] * Sg[8] - Sg[5] * Sg[7]) - Sg[1] * (Sg[3] * Sg[8] - Sg[5] * Sg[6]) +
                     Sg[2] * (Sg[3] * Sg[7] - Sg[4] * Sg[6]);
                const double c00 = Sg[4] * Sg[8] - Sg[5] * Sg[7];
                const double c01 = Sg[5] * Sg[6] - Sg[3] * Sg[8];
                const double c02 = Sg[3] * Sg[7] - Sg[4] * Sg[6];
                const double c11 = Sg[0] * Sg[8] - Sg[2] * Sg[6];
                const double c12 = Sg[2] * Sg[3] - Sg[0] * Sg[5];
                const double c22 = Sg[0] * Sg[4] - Sg[1] * Sg[3];
                P[0] = c00 / dS; P[1] = c01 / dS; P[2] = c02 / dS;
                P[4] = c11 / dS; P[5] = c12 / dS; P[8] = c22 / dS;
            }
            const T pref = T(1.0 / sqrt(dS));
            const T e2 = T(9.0 * tr);
            if (D == 2) {
                r[0] = sv[0]; r[1] = sv[1]; r[2] = pref; r[3] = e2;
                r[4] = T(P[0]); r[5] = T(P[1]); r[6] = T(P[3]);
                r[8] = am[0]; r[9] = am[1]; r[10] = am[2];
            } else {
                r[0] = sv[0]; r[1] = sv[1]; r[2] = sv[2]; r[3] = pref;
                r[4] = T(P[0]); r[5] = T(P[1]); r[6] = T(P[2]); r[7] = T(P[4]);
                r[8] = T(P[5]); r[9] = T(P[8]); r[10] = e2;
                r[12] = am[0]; r[13] = am[1]; r[14] = am[2]; r[15] = am[3];
            }
            ext2 = (float)e2;
            bad = !isfinite(nd) || !(dS > 0.0) || !isfinite(dS);
        }
#pragma unroll
        for (int q = 0; q <= D; ++q) bad |= !isfinite((double)am[q]);
#pragma unroll
        for (int v = 0; v < RV / 4; ++v) store4<T>((T*)a.rec, j * (RV / 4) + v, r + 4 * v);
        if (!(ext2 >= 0.0f) || !isfinite(ext2)) ext2 = 0.0f;
    }
    // block maximum of the support extent, one atomic per block
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
        int cnt = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { m = fmaxf(m, s_ext[q]); nb += s_bad[q]; }
        const int64_t lo = blockIdx.x * (int64_t)blockDim.x;
        cnt = (int)(nvalid > lo ? ((nvalid - lo) < (int64_t)blockDim.x ? (nvalid - lo) : (int64_t)blockDim.x) : 0);
        if (m > 0.0f) atomicMax(a.ext_max, __float_as_uint(m));
        if (nb) atomicAdd(&a.status->nonfinite, (unsigned long long)nb);
        if (cnt) atomicAdd(&a.status->deposited, (unsigned long long)cnt);
    }
}

template <typename T, int D, int KER>
cudaError_t launch_t(const RecArgs& a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((a.n + 255) / 256);
    k_records<T, D, KER><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_records(const fla_cloud& cl, const fla_mesh& m, const fla_deposit_cfg& cfg,
                           const uint32_t* perm, const uint32_t* bin_start, int64_t n_cells, void* rec,
                           unsigned int* ext_max, DevStatus* st, cudaStream_t s)
{
    RecArgs a{};
    a.state = cl.state_dev;
    a.meta = cl.meta_dev;
    a.batches = cl.batches_dev;
    a.perm = perm;
    a.bin_start = bin_start;
    a.n = cl.n;
    a.n_cells = n_cells;
    a.kernel = cfg.kernel;
    a.h_min = cfg.h_min;
    a.h_max = cfg.h_max;
    a.p = cfg.p;
    a.window_dt = cfg.window_dt;
    a.rec = rec;
    a.ext_max = ext_max;
    a.status = st;
    if (a.n == 0) return cudaSuccess;
    const bool iso = cfg.kernel == FLA_KERNEL_ISO;
    if (cl.dtype == FLA_F32) {
        if (m.dim == 2) return iso ? launch_t<float, 2, 0>(a, s) : launch_t<float, 2, 1>(a, s);
        return iso ? launch_t<float, 3, 0>(a, s) : launch_t<float, 3, 1>(a, s);
    }
    if (m.dim == 2) return iso ? launch_t<double, 2, 0>(a, s) : launch_t<double, 2, 1>(a, s);
    return iso ? launch_t<double, 3, 0>(a, s) : launch_t<double, 3, 1>(a, s);
}

}  // namespace fla
