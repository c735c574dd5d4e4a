// Training of the learned bandwidth correction: loss at the training cells,
// dL/dc per droplet through the Nadaraya-Watson ratio (Eqs. 13 and 16), the
// deterministic reduction of the per-CTA parameter gradients, and Adam.
//
// With S_kc = -sum_i w_ic a_ki / D_c, D_c = sum_i w_ic:
//   dS_kc/dw_ic = -(a_ki + S_kc)/D_c,
// and for the spherical kernel, w_ic = exp(-q/2)/h_i, q = r^2/h_i^2 and
// h_i = h_raw,i exp(c_i) (unclamped):   dw_ic/dc_i = w_ic (q - 1);
// for the J-scaled kernel, w_ic = det(Sigma_i)^-1/2 exp(-q/2), q = r'P_i r,
// Sigma_i = e^(2 c_i) A_i + h_min^2 I (below the trace cap):
//   dw_ic/dc_i = w_ic ((q - h_min^2 |P_i r|^2) - (d - h_min^2 tr P_i)).
// With g_kc = dL/dS_kc and per-cell H_kc = g_kc/D_c, G_c = sum_k g_kc S_kc:
//   dL/dc_i = -sum_c dw_ic/dc_i (sum_k H_kc a_ki + G_c/D_c),
// a gather over the cells inside droplet i's truncated support.  The
// truncation edge is held fixed.
#include "mlp_tc.cuh"

namespace fla {
namespace {

constexpr int kNormThreads = 512;

// Single block: per component k, norm_k = sum_o T_ko^2 and sse_k = sum_o (S_ko - T_ko)^2
// in a fixed order (double precision); loss += sum_k sse_k/norm_k / (1 + dim).
__global__ void __launch_bounds__(kNormThreads) k_learn_norms(LearnArgs a)
{
    const int K = 1 + a.dim;
    __shared__ double s_n[4][kNormThreads];
    __shared__ double s_e[4][kNormThreads];
    double pn[4] = {0, 0, 0, 0}, pe[4] = {0, 0, 0, 0};
    for (int64_t o = threadIdx.x; o < a.n_train; o += kNormThreads) {
        const int64_t c = a.cells[o];
        for (int k = 0; k < K; ++k) {
            const double S = k == 0 ? a.s_mass[c] : a.s_mom[(int64_t)(k - 1) * a.n_cells + c];
            const double T = a.targets[o * K + k];
            pn[k] += T * T;
            pe[k] += (S - T) * (S - T);
        }
    }
    for (int k = 0; k < 4; ++k) {
        s_n[k][threadIdx.x] = pn[k];
        s_e[k][threadIdx.x] = pe[k];
    }
    __syncthreads();
    for (int w = kNormThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 4; ++k) {
                s_n[k][threadIdx.x] += s_n[k][threadIdx.x + w];
                s_e[k][threadIdx.x] += s_e[k][threadIdx.x + w];
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double L = 0.0;
        for (int k = 0; k < K; ++k) {
            a.scal[k] = (float)s_n[k][0];
            if (s_n[k][0] > 0.0) L += s_e[k][0] / s_n[k][0];
        }
        *a.loss += (float)(L / K);
    }
}

// Per training cell: H_kc = g_kc / D_c and G_c / D_c (zero where D_c = 0).
__global__ void k_learn_cells(LearnArgs a)
{
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= a.n_train) return;
    const int K = 1 + a.dim;
    const int64_t c = a.cells[o];
    const float D = a.dsum[c];
    float* q = a.q + c * a.q_stride;
    if (!(D > 0.0f)) {
        for (int k = 0; k <= K; ++k) q[k] = 0.0f;
        return;
    }
    float G = 0.0f;
    for (int k = 0; k < K; ++k) {
        const float S = k == 0 ? a.s_mass[c] : a.s_mom[(int64_t)(k - 1) * a.n_cells + c];
        const float T = a.targets[o * K + k];
        const float nk = a.scal[k];
        const float g = nk > 0.0f ? 2.0f * (S - T) / (nk * (float)K) : 0.0f;
        q[k] = g / D;
        G = fmaf(g, S, G);
    }
    q[K] = G / D;
}

// dL/dc per sorted record (spherical kernel, single precision): the cells of
// the support, decided as the gathers decide them (r^2 = dx^2 + dy^2 (+ dz^2)
// with fused multiply-adds, r^2 <= 9 h^2).
template <int D>
__global__ void k_learn_dc(LearnArgs a)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    if (j >= nvalid) return;
    if (!(a.aux[2 * j + 1] > 0.0f)) {   // h does not move with c (clipped or clamped)
        a.dldc[j] = 0.0f;
        return;
    }
    constexpr int RV = D == 2 ? 8 : 12;
    const float* r = reinterpret_cast<const float*>(a.rec) + j * RV;
    const float x[3] = {r[0], r[1], D == 3 ? r[2] : 0.0f};
    const float cexp = D == 2 ? r[2] : r[4];     // -log2(e) / (2 h^2)
    const float lih = D == 2 ? r[3] : r[5];      // log2(1/h)
    const float r2max = D == 2 ? r[7] : r[3];
    const float* am = D == 2 ? r + 4 : r + 8;
    const int N = a.N;
    const float fN = (float)N;
    const float R = sqrtf(r2max);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < D; ++q) {
        lo[q] = max(0, (int)floorf((x[q] - R) * fN - 0.5f) - 1);
        hi[q] = min(N - 1, (int)ceilf((x[q] + R) * fN - 0.5f) + 1);
    }
    const int K = 1 + D;
    float acc = 0.0f;
    for (int iz = lo[2]; iz <= hi[2]; ++iz) {
        const float dz = D == 3 ? __fsub_rn(((float)iz + 0.5f) / fN, x[2]) : 0.0f;
        for (int iy = lo[1]; iy <= hi[1]; ++iy) {
            const float dy = __fsub_rn(((float)iy + 0.5f) / fN, x[1]);
            for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                const float dx = __fsub_rn(((float)ix + 0.5f) / fN, x[0]);
                float r2 = __fmul_rn(dx, dx);
                r2 = __fmaf_rn(dy, dy, r2);
                if (D == 3) r2 = __fmaf_rn(dz, dz, r2);
                if (!(r2 <= r2max)) continue;
                const int64_t cell = ix + (int64_t)N * (iy + (int64_t)N * iz);
                const float* qc = a.q + cell * a.q_stride;
                float t = qc[K];
#pragma unroll
                for (int k = 0; k < K; ++k) t = fmaf(qc[k], am[k], t);
                if (t == 0.0f) continue;
                const float w = exp2f(fmaf(r2, cexp, lih));
                const float qq = -1.38629436111989061883f * cexp * r2;   // r^2 / h^2
                acc = fmaf(-w * (qq - 1.0f), t, acc);
            }
        }
    }
    a.dldc[j] = acc;
}

// dL/dc per sorted record, J-scaled kernel (single precision): the cells of
// the support's bounding box, each decided as the gathers decide it (P r, then
// r'(P r), with fused multiply-adds, q <= 9).  Records: 2D (x, y, lpref, 9 tr
// Sigma | P00, P01, P11, 0 | a_m, a_x, a_y, 0), 3D (x, y, z, lpref | P00, P01,
// P02, P11 | P12, P22, 9 tr Sigma, 0 | a_m, a_x, a_y, a_z).
template <int D>
__global__ void k_learn_dc_aniso(LearnArgs a)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nvalid = a.bin_start[a.n_cells];
    if (j >= nvalid) return;
    if (!(a.aux[2 * j + 1] > 0.0f)) {   // Sigma does not move with c (clipped, capped or near a fold)
        a.dldc[j] = 0.0f;
        return;
    }
    constexpr int RV = D == 2 ? 12 : 16;
    const float* r = reinterpret_cast<const float*>(a.rec) + j * RV;
    float x[3] = {r[0], r[1], D == 3 ? r[2] : 0.0f};
    float P[9];
    float lpref, e2;
    const float* am;
    if (D == 2) {
        lpref = r[2]; e2 = r[3];
        P[0] = r[4]; P[1] = r[5]; P[2] = r[5]; P[3] = r[6];
        am = r + 8;
    } else {
        lpref = r[3]; e2 = r[10];
        P[0] = r[4]; P[1] = r[5]; P[2] = r[6];
        P[3] = r[5]; P[4] = r[7]; P[5] = r[8];
        P[6] = r[6]; P[7] = r[8]; P[8] = r[9];
        am = r + 12;
    }
    float trP = 0.0f;
#pragma unroll
    for (int q = 0; q < D; ++q) trP += P[q * D + q];
    const float base = (float)D - a.hmin2 * trP;
    const int N = a.N;
    const float fN = (float)N;
    const float R = sqrtf(e2);       // the support lies within 3 sqrt(tr Sigma) of x
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < D; ++q) {
        lo[q] = max(0, (int)floorf((x[q] - R) * fN - 0.5f) - 1);
        hi[q] = min(N - 1, (int)ceilf((x[q] + R) * fN - 0.5f) + 1);
    }
    const int K = 1 + D;
    float acc = 0.0f;
    for (int iz = lo[2]; iz <= hi[2]; ++iz)
        for (int iy = lo[1]; iy <= hi[1]; ++iy)
            for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                const int ic[3] = {ix, iy, iz};
                float df[3];
#pragma unroll
                for (int q = 0; q < D; ++q) df[q] = __fsub_rn(((float)ic[q] + 0.5f) / fN, x[q]);
                float pd[3];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float t = __fmul_rn(P[i * D], df[0]);
#pragma unroll
                    for (int k = 1; k < D; ++k) t = __fmaf_rn(P[i * D + k], df[k], t);
                    pd[i] = t;
                }
                float q = __fmul_rn(pd[0], df[0]);
#pragma unroll
                for (int i = 1; i < D; ++i) q = __fmaf_rn(pd[i], df[i], q);
                if (!(q <= 9.0f)) continue;
                const int64_t cell = ix + (int64_t)N * (iy + (int64_t)N * iz);
                const float* qc = a.q + cell * a.q_stride;
                float t = qc[K];
#pragma unroll
                for (int k = 0; k < K; ++k) t = fmaf(qc[k], am[k], t);
                if (t == 0.0f) continue;
                float pr2 = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) pr2 = fmaf(pd[i], pd[i], pr2);
                const float w = exp2f(fmaf(q, -0.72134752044448170368f, lpref));
                acc = fmaf(-w * ((q - a.hmin2 * pr2) - base), t, acc);
            }
    a.dldc[j] = acc;
}

// grad[p] += sum over the backward CTAs of their partial gradients, in CTA order.
__global__ void k_grad_reduce(const float* __restrict__ partial, int n_parts, float* __restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpParams) return;
    float s = 0.0f;
    for (int b = 0; b < n_parts; ++b) s += partial[(int64_t)b * kMlpParams + p];
    grad[p] += s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

cudaError_t launch_learn_cells(const LearnArgs& a, cudaStream_t s)
{
    if (cudaMemsetAsync(a.q, 0, (size_t)a.n_cells * a.q_stride * 4, s) != cudaSuccess) return cudaGetLastError();
    k_learn_norms<<<1, kNormThreads, 0, s>>>(a);
    if (a.n_train > 0) k_learn_cells<<<(unsigned)((a.n_train + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_learn_dc(const LearnArgs& a, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    if (a.kernel == FLA_KERNEL_ISO) {
        if (a.dim == 2) k_learn_dc<2><<<blocks, 128, 0, s>>>(a);
        else k_learn_dc<3><<<blocks, 128, 0, s>>>(a);
    } else {
        if (a.dim == 2) k_learn_dc_aniso<2><<<blocks, 128, 0, s>>>(a);
        else k_learn_dc_aniso<3><<<blocks, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const float* partial, int n_parts, float* grad, cudaStream_t s)
{
    k_grad_reduce<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, n_parts, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace fla
