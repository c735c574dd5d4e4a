// Analytic carrier velocity and gradient sampled on the mesh nodes.
//
// The paper's carrier is an incompressible Navier-Stokes solution (Eq. 1);
// the droplet equations need u and grad u at the droplet position (Eqs. 3
// and 8).  Here synthetic analytic carriers stand in for it: they are sampled
// once per carrier step on the (n+1)^dim mesh nodes and the advance kernel
// interpolates the node values, as a mesh-based solver would.
#include "batch.cuh"

namespace fla {
namespace {

struct CarrierArgs {
    int kind, dim, N, n_vortex;
    double U[3], A[9], xref[3];
    double vort[FLA_MAX_VORTICES][5];  // centre x at the sampling time (wrapped), yc, 1/rc^2, c/rc^2, c/rc^4
    double jet_width, abc[3], jet_amp, jet_radius;
    // the same values rounded to single precision once, for the single-precision
    // kernels (a conversion from double per node would run on the FP64 pipe)
    float Uf[3], Af[9], xreff[3];
    float vortf[FLA_MAX_VORTICES][5];
    float jet_width_f, abcf[3], jet_amp_f, jet_radius_f;
};

// A carrier constant in the kernel's precision.
template <typename T> __device__ __forceinline__ T cv(double d, float f);
template <> __device__ __forceinline__ float cv<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double cv<double>(double d, float) { return d; }

__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_sinpi(float x) { return sinpif(x); }
__device__ __forceinline__ double m_sinpi(double x) { return sinpi(x); }
__device__ __forceinline__ float m_cospi(float x) { return cospif(x); }
__device__ __forceinline__ double m_cospi(double x) { return cospi(x); }

// Lamb-Oseen vortex, azimuthal speed Gam/(2 pi rho) (1 - exp(-rho^2/rc^2)),
// written u = f(s) (-dy, dx) with s = rho^2, X = s/rc^2:
//   f  = (c/a) h(X),    h(X) = (1 - e^-X)/X,
//   f' = (c/a^2) g(X),  g(X) = (X e^-X - (1 - e^-X))/X^2,
// with a = rc^2, c = Gam/(2 pi); h and g use their Taylor series near X = 0.
// inv_a = 1/a, ca = c/a and ca2 = c/a^2 are formed on the host.
// Single precision: the series near X = 0, expm1 up to X = 1.5 (where e^-X - 1
// and X e^-X + e^-X - 1 would otherwise cancel), and the fast exponential and
// reciprocal above, where neither cancels (error below 1e-6 relative).
__device__ __forceinline__ void lo_hg(float X, float& h, float& g)
{
    if (X < 1e-2f) {
        h = 1.0f + X * (-0.5f + X * (1.0f / 6.0f + X * (-1.0f / 24.0f)));
        g = -0.5f + X * (1.0f / 3.0f + X * (-0.125f + X * (1.0f / 30.0f)));
    } else if (X < 1.5f) {
        const float em = expm1f(-X);   // e^-X - 1
        const float iX = 1.0f / X;
        h = -em * iX;
        g = (X * (em + 1.0f) + em) * iX * iX;
    } else {   // the path nearly every node takes: approximate reciprocal (<= 2 ulp)
        const float e = __expf(-X);
        const float iX = __fdividef(1.0f, X);
        h = (1.0f - e) * iX;
        g = (X * e + (e - 1.0f)) * iX * iX;
    }
}
__device__ __forceinline__ void lo_hg(double X, double& h, double& g)
{
    if (X > 45.0) {   // e^-X < 2^-64: the general branch would give exactly these values
        const double iX = 1.0 / X;
        h = iX;
        g = -iX * iX;
        return;
    }
    if (X < 1e-3) {
        h = 1.0 + X * (-0.5 + X * (1.0 / 6.0 + X * (-1.0 / 24.0)));
        g = -0.5 + X * (1.0 / 3.0 + X * (-0.125 + X * (1.0 / 30.0)));
    } else {
        const double em = expm1(-X);    // e^-X - 1
        const double iX = 1.0 / X;
        h = -em * iX;
        g = (X * (em + 1.0) + em) * iX * iX;
    }
}

template <typename T>
__device__ __forceinline__ void lamb_oseen(T inv_a, T ca, T ca2, T xc, T yc, T x, T y, T* u, T* G)
{
    const T dx = x - xc, dy = y - yc;
    const T X = (dx * dx + dy * dy) * inv_a;
    T h, g;
    lo_hg(X, h, g);
    const T f = ca * h;
    const T fp2 = T(2) * ca2 * g;
    u[0] -= dy * f;
    u[1] += dx * f;
    G[0] -= fp2 * dx * dy;
    G[1] -= f + fp2 * dy * dy;
    G[2] += f + fp2 * dx * dx;
    G[3] += fp2 * dx * dy;
}

template <typename T, int D>
__device__ void eval_carrier(const CarrierArgs& p, const T* x, T* u, T* G)
{
#pragma unroll
    for (int i = 0; i < D; ++i) u[i] = T(0);
#pragma unroll
    for (int i = 0; i < D * D; ++i) G[i] = T(0);
    switch (p.kind) {
    case FLA_CARRIER_UNIFORM:
        for (int i = 0; i < D; ++i) u[i] = cv<T>(p.U[i], p.Uf[i]);
        break;
    case FLA_CARRIER_LINEAR:
        for (int i = 0; i < D; ++i) {
            T s = cv<T>(p.U[i], p.Uf[i]);
            for (int j = 0; j < D; ++j) {
                s += cv<T>(p.A[3 * i + j], p.Af[3 * i + j]) * (x[j] - cv<T>(p.xref[j], p.xreff[j]));
                G[i * D + j] = cv<T>(p.A[3 * i + j], p.Af[3 * i + j]);
            }
            u[i] = s;
        }
        break;
    case FLA_CARRIER_TG2:
        if (D == 2) {
            const T sx = m_sinpi(x[0]), cx = m_cospi(x[0]);
            const T sy = m_sinpi(x[1]), cy = m_cospi(x[1]);
            const T pi = T(3.14159265358979323846);
            u[0] = sx * cy;
            u[1] = -cx * sy;
            G[0] = pi * cx * cy;
            G[1] = -pi * sx * sy;
            G[2] = pi * sx * sy;
            G[3] = -pi * cx * cy;
        }
        break;
    case FLA_CARRIER_JETVORT2:
        if (D == 2) {
            const T w = cv<T>(p.jet_width, p.jet_width_f);
            const T eta = (x[1] - T(0.5)) / w;
            const T uj = m_exp(-eta * eta);
            u[0] = uj;
            G[1] = T(-2) * eta / w * uj;
            for (int k = 0; k < p.n_vortex; ++k) {
                const T xc = cv<T>(p.vort[k][0], p.vortf[k][0]), yc = cv<T>(p.vort[k][1], p.vortf[k][1]);
                const T inv_a = cv<T>(p.vort[k][2], p.vortf[k][2]), ca = cv<T>(p.vort[k][3], p.vortf[k][3]);
                const T ca2 = cv<T>(p.vort[k][4], p.vortf[k][4]);
                for (int img = -1; img <= 1; ++img)   // periodic images along x
                    lamb_oseen<T>(inv_a, ca, ca2, xc + T(img), yc, x[0], x[1], u, G);
            }
        }
        break;
    case FLA_CARRIER_ABCJET3:
        if (D == 3) {
            const T A = cv<T>(p.abc[0], p.abcf[0]), B = cv<T>(p.abc[1], p.abcf[1]), C = cv<T>(p.abc[2], p.abcf[2]);
            const T k = T(6.28318530717958647692);
            const T sxv = m_sinpi(T(2) * x[0]), cxv = m_cospi(T(2) * x[0]);
            const T syv = m_sinpi(T(2) * x[1]), cyv = m_cospi(T(2) * x[1]);
            const T szv = m_sinpi(T(2) * x[2]), czv = m_cospi(T(2) * x[2]);
            u[0] = A * szv + C * cyv;
            u[1] = B * sxv + A * czv;
            u[2] = C * syv + B * cxv;
            G[1] = -k * C * syv;
            G[2] = k * A * czv;
            G[3] = k * B * cxv;
            G[5] = -k * A * szv;
            G[6] = -k * B * sxv;
            G[7] = k * C * cyv;
            const T rx = x[0] - T(0.5), ry = x[1] - T(0.5);
            const T jr = cv<T>(p.jet_radius, p.jet_radius_f);
            const T r2j = jr * jr;
            const T e = cv<T>(p.jet_amp, p.jet_amp_f) * m_exp(-(rx * rx + ry * ry) / r2j);
            u[2] += e;
            G[6] += T(-2) * rx / r2j * e;
            G[7] += T(-2) * ry / r2j * e;
        }
        break;
    default:
        break;
    }
}

// u and grad u at node k (x fastest) written as one node record.
template <typename T, int D>
__device__ __forceinline__ void sample_node(const CarrierArgs& p, T* __restrict__ nodes, int64_t k)
{
    const int nn = p.N + 1;
    T x[3];
    int64_t r = k;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = T(r % nn) / T(p.N);   // node coordinate i/N in the storage precision
        r /= nn;
    }
    T u[3], G[9];
    eval_carrier<T, D>(p, x, u, G);
    constexpr int S = node_stride(D);
    T out[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) out[a] = u[a];
#pragma unroll
    for (int q = 0; q < D * D; ++q) out[D + q] = G[q];
#pragma unroll
    for (int v = 0; v < S / 4; ++v) store4<T>(nodes, k * (S / 4) + v, out + 4 * v);
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_carrier_sample(CarrierArgs p, T* __restrict__ nodes, int64_t total)
{
    pdl_entry();
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= total) return;
    sample_node<T, D>(p, nodes, k);
}

// Double-float nodes (FLA_F32X2), first pass: each value evaluated in double
// precision and stored as the nearest float (first array) and the nearest
// float to the remainder (second array, n_nodes * stride values further on);
// the largest |value| of each component goes to its word of the tail (float
// bits, cleared before the launch).
template <int D>
__global__ void __launch_bounds__(256) k_carrier_sample_x2(CarrierArgs p, float* __restrict__ nodes, int64_t total)
{
    pdl_entry();
    constexpr int S = node_stride(D);
    __shared__ unsigned int s_max[S];
    if (threadIdx.x < S) s_max[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float hi[12], lo[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) hi[q] = lo[q] = 0.0f;
    if (k < total) {
        const int nn = p.N + 1;
        double x[3];
        int64_t r = k;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            x[a] = (double)(r % nn) / (double)p.N;
            r /= nn;
        }
        double u[3], G[9];
        eval_carrier<double, D>(p, x, u, G);
        double v[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = u[a];
#pragma unroll
        for (int q = 0; q < D * D; ++q) v[D + q] = G[q];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            hi[q] = __double2float_rn(v[q]);
            lo[q] = __double2float_rn(__dsub_rn(v[q], (double)hi[q]));
        }
#pragma unroll
        for (int c = 0; c < S / 4; ++c) {
            store4<float>(nodes, k * (S / 4) + c, hi + 4 * c);
            store4<float>(nodes + total * S, k * (S / 4) + c, lo + 4 * c);
        }
    }
    // |x| of a float orders like its bit pattern without the sign
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(hi[q]) & 0x7fffffffu);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(&s_max[q], m);
    }
    __syncthreads();
    if (threadIdx.x < S && s_max[threadIdx.x])
        atomicMax(reinterpret_cast<unsigned int*>(nodes + 2 * total * S) + threadIdx.x, s_max[threadIdx.x]);
}

// Second pass: each value v = hi + lo becomes a + b with a = RN(hi / Q) Q on
// the component's grid Q = 2^(e - 11), where 2^e bounds the component's
// largest |hi| (so |a / Q| <= 2^11, a has at most 12 significant bits), and
// b = RN((hi - a) + lo) (hi - a is exact; |b| <= Q/2 + 2^(e - 25)).  a + b
// is within 2^-24 |b|, about 2^(e - 36), of v.  The advance then sums weights
// on a 2^-10 grid times a exactly in single precision (products of at most 22
// bits on a common grid, partial sums below 2^24 units) and everything else,
// 2^-11 of the value's scale, in plain single precision.
template <int D>
__global__ void __launch_bounds__(256) k_carrier_split_x2(float* __restrict__ nodes, int64_t total)
{
    pdl_entry();
    constexpr int S = node_stride(D);
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= total * (S / 4)) return;
    const int c0 = (int)(k % (S / 4)) * 4;
    const unsigned int* mx = reinterpret_cast<const unsigned int*>(nodes + 2 * total * S);
    float hi[4], lo[4];
    load4<float>(nodes, k, hi);
    load4<float>(nodes + total * S, k, lo);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int e;
        frexpf(__uint_as_float(mx[c0 + q]), &e);     // largest |hi| < 2^e (e = 0 for an all-zero component)
        const float iq = ldexpf(1.0f, 11 - e), qq = ldexpf(1.0f, e - 11);
        const float a = __fmul_rn(rintf(__fmul_rn(hi[q], iq)), qq);
        lo[q] = __fadd_rn(__fsub_rn(hi[q], a), lo[q]);
        hi[q] = a;
    }
    store4<float>(nodes, k, hi);
    store4<float>(nodes + total * S, k, lo);
}

// The carrier's arguments at time t (vortex centres carried with the jet and
// wrapped; Lamb-Oseen constants), each operation rounded once.
__host__ __device__ inline CarrierArgs carrier_args(const fla_carrier_desc& c, int N, double t)
{
    CarrierArgs p{};
    p.kind = c.kind;
    p.dim = c.dim;
    p.N = N;
    p.n_vortex = c.n_vortex;
    for (int i = 0; i < 3; ++i) {
        p.U[i] = c.U[i];
        p.xref[i] = c.xref[i];
        p.abc[i] = c.abc[i];
    }
    for (int i = 0; i < 9; ++i) p.A[i] = c.A[i];
    for (int k = 0; k < c.n_vortex && k < FLA_MAX_VORTICES; ++k) {
#ifdef __CUDA_ARCH__
        double xc = __dadd_rn(c.vortex[k][0], __dmul_rn(c.vortex[k][4], t));
        xc = __dsub_rn(xc, floor(xc));
        const double rc2 = __dmul_rn(c.vortex[k][3], c.vortex[k][3]);
        const double cg = __ddiv_rn(c.vortex[k][2], 2.0 * 3.14159265358979323846);
        p.vort[k][2] = __ddiv_rn(1.0, rc2);
        p.vort[k][3] = __ddiv_rn(cg, rc2);
        p.vort[k][4] = __ddiv_rn(cg, __dmul_rn(rc2, rc2));
#else
        double xc = c.vortex[k][0] + c.vortex[k][4] * t;   // carried with the jet
        xc -= floor(xc);                                   // wrapped into [0, 1)
        const double rc2 = c.vortex[k][3] * c.vortex[k][3];
        const double cg = c.vortex[k][2] / (2.0 * 3.14159265358979323846);   // Gamma / (2 pi)
        p.vort[k][2] = 1.0 / rc2;
        p.vort[k][3] = cg / rc2;
        p.vort[k][4] = cg / (rc2 * rc2);
#endif
        p.vort[k][0] = xc;
        p.vort[k][1] = c.vortex[k][1];
    }
    p.jet_width = c.jet_width;
    p.jet_amp = c.jet_amp;
    p.jet_radius = c.jet_radius;
    for (int i = 0; i < 3; ++i) {
        p.Uf[i] = (float)p.U[i];
        p.xreff[i] = (float)p.xref[i];
        p.abcf[i] = (float)p.abc[i];
    }
    for (int i = 0; i < 9; ++i) p.Af[i] = (float)p.A[i];
    for (int k = 0; k < FLA_MAX_VORTICES; ++k)
        for (int q = 0; q < 5; ++q) p.vortf[k][q] = (float)p.vort[k][q];
    p.jet_width_f = (float)p.jet_width;
    p.jet_amp_f = (float)p.jet_amp;
    p.jet_radius_f = (float)p.jet_radius;
    return p;
}

// Batched clouds: the carrier arguments of each cloud at the window's start
// (and its largest support cleared for this window's records) ...
__device__ __forceinline__ void batch_carrier_args_of(const BatchDev& b, double dt, int k)
{
    b.ext_max[k] = 0u;
    const BatchCloud& c = b.clouds[k];
    const double t = __dmul_rn((double)*b.step, dt);
    reinterpret_cast<CarrierArgs*>(b.cargs)[k] = carrier_args(c.car, c.N, t);
}

__global__ void k_batch_carrier_args(BatchDev b, double dt)
{
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b.n_clouds) return;
    batch_carrier_args_of(b, dt, k);
}

// ... and every node of every cloud (single precision).
__device__ __forceinline__ void batch_carrier_node(const BatchDev& b, int64_t g)
{
    const int k = batch_find(b.node_pre, b.n_clouds, g);
    const BatchCloud& c = b.clouds[k];
    const CarrierArgs& p = reinterpret_cast<const CarrierArgs*>(b.cargs)[k];
    const int64_t r = g - b.node_pre[k];
    if (c.dim == 2) sample_node<float, 2>(p, c.nodes, r);
    else sample_node<float, 3>(p, c.nodes, r);
}

__global__ void __launch_bounds__(256) k_batch_carrier_sample(BatchDev b)
{
    pdl_entry();
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= b.nodes_total) return;
    batch_carrier_node(b, g);
}

}  // namespace

cudaError_t launch_carrier_sample(const fla_carrier_desc& c, const fla_mesh& m, double t, int dtype, void* nodes,
                                  cudaStream_t s)
{
    const CarrierArgs p = carrier_args(c, m.n, t);
    const int64_t nn = m.n + 1;
    const int64_t total = m.dim == 2 ? nn * nn : nn * nn * nn;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    if (dtype == FLA_F32X2) {
        const int S = node_stride(m.dim);
        float* tail = (float*)nodes + 2 * total * S;
        if (cudaMemsetAsync(tail, 0, kNodesX2TailBytes, s) != cudaSuccess) return cudaGetLastError();
        const unsigned vblocks = (unsigned)((total * (S / 4) + threads - 1) / threads);
        if (m.dim == 2) {
            launch_pdl(k_carrier_sample_x2<2>, dim3(blocks), dim3(threads), 0, s, p, (float*)nodes, total);
            launch_pdl(k_carrier_split_x2<2>, dim3(vblocks), dim3(threads), 0, s, (float*)nodes, total);
        } else {
            launch_pdl(k_carrier_sample_x2<3>, dim3(blocks), dim3(threads), 0, s, p, (float*)nodes, total);
            launch_pdl(k_carrier_split_x2<3>, dim3(vblocks), dim3(threads), 0, s, (float*)nodes, total);
        }
        return cudaGetLastError();
    }
    if (dtype == FLA_F32) {
        if (m.dim == 2) launch_pdl(k_carrier_sample<float, 2>, dim3(blocks), dim3(threads), 0, s, p, (float*)nodes, total);
        else launch_pdl(k_carrier_sample<float, 3>, dim3(blocks), dim3(threads), 0, s, p, (float*)nodes, total);
    } else {
        if (m.dim == 2) launch_pdl(k_carrier_sample<double, 2>, dim3(blocks), dim3(threads), 0, s, p, (double*)nodes, total);
        else launch_pdl(k_carrier_sample<double, 3>, dim3(blocks), dim3(threads), 0, s, p, (double*)nodes, total);
    }
    return cudaGetLastError();
}

size_t batch_carrier_args_bytes() { return sizeof(CarrierArgs); }

cudaError_t launch_batch_carrier(const BatchDev& b, double dt, cudaStream_t s)
{
    launch_pdl(k_batch_carrier_args, dim3((b.n_clouds + 63) / 64), dim3(64), 0, s, b, dt);
    if (b.nodes_total > 0)
        launch_pdl(k_batch_carrier_sample, dim3((unsigned)((b.nodes_total + 255) / 256)), dim3(256), 0, s, b);
    return cudaGetLastError();
}

}  // namespace fla

#ifdef FLA_WINDOW_PHASES
// Phases of the persistent window kernel (window.cuh).
#include "window.cuh"
namespace fla {

__device__ void window_carrier_args(const BatchDev& b, double dt)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < b.n_clouds; k += gridDim.x * blockDim.x)
        batch_carrier_args_of(b, dt, k);
}

__device__ void window_carrier_sample(const BatchDev& b)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < b.nodes_total;
         g += (int64_t)gridDim.x * blockDim.x)
        batch_carrier_node(b, g);
}

}  // namespace fla
#endif
