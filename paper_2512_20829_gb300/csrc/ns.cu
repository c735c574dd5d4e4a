// Two-way coupling: the carrier flow that the droplets' sources act on.
//
// Eq. 1 (incompressible Navier-Stokes with the momentum source S_Mom) in
// vorticity-streamfunction form and Eq. 2 (vapour transport with the mass
// source S_Mass) on a periodic unit square of n x n cells, in double
// precision (the carrier is small next to the droplet path, and double keeps
// it at the oracle's rounding level):
//   omega at the nodes (i h, j h), h = 1/n, held as its Fourier coefficients;
//   psi from Lap_h psi = -omega (5-point Laplacian, diagonal in Fourier space);
//   u = U_x + D_y psi, v = U_y - D_x psi (central differences), U the mean
//   flow, which a periodic streamfunction cannot carry;
//   one step of dt: R = -(u D_x omega + v D_y omega) + curl S_Mom at the nodes,
//   omega <- (omega + dt R) / (1 - dt nu lambda) in Fourier space, the mean
//   vorticity kept zero, U <- U + dt mean(S_Mom);
//   vapour rho at the cell centres: rho <- rho + dt (-div_h F + D Lap_h rho +
//   S_Mass), F the first-order upwind fluxes with face velocities from psi at
//   each face's two corner nodes (divergence-free cell by cell).  Eq. 2's
//   diffusion term is read with its physical sign.
// The 2D FFTs are radix-2 transforms of the rows in shared memory (one CTA
// per row, twiddles from a table made once) with a tiled transpose between
// the passes; spectral arrays are kept transposed ([kx][ky]).
// Node values for the droplets: u, v and grad u at the (n+1)^2 mesh nodes
// (node n repeats node 0), grad u by central differences of the nodal velocity.
#include "fla_internal.cuh"

namespace fla {
namespace {

constexpr int kNsThreads = 256;

// Workspace layout (bytes), each array on a 256-byte boundary.
struct NsLayout {
    size_t omega_hat, a, b, c, psi, omega, u, v, chi, rho, rho2, twiddle, scal, partial, total;
};

inline size_t ns_up(size_t x) { return (x + 255) & ~(size_t)255; }

inline NsLayout ns_layout(int n)
{
    NsLayout L{};
    const size_t c = (size_t)n * n * sizeof(double2), r = (size_t)n * n * sizeof(double);
    size_t o = 0;
    L.omega_hat = o; o += ns_up(c);
    L.a = o; o += ns_up(c);
    L.b = o; o += ns_up(c);
    L.c = o; o += ns_up(c);
    L.psi = o; o += ns_up(r);
    L.omega = o; o += ns_up(r);
    L.u = o; o += ns_up(r);
    L.v = o; o += ns_up(r);
    L.chi = o; o += ns_up(r);
    L.rho = o; o += ns_up(r);
    L.rho2 = o; o += ns_up(r);
    L.twiddle = o; o += ns_up((size_t)(n / 2) * sizeof(double2));
    L.scal = o; o += 256;                                  // U[2], mean S[2], mean chi u[2]
    L.partial = o; o += ns_up((size_t)2 * kNsThreads * sizeof(double));
    L.total = o;
    return L;
}

struct NsArgs {
    int n, logn;
    double h, inv_h, nu, D, dt;
    double2* omega_hat;   // [kx][ky]
    double2* a;           // psi's Fourier coefficients between steps ([kx][ky])
    double2* b;           // FFT buffers
    double2* c;
    double* psi;          // nodes [j][i]
    double* omega;
    double* u;            // nodal velocity
    double* v;
    double* chi;          // penalisation mask over eta (body)
    int body, hold;
    double fx0, fx1, fsig; // fringe
    double* rho;          // cells [j][i]
    double* rho2;
    const double2* twiddle;   // exp(-2 pi i t / n), t < n/2
    double* scal;         // U[2], mean S[2], mean chi u[2]
    double* partial;
};

NsArgs ns_args(const fla_ns_cfg& cfg, void* ws)
{
    const NsLayout L = ns_layout(cfg.n);
    char* w = static_cast<char*>(ws);
    NsArgs a{};
    a.n = cfg.n;
    int lg = 0;
    while ((1 << lg) < cfg.n) ++lg;
    a.logn = lg;
    a.h = 1.0 / cfg.n;
    a.inv_h = (double)cfg.n;
    a.nu = cfg.nu;
    a.D = cfg.diff;
    a.dt = cfg.dt;
    a.omega_hat = reinterpret_cast<double2*>(w + L.omega_hat);
    a.a = reinterpret_cast<double2*>(w + L.a);
    a.b = reinterpret_cast<double2*>(w + L.b);
    a.c = reinterpret_cast<double2*>(w + L.c);
    a.psi = reinterpret_cast<double*>(w + L.psi);
    a.omega = reinterpret_cast<double*>(w + L.omega);
    a.u = reinterpret_cast<double*>(w + L.u);
    a.v = reinterpret_cast<double*>(w + L.v);
    a.chi = reinterpret_cast<double*>(w + L.chi);
    a.body = cfg.body != 0;
    a.hold = cfg.hold_mean_flow != 0;
    a.fx0 = cfg.fringe_x0;
    a.fx1 = cfg.fringe_x1;
    a.fsig = cfg.fringe_sigma;
    a.rho = reinterpret_cast<double*>(w + L.rho);
    a.rho2 = reinterpret_cast<double*>(w + L.rho2);
    a.twiddle = reinterpret_cast<const double2*>(w + L.twiddle);
    a.scal = reinterpret_cast<double*>(w + L.scal);
    a.partial = reinterpret_cast<double*>(w + L.partial);
    return a;
}

__device__ __forceinline__ int wrap(int i, int n) { return i & (n - 1); }   // n a power of two

// Twiddle table: exp(-2 pi i t / n) for t < n/2.
__global__ void k_ns_twiddle(double2* tw, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n / 2) return;
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_double2(c, s);
}

// One radix-2 transform per row (decimation in time: bit-reversed load, then
// log2 n stages of butterflies in shared memory; in may equal out, each CTA
// reading its whole row before it writes).  Forward: X_k = sum_m x_m
// e^(-2 pi i k m / n); inverse: the conjugate twiddles and a factor 1/n.
template <bool INV>
__global__ void __launch_bounds__(kNsThreads) k_fft_rows(const double2* in, double2* out,
                                                         const double2* __restrict__ tw, int n, int logn)
{
    extern __shared__ double2 s_row[];
    const double2* src = in + (size_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_row[__brev((unsigned)i) >> (32 - logn)] = src[i];
    __syncthreads();
    for (int m = 1, step = n >> 1; m < n; m <<= 1, step >>= 1) {   // butterflies of span m, twiddle stride n/(2m)
        for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
            const int k = j & (m - 1);
            const int i0 = ((j - k) << 1) + k, i1 = i0 + m;
            double2 w = tw[k * step];
            if (INV) w.y = -w.y;
            const double2 a = s_row[i0], b = s_row[i1];
            const double2 t = make_double2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
            s_row[i0] = make_double2(a.x + t.x, a.y + t.y);
            s_row[i1] = make_double2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
    const double sc = INV ? 1.0 / (double)n : 1.0;
    double2* dst = out + (size_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = make_double2(s_row[i].x * sc, s_row[i].y * sc);
}

// out[c][r] = in[r][c] through 32 x 32 shared-memory tiles.
__global__ void __launch_bounds__(kNsThreads) k_transpose(const double2* __restrict__ in, double2* __restrict__ out,
                                                          int n)
{
    __shared__ double2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int r = ty; r < 32; r += 8)
        if (by + r < n && bx + tx < n) tile[r][tx] = in[(size_t)(by + r) * n + bx + tx];
    __syncthreads();
    for (int r = ty; r < 32; r += 8)
        if (bx + r < n && by + tx < n) out[(size_t)(bx + r) * n + by + tx] = tile[tx][r];
}

// Eigenvalue of the periodic 5-point Laplacian for mode (kx, ky).
__device__ __forceinline__ double lap_eig(int kx, int ky, int n)
{
    double sx, sy, c;
    sincospi((double)kx / (double)n, &sx, &c);
    sincospi((double)ky / (double)n, &sy, &c);
    return -4.0 * (double)n * (double)n * (sx * sx + sy * sy);
}

// Per node: psi (the real part of the inverse transform) and omega = -Lap_h psi.
__global__ void __launch_bounds__(kNsThreads) k_ns_vort(NsArgs a, const double2* __restrict__ phys)
{
    const int n = a.n;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * n) return;
    const int i = (int)(k & (n - 1)), j = (int)(k >> a.logn);
    const double c = phys[k].x;
    const double s = phys[(int64_t)j * n + wrap(i + 1, n)].x + phys[(int64_t)j * n + wrap(i - 1, n)].x +
                     phys[(int64_t)wrap(j + 1, n) * n + i].x + phys[(int64_t)wrap(j - 1, n) * n + i].x;
    a.psi[k] = c;
    a.omega[k] = -(s - 4.0 * c) * (a.inv_h * a.inv_h);
    const double h2 = 0.5 * a.inv_h;
    a.u[k] = a.scal[0] + (phys[(int64_t)wrap(j + 1, n) * n + i].x - phys[(int64_t)wrap(j - 1, n) * n + i].x) * h2;
    a.v[k] = a.scal[1] - (phys[(int64_t)j * n + wrap(i + 1, n)].x - phys[(int64_t)j * n + wrap(i - 1, n)].x) * h2;
}

template <typename S>
__device__ __forceinline__ double src_at(const S* p, int64_t k) { return p ? (double)p[k] : 0.0; }

// Per node: R = -(u D_x omega + v D_y omega) + curl S_Mom (from the four
// cells around the node), as the real input of the forward transform.
template <typename S>
__global__ void __launch_bounds__(kNsThreads) k_ns_rhs(NsArgs a, const S* __restrict__ sx, const S* __restrict__ sy,
                                                      double2* __restrict__ out)
{
    const int n = a.n;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * n) return;
    const int i = (int)(k & (n - 1)), j = (int)(k >> a.logn);
    const int ip = wrap(i + 1, n), im = wrap(i - 1, n), jp = wrap(j + 1, n), jm = wrap(j - 1, n);
    const double h2 = 0.5 * a.inv_h;
    const double* W = a.omega;
    const double u = a.u[k], v = a.v[k];
    const double wx = (W[(int64_t)j * n + ip] - W[(int64_t)j * n + im]) * h2;
    const double wy = (W[(int64_t)jp * n + i] - W[(int64_t)jm * n + i]) * h2;
    double curl = 0.0;
    if (sx) {
        const double syr = src_at(sy, (int64_t)j * n + i) + src_at(sy, (int64_t)jm * n + i);
        const double syl = src_at(sy, (int64_t)j * n + im) + src_at(sy, (int64_t)jm * n + im);
        const double sxt = src_at(sx, (int64_t)j * n + i) + src_at(sx, (int64_t)j * n + im);
        const double sxb = src_at(sx, (int64_t)jm * n + i) + src_at(sx, (int64_t)jm * n + im);
        curl = (syr - syl) * h2 - (sxt - sxb) * h2;
    }
    double r = -(u * wx + v * wy) + curl;
    if (a.body) {
        // curl of -chi u / eta (central differences of the nodal products), the fringe
        const int64_t kp = (int64_t)j * n + ip, km = (int64_t)j * n + im;
        const int64_t kt = (int64_t)jp * n + i, kb = (int64_t)jm * n + i;
        const double dcv = (a.chi[kp] * a.v[kp] - a.chi[km] * a.v[km]) * h2;
        const double dcu = (a.chi[kt] * a.u[kt] - a.chi[kb] * a.u[kb]) * h2;
        r += -(dcv - dcu);
        const double x = (double)i * a.h;
        if (a.fsig > 0.0 && a.fx1 > a.fx0 && x >= a.fx0 && x <= a.fx1) {
            const double sn = sin(M_PI * (x - a.fx0) / (a.fx1 - a.fx0));
            r -= a.fsig * sn * sn * W[k];
        }
    }
    out[k] = make_double2(r, 0.0);
}

// Per cell: the vapour step (upwind fluxes through divergence-free faces,
// diffusion, mass source) into rho2.
template <typename S>
__global__ void __launch_bounds__(kNsThreads) k_ns_vapour(NsArgs a, const S* __restrict__ sm)
{
    const int n = a.n;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * n) return;
    const int i = (int)(k & (n - 1)), j = (int)(k >> a.logn);
    const int ip = wrap(i + 1, n), im = wrap(i - 1, n), jp = wrap(j + 1, n), jm = wrap(j - 1, n);
    const double* P = a.psi;
    const double* r = a.rho;
    // faces: x at i (cells i-1 | i) and i+1, corners (i, j), (i, j+1); y at j and j+1
    const double ux0 = a.scal[0] + (P[(int64_t)jp * n + i] - P[(int64_t)j * n + i]) * a.inv_h;
    const double ux1 = a.scal[0] + (P[(int64_t)jp * n + ip] - P[(int64_t)j * n + ip]) * a.inv_h;
    const double vy0 = a.scal[1] - (P[(int64_t)j * n + ip] - P[(int64_t)j * n + i]) * a.inv_h;
    const double vy1 = a.scal[1] - (P[(int64_t)jp * n + ip] - P[(int64_t)jp * n + i]) * a.inv_h;
    const double rc = r[k];
    const double rl = r[(int64_t)j * n + im], rr = r[(int64_t)j * n + ip];
    const double rb = r[(int64_t)jm * n + i], rt = r[(int64_t)jp * n + i];
    const double fx0 = ux0 > 0.0 ? ux0 * rl : ux0 * rc;
    const double fx1 = ux1 > 0.0 ? ux1 * rc : ux1 * rr;
    const double fy0 = vy0 > 0.0 ? vy0 * rb : vy0 * rc;
    const double fy1 = vy1 > 0.0 ? vy1 * rc : vy1 * rt;
    const double div = (fx1 - fx0 + fy1 - fy0) * a.inv_h;
    const double lap = (rl + rr + rb + rt - 4.0 * rc) * (a.inv_h * a.inv_h);
    a.rho2[k] = rc + a.dt * (-div + a.D * lap + src_at(sm, k));
}

// Per mode ([kx][ky]): with R^ in spec (or without), omega^ <- (omega^ + dt R^)
// / (1 - dt nu lambda), the mean mode zero; psi^ = -omega^/lambda into spec.
// Also the step's last bookkeeping: rho <- rho2, U <- U + dt mean(S_Mom).
__global__ void __launch_bounds__(kNsThreads) k_ns_spectral(NsArgs a, double2* __restrict__ spec, int update)
{
    const int n = a.n;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k == 0 && update) {
        if (!a.body) {
            a.scal[0] += a.dt * a.scal[2];
            a.scal[1] += a.dt * a.scal[3];
        } else if (!a.hold) {   // the mean of the penalisation force decelerates the flow
            a.scal[0] += a.dt * (a.scal[2] - a.scal[4]);
            a.scal[1] += a.dt * (a.scal[3] - a.scal[5]);
        }
    }
    if (k >= (int64_t)n * n) return;
    const int kx = (int)(k >> a.logn), ky = (int)(k & (n - 1));
    const double lam = lap_eig(kx, ky, n);
    double2 w = a.omega_hat[k];
    if (update) {
        const double2 r = spec[k];
        const double den = 1.0 - a.dt * a.nu * lam;
        w = make_double2((w.x + a.dt * r.x) / den, (w.y + a.dt * r.y) / den);
        a.rho[k] = a.rho2[k];
    }
    if (k == 0) w = make_double2(0.0, 0.0);
    a.omega_hat[k] = w;
    spec[k] = k == 0 ? make_double2(0.0, 0.0) : make_double2(-w.x / lam, -w.y / lam);
}

// mean(S_Mom) over the cells, one CTA, a fixed order (deterministic).
template <typename S>
__global__ void __launch_bounds__(kNsThreads) k_ns_mean(NsArgs a, const S* __restrict__ sx, const S* __restrict__ sy)
{
    __shared__ double s_x[kNsThreads], s_y[kNsThreads];
    const int64_t nc = (int64_t)a.n * a.n;
    double px = 0.0, py = 0.0;
    for (int64_t c = threadIdx.x; c < nc; c += kNsThreads) {
        px += src_at(sx, c);
        py += src_at(sy, c);
    }
    s_x[threadIdx.x] = px;
    s_y[threadIdx.x] = py;
    __syncthreads();
    for (int w = kNsThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_x[threadIdx.x] += s_x[threadIdx.x + w];
            s_y[threadIdx.x] += s_y[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.scal[2] = s_x[0] / (double)nc;
        a.scal[3] = s_y[0] / (double)nc;
    }
}

// u, v and grad u at the (n+1)^2 mesh nodes (node n repeats node 0) in the
// analytic carriers' layout: (u, v, du/dx, du/dy, dv/dx, dv/dy, 0, 0).
template <typename T>
__global__ void __launch_bounds__(kNsThreads) k_ns_nodes(NsArgs a, T* __restrict__ nodes)
{
    const int n = a.n, nn = n + 1;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)nn * nn) return;
    const int i = wrap((int)(k % nn), n), j = wrap((int)(k / nn), n);
    const double* P = a.psi;
    const double h2 = 0.5 * a.inv_h;
    auto psi = [&](int ii, int jj) { return P[(int64_t)wrap(jj, n) * n + wrap(ii, n)]; };
    auto uu = [&](int ii, int jj) { return a.scal[0] + (psi(ii, jj + 1) - psi(ii, jj - 1)) * h2; };
    auto vv = [&](int ii, int jj) { return a.scal[1] - (psi(ii + 1, jj) - psi(ii - 1, jj)) * h2; };
    T out[8];
    out[0] = (T)uu(i, j);
    out[1] = (T)vv(i, j);
    out[2] = (T)((uu(i + 1, j) - uu(i - 1, j)) * h2);
    out[3] = (T)((uu(i, j + 1) - uu(i, j - 1)) * h2);
    out[4] = (T)((vv(i + 1, j) - vv(i - 1, j)) * h2);
    out[5] = (T)((vv(i, j + 1) - vv(i, j - 1)) * h2);
    out[6] = out[7] = (T)0;
#pragma unroll
    for (int q = 0; q < 8; ++q) nodes[k * 8 + q] = out[q];
}

// State from a nodal vorticity: its values as the real input of the forward
// transform; U from the arguments; rho copied or zero.
__global__ void __launch_bounds__(kNsThreads) k_ns_load(NsArgs a, const double* __restrict__ omega,
                                                        const double* __restrict__ rho, double ux, double uy)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k == 0) {
        a.scal[0] = ux;
        a.scal[1] = uy;
        a.scal[2] = a.scal[3] = 0.0;
    }
    if (k >= (int64_t)a.n * a.n) return;
    a.b[k] = make_double2(omega[k], 0.0);
    a.rho[k] = rho ? rho[k] : 0.0;
}

unsigned ns_blocks(int64_t count) { return (unsigned)((count + kNsThreads - 1) / kNsThreads); }

// 2D transform of in ([j][i] forward, [kx][ky] inverse) into out
// ([kx][ky] forward, [j][i] inverse): rows, transpose, rows (in place) through
// tmp; in is left as it was when it differs from tmp and out.
cudaError_t fft2(const NsArgs& a, const double2* in, double2* tmp, double2* out, bool inverse, cudaStream_t s)
{
    const int n = a.n;
    const size_t smem = (size_t)n * sizeof(double2);
    const dim3 tg((n + 31) / 32, (n + 31) / 32);
    if (inverse) k_fft_rows<true><<<n, kNsThreads, smem, s>>>(in, tmp, a.twiddle, n, a.logn);
    else k_fft_rows<false><<<n, kNsThreads, smem, s>>>(in, tmp, a.twiddle, n, a.logn);
    k_transpose<<<tg, kNsThreads, 0, s>>>(tmp, out, n);
    if (inverse) k_fft_rows<true><<<n, kNsThreads, smem, s>>>(out, out, a.twiddle, n, a.logn);
    else k_fft_rows<false><<<n, kNsThreads, smem, s>>>(out, out, a.twiddle, n, a.logn);
    return cudaGetLastError();
}

// The penalisation mask over eta at the nodes: (1 - tanh((r - R) n))/2 / eta.
__global__ void __launch_bounds__(kNsThreads) k_ns_mask(NsArgs a, double xc, double yc, double R, double eta)
{
    const int n = a.n;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * n) return;
    const int i = (int)(k & (n - 1)), j = (int)(k >> a.logn);
    const double r = hypot((double)i * a.h - xc, (double)j * a.h - yc);
    a.chi[k] = 0.5 * (1.0 - tanh((r - R) * (double)n)) / eta;
}

// mean(chi u), mean(chi v) over the nodes into scal[4], scal[5]: one CTA, a
// fixed order (deterministic).
__global__ void __launch_bounds__(kNsThreads) k_ns_body_mean(NsArgs a)
{
    __shared__ double s_x[kNsThreads], s_y[kNsThreads];
    const int64_t nc = (int64_t)a.n * a.n;
    double px = 0.0, py = 0.0;
    for (int64_t c = threadIdx.x; c < nc; c += kNsThreads) {
        px += a.chi[c] * a.u[c];
        py += a.chi[c] * a.v[c];
    }
    s_x[threadIdx.x] = px;
    s_y[threadIdx.x] = py;
    __syncthreads();
    for (int w = kNsThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_x[threadIdx.x] += s_x[threadIdx.x + w];
            s_y[threadIdx.x] += s_y[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.scal[4] = s_x[0] / (double)nc;
        a.scal[5] = s_y[0] / (double)nc;
    }
}

}  // namespace
}  // namespace fla

// ------------------------------------------------------------------ C ABI
using namespace fla;

namespace {

bool ns_cfg_ok(const fla_ns_cfg* c)
{
    if (!c || c->n < 8 || c->n > 1024 || (c->n & (c->n - 1)) != 0) return false;
    if (!(c->nu >= 0.0) || !isfinite(c->nu) || !(c->diff >= 0.0) || !isfinite(c->diff)) return false;
    if (!(c->dt > 0.0) || !isfinite(c->dt)) return false;
    if (!(c->diff * c->dt * (double)c->n * (double)c->n <= 0.25)) return false;   // explicit diffusion stays stable
    if (c->body) {
        const double vals[7] = {c->body_xc, c->body_yc, c->body_r, c->body_eta, c->fringe_x0, c->fringe_x1,
                                c->fringe_sigma};
        for (double x : vals)
            if (!isfinite(x)) return false;
        if (!(c->body_r > 0.0) || !(c->body_eta > 0.0) || c->dt > c->body_eta) return false;   // explicit penalisation
        if (c->fringe_sigma < 0.0 || c->fringe_sigma * c->dt > 1.0) return false;
        if (c->fringe_sigma > 0.0 && !(c->fringe_x1 > c->fringe_x0)) return false;
    }
    return true;
}

bool ws_ok(const fla_ns_cfg* c, const void* ws, size_t bytes)
{
    return ws && ((uintptr_t)ws % 256) == 0 && bytes >= ns_layout(c->n).total;
}

int ns_status(cudaError_t e) { return e == cudaSuccess ? FLA_OK : FLA_ERR_CUDA; }

// psi (and omega = -Lap_h psi) at the nodes from psi's coefficients in a.a.
cudaError_t ns_physical(const NsArgs& a, cudaStream_t s)
{
    const cudaError_t e = fft2(a, a.a, a.c, a.b, true, s);
    if (e != cudaSuccess) return e;
    k_ns_vort<<<ns_blocks((int64_t)a.n * a.n), kNsThreads, 0, s>>>(a, a.b);
    return cudaGetLastError();
}

template <typename S>
cudaError_t ns_steps(const NsArgs& a, const S* sm, const S* sx, const S* sy, int nsub, cudaStream_t s)
{
    const int64_t nc = (int64_t)a.n * a.n;
    k_ns_mean<S><<<1, kNsThreads, 0, s>>>(a, sx, sy);
    for (int q = 0; q < nsub; ++q) {
        cudaError_t e = ns_physical(a, s);
        if (e != cudaSuccess) return e;
        if (a.body && !a.hold) k_ns_body_mean<<<1, kNsThreads, 0, s>>>(a);
        k_ns_rhs<S><<<ns_blocks(nc), kNsThreads, 0, s>>>(a, sx, sy, a.c);
        k_ns_vapour<S><<<ns_blocks(nc), kNsThreads, 0, s>>>(a, sm);
        e = fft2(a, a.c, a.b, a.a, false, s);
        if (e != cudaSuccess) return e;
        k_ns_spectral<<<ns_blocks(nc), kNsThreads, 0, s>>>(a, a.a, 1);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" size_t fla_ns_workspace_size(const fla_ns_cfg* cfg)
{
    return ns_cfg_ok(cfg) ? ns_layout(cfg->n).total : 0;
}

extern "C" int fla_ns_init(fla_ctx* ctx, const fla_ns_cfg* cfg, const double* omega_dev, const double* mean_u,
                           const double* rho_dev, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    if (!ctx || !ns_cfg_ok(cfg) || !omega_dev || !mean_u || !isfinite(mean_u[0]) || !isfinite(mean_u[1]))
        return FLA_ERR_ARG;
    if (!ws_ok(cfg, ws, ws_bytes)) return FLA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const NsArgs a = ns_args(*cfg, ws);
    const int64_t nc = (int64_t)a.n * a.n;
    k_ns_twiddle<<<(unsigned)((a.n / 2 + 255) / 256), 256, 0, s>>>(const_cast<double2*>(a.twiddle), a.n);
    k_ns_load<<<ns_blocks(nc), kNsThreads, 0, s>>>(a, omega_dev, rho_dev, mean_u[0], mean_u[1]);
    if (a.body) k_ns_mask<<<ns_blocks(nc), kNsThreads, 0, s>>>(a, cfg->body_xc, cfg->body_yc, cfg->body_r, cfg->body_eta);
    cudaError_t e = fft2(a, a.b, a.c, a.omega_hat, false, s);
    if (e != cudaSuccess) return FLA_ERR_CUDA;
    k_ns_spectral<<<ns_blocks(nc), kNsThreads, 0, s>>>(a, a.a, 0);
    return ns_status(cudaGetLastError());
}

extern "C" int fla_ns_step(fla_ctx* ctx, const fla_ns_cfg* cfg, const void* s_mass_dev, const void* s_mom_dev,
                           int32_t src_dtype, int32_t nsub, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    if (!ctx || !ns_cfg_ok(cfg) || nsub < 0) return FLA_ERR_ARG;
    if ((s_mass_dev || s_mom_dev) && src_dtype != FLA_F32 && src_dtype != FLA_F64) return FLA_ERR_ARG;
    if (!ws_ok(cfg, ws, ws_bytes)) return FLA_ERR_WORKSPACE;
    if (nsub == 0) return FLA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const NsArgs a = ns_args(*cfg, ws);
    const int64_t nc = (int64_t)a.n * a.n;
    if (src_dtype == FLA_F64) {
        const double* sx = (const double*)s_mom_dev;
        return ns_status(ns_steps<double>(a, (const double*)s_mass_dev, sx, sx ? sx + nc : nullptr, nsub, s));
    }
    const float* sx = (const float*)s_mom_dev;
    return ns_status(ns_steps<float>(a, (const float*)s_mass_dev, sx, sx ? sx + nc : nullptr, nsub, s));
}

extern "C" int fla_ns_nodes(fla_ctx* ctx, const fla_ns_cfg* cfg, int32_t dtype, void* nodes_dev, void* ws,
                            size_t ws_bytes, fla_stream_t stream)
{
    if (!ctx || !ns_cfg_ok(cfg) || !nodes_dev || ((uintptr_t)nodes_dev % 16) != 0) return FLA_ERR_ARG;
    if (dtype != FLA_F32 && dtype != FLA_F64) return FLA_ERR_UNSUPPORTED;
    if (!ws_ok(cfg, ws, ws_bytes)) return FLA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const NsArgs a = ns_args(*cfg, ws);
    if (ns_physical(a, s) != cudaSuccess) return FLA_ERR_CUDA;
    const int64_t nodes = (int64_t)(a.n + 1) * (a.n + 1);
    if (dtype == FLA_F32) k_ns_nodes<float><<<ns_blocks(nodes), kNsThreads, 0, s>>>(a, (float*)nodes_dev);
    else k_ns_nodes<double><<<ns_blocks(nodes), kNsThreads, 0, s>>>(a, (double*)nodes_dev);
    return ns_status(cudaGetLastError());
}

extern "C" int fla_ns_fields(fla_ctx* ctx, const fla_ns_cfg* cfg, double* omega_dev, double* psi_dev,
                             double* rho_dev, double* mean_u, void* ws, size_t ws_bytes, fla_stream_t stream)
{
    if (!ctx || !ns_cfg_ok(cfg)) return FLA_ERR_ARG;
    if (!ws_ok(cfg, ws, ws_bytes)) return FLA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const NsArgs a = ns_args(*cfg, ws);
    const size_t bytes = (size_t)a.n * a.n * sizeof(double);
    if (ns_physical(a, s) != cudaSuccess) return FLA_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (omega_dev) e = cudaMemcpyAsync(omega_dev, a.omega, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && psi_dev) e = cudaMemcpyAsync(psi_dev, a.psi, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && rho_dev) e = cudaMemcpyAsync(rho_dev, a.rho, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mean_u) {
        e = cudaMemcpyAsync(mean_u, a.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return ns_status(e);
}

extern "C" int fla_ns_body_force(fla_ctx* ctx, const fla_ns_cfg* cfg, double* force, void* ws, size_t ws_bytes,
                                 fla_stream_t stream)
{
    if (!ctx || !ns_cfg_ok(cfg) || !cfg->body || !force) return FLA_ERR_ARG;
    if (!ws_ok(cfg, ws, ws_bytes)) return FLA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const NsArgs a = ns_args(*cfg, ws);
    if (ns_physical(a, s) != cudaSuccess) return FLA_ERR_CUDA;
    k_ns_body_mean<<<1, kNsThreads, 0, s>>>(a);
    cudaError_t e = cudaMemcpyAsync(force, a.scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return ns_status(e);
}
