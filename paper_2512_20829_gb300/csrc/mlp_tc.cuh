// Learned bandwidth correction: a 6 -> 64 -> 64 -> 64 -> 1 SiLU network
// evaluated on the fifth-generation tensor cores (tcgen05), 128 droplets per
// CTA.  The paper has no counterpart; see fla.h (fla_mlp_*) for the contract.
//
// Per CTA (128 threads = 4 warps, thread t <-> droplet row t <-> TMEM lane t):
//   layer 1:  D[128 x 64]  = A0[128 x 16] . W1^T   (one MMA, K = 16; features 6, zero padded)
//   layer 2:  D            = A1[128 x 64] . W2^T   (four MMAs, K = 16 each)
//   layer 3:  D            = A2[128 x 64] . W3^T
//   layer 4:  c = W4 . silu(D + b3) + b4 on the CUDA cores, FP32
// A and B are BF16 in shared memory in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per 128-byte core matrix; the next 8 k at +128 B,
// the next 8 rows at +K/8 * 128 B); the FP32 accumulator lives in 64 TMEM
// columns.  Bias and SiLU are applied in FP32 on the way from TMEM to the next
// layer's BF16 operand.  One elected thread issues the MMAs and commits them
// to an mbarrier that the CTA waits on with a bounded spin.
#pragma once

#include <cuda_bf16.h>

#include "fla_internal.cuh"

namespace fla {

constexpr int kMlpIn = 6;
constexpr int kMlpH = 64;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + 2 * (kMlpH * kMlpH + kMlpH) + kMlpH + 1;   // 8833
// master parameter offsets (floats): W1[64][6], b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH * kMlpH;
constexpr int kOffW4 = kOffB3 + kMlpH;
constexpr int kOffB4 = kOffW4 + kMlpH;

// packed image (bytes): BF16 operand images of W1 (64 x 16), W2, W3 (64 x 64),
// then FP32 b1, b2, b3, W4 (BF16-rounded values), b4
constexpr int kPkW1 = 0;
constexpr int kPkW2 = kPkW1 + kMlpH * 16 * 2;
constexpr int kPkW3 = kPkW2 + kMlpH * kMlpH * 2;
constexpr int kPkB1 = kPkW3 + kMlpH * kMlpH * 2;
constexpr int kPkB2 = kPkB1 + kMlpH * 4;
constexpr int kPkB3 = kPkB2 + kMlpH * 4;
constexpr int kPkW4 = kPkB3 + kMlpH * 4;
constexpr int kPkB4 = kPkW4 + kMlpH * 4;
constexpr int kPkBytes = kPkB4 + 16;   // 19,472
static_assert(kPkBytes % 16 == 0, "packed image is copied in 16-byte pieces");

constexpr int kMlpRows = 128;                          // droplets per CTA
constexpr int kActBytes = kMlpRows * kMlpH * 2;        // 16 KB activation operand
constexpr int kMlpSmemBytes = kPkBytes + kActBytes + 64;

// Byte offset of element (row, k) in a K-major operand of K columns.
__host__ __device__ constexpr int cm_offset(int row, int k, int K)
{
    return (row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------------------
// PTX wrappers (sm_100 family)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: start, leading (K-direction)
// and stride (row-group) byte offsets, version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N x M.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait for the phase with the given parity; gives up after max_iter polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Warp-wide TMEM allocation of ncols columns; the address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// z sigma(z) with the fast exponential and reciprocal (a few ulp)
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Bounded waits: about a second at most before giving up with an error flag.
constexpr uint32_t kMbarPolls = 1u << 24;

// Shared state of one CTA's network evaluation.
struct MlpCta {
    unsigned char* img;     // packed image copy (kPkBytes, 16-byte aligned)
    unsigned char* act;     // activation operand (kActBytes, 16-byte aligned)
    uint64_t* bar;
    uint32_t* tmem_slot;
    uint32_t phase;         // completed phases of bar (each thread tracks the same count)
};

__device__ __forceinline__ MlpCta mlp_cta_layout(unsigned char* smem)
{
    MlpCta m;
    m.img = smem;
    m.act = smem + kPkBytes;
    m.bar = reinterpret_cast<uint64_t*>(smem + kPkBytes + kActBytes);
    m.tmem_slot = reinterpret_cast<uint32_t*>(smem + kPkBytes + kActBytes + 16);
    m.phase = 0;
    return m;
}

// Copy the packed image, set up the barrier and the 64 TMEM columns.  All 128 threads.
__device__ __forceinline__ void mlp_cta_begin(const MlpCta& m, const unsigned char* __restrict__ packed)
{
    const uint4* src = reinterpret_cast<const uint4*>(packed);
    uint4* dst = reinterpret_cast<uint4*>(m.img);
    for (int q = threadIdx.x; q < kPkBytes / 16; q += blockDim.x) dst[q] = __ldg(src + q);
    if (threadIdx.x == 0) {
        mbar_init(m.bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) tmem_alloc(m.tmem_slot, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void mlp_cta_end(const MlpCta& m)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(*m.tmem_slot, 64);
}

// Issue one layer (K = 16 * ksteps) into the TMEM accumulator and wait for it.
// Returns false if the wait gave up.
__device__ __forceinline__ bool mlp_layer(MlpCta& m, uint32_t w_off, int K)
{
    const uint32_t parity = m.phase & 1u;
    ++m.phase;
    fence_proxy_async_smem();     // generic-proxy writes of the operand -> async proxy
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(m.act), b0 = smem_u32(m.img + w_off);
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        constexpr uint32_t idesc = idesc_bf16_f32(kMlpRows, kMlpH);
        for (int s = 0; s < K / 16; ++s)
            tc_mma_bf16(*m.tmem_slot, smem_desc(a0 + 256u * s, 128u, sbo), smem_desc(b0 + 256u * s, 128u, sbo),
                        idesc, s > 0 ? 1u : 0u);
        tc_commit(m.bar);
    }
    const bool ok = mbar_wait(m.bar, parity, kMbarPolls);
    tc_fence_after();
    return ok;
}

// Bias + SiLU of this thread's accumulator row written as the next layer's
// BF16 operand row (K = 64); if last, the post-SiLU FP32 values go to out[64].
__device__ __forceinline__ void mlp_epilogue(const MlpCta& m, int bias_off, bool last, float* out)
{
    const int row = threadIdx.x;
    const uint32_t lane_base = *m.tmem_slot + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
    const float* bias = reinterpret_cast<const float*>(m.img + bias_off);
#pragma unroll
    for (int c0 = 0; c0 < kMlpH; c0 += 16) {
        float v[16];
        tmem_ld16(lane_base + (uint32_t)c0, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = silu_f(v[q] + bias[c0 + q]);
        if (last) {
#pragma unroll
            for (int q = 0; q < 16; ++q) out[c0 + q] = v[q];
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint4 u;
                u.x = pack_bf16x2(v[8 * h + 0], v[8 * h + 1]);
                u.y = pack_bf16x2(v[8 * h + 2], v[8 * h + 3]);
                u.z = pack_bf16x2(v[8 * h + 4], v[8 * h + 5]);
                u.w = pack_bf16x2(v[8 * h + 6], v[8 * h + 7]);
                *reinterpret_cast<uint4*>(m.act + cm_offset(row, c0 + 8 * h, kMlpH)) = u;
            }
        }
    }
}

// c = g(f) for this thread's row.  f: the 6 features (FP32).  Every thread of
// the 128-thread CTA calls it (rows without a droplet pass zeros).  Sets *ok
// false if a wait gave up (the result is then meaningless).
__device__ __forceinline__ float mlp_cta_forward(MlpCta& m, const float* f, bool* ok, float* a3_out = nullptr)
{
    const int row = threadIdx.x;
    {   // layer-1 operand: 16 BF16 per row (features then zeros)
        uint4 u0, u1;
        u0.x = pack_bf16x2(f[0], f[1]);
        u0.y = pack_bf16x2(f[2], f[3]);
        u0.z = pack_bf16x2(f[4], f[5]);
        u0.w = 0u;
        u1 = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(m.act + cm_offset(row, 0, 16)) = u0;
        *reinterpret_cast<uint4*>(m.act + cm_offset(row, 8, 16)) = u1;
    }
    bool good = mlp_layer(m, kPkW1, 16);
    float a3[kMlpH];
    mlp_epilogue(m, kPkB1, false, a3);
    good &= mlp_layer(m, kPkW2, kMlpH);
    mlp_epilogue(m, kPkB2, false, a3);
    good &= mlp_layer(m, kPkW3, kMlpH);
    mlp_epilogue(m, kPkB3, true, a3);
    const float* w4 = reinterpret_cast<const float*>(m.img + kPkW4);
    float c = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) c = fmaf(w4[k], a3[k], c);
    c += *reinterpret_cast<const float*>(m.img + kPkB4);
    if (a3_out) {
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) a3_out[k] = a3[k];
    }
    *ok = good;
    return c;
}

// The forward of mlp_cta_forward that also keeps, for the backward pass, this
// row's pre-activations z1, z2, z3 (FP32) and the BF16 activations a1, a2 (as
// FP32 values) in the given shared-memory rows (64 values each).
__device__ __forceinline__ float mlp_cta_forward_keep(MlpCta& m, const float* f, float* z1, float* z2, float* z3,
                                                      float* a1, float* a2, bool* ok)
{
    const int row = threadIdx.x;
    {
        uint4 u0;
        u0.x = pack_bf16x2(f[0], f[1]);
        u0.y = pack_bf16x2(f[2], f[3]);
        u0.z = pack_bf16x2(f[4], f[5]);
        u0.w = 0u;
        *reinterpret_cast<uint4*>(m.act + cm_offset(row, 0, 16)) = u0;
        *reinterpret_cast<uint4*>(m.act + cm_offset(row, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
    }
    const uint32_t lane_base = *m.tmem_slot + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
    bool good = true;
    float c = 0.0f;
    const float* w4 = reinterpret_cast<const float*>(m.img + kPkW4);
    for (int layer = 0; layer < 3; ++layer) {
        good &= mlp_layer(m, layer == 0 ? kPkW1 : (layer == 1 ? kPkW2 : kPkW3), layer == 0 ? 16 : kMlpH);
        const float* bias = reinterpret_cast<const float*>(m.img + (layer == 0 ? kPkB1 : (layer == 1 ? kPkB2 : kPkB3)));
        float* zr = layer == 0 ? z1 : (layer == 1 ? z2 : z3);
        float* ar = layer == 0 ? a1 : a2;
#pragma unroll 1
        for (int c0 = 0; c0 < kMlpH; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float z = v[q] + bias[c0 + q];
                zr[c0 + q] = z;
                v[q] = silu_f(z);
            }
            if (layer < 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint4 u;
                    u.x = pack_bf16x2(v[8 * h + 0], v[8 * h + 1]);
                    u.y = pack_bf16x2(v[8 * h + 2], v[8 * h + 3]);
                    u.z = pack_bf16x2(v[8 * h + 4], v[8 * h + 5]);
                    u.w = pack_bf16x2(v[8 * h + 6], v[8 * h + 7]);
                    *reinterpret_cast<uint4*>(m.act + cm_offset(row, c0 + 8 * h, kMlpH)) = u;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) ar[c0 + q] = __bfloat162float(__float2bfloat16_rn(v[q]));
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) c = fmaf(w4[c0 + q], v[q], c);
            }
        }
    }
    c += *reinterpret_cast<const float*>(m.img + kPkB4);
    *ok = good;
    return c;
}

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// BF16 weight (n, k) of a K-major operand image, as FP32.
__device__ __forceinline__ float img_weight(const unsigned char* img, int off, int n, int k, int K)
{
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(img + off + cm_offset(n, k, K)));
}

// Arguments of the training kernels (learn.cu).
struct LearnArgs {
    int dim, N;
    int kernel;                 // FLA_KERNEL_ISO or FLA_KERNEL_ANISO
    float hmin2;                // h_min^2 (J-scaled kernel)
    int64_t n_cells;
    const float* s_mass;        // deposit outputs of the learned forward
    const float* s_mom;
    const float* dsum;
    const uint32_t* cells;      // training cells (distinct), n_train
    int64_t n_train;
    const float* targets;       // n_train x (1 + dim)
    float* q;                   // per cell: H_0..H_dim, G/D (q_stride floats)
    int q_stride;
    float* scal;                // norm_k of the targets
    float* loss;                // += loss
    const uint32_t* bin_start;  // cell list of the deposit
    const void* rec;            // records in sorted order
    const float* aux;           // per sorted record: g(f), 1 if the bandwidth moves with it
    float* dldc;                // per sorted record: dL/dc
};

constexpr int kLearnRowPad = kMlpH + 1;   // padded FP32 rows of the backward's shared arrays
constexpr int kLearnSmemBytes =
    kMlpSmemBytes + (5 * kMlpRows * kLearnRowPad + kMlpRows * 8 + kMlpRows) * 4;

cudaError_t launch_learn_cells(const LearnArgs& a, cudaStream_t s);
cudaError_t launch_learn_dc(const LearnArgs& a, int64_t n, cudaStream_t s);
cudaError_t launch_grad_reduce(const float* partial, int n_parts, float* grad, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s);

cudaError_t launch_mlp_pack(const float* params, void* packed, cudaStream_t s);
cudaError_t launch_mlp_forward(const void* packed, const float* feats, int64_t n, float* out, DevStatus* st,
                               cudaStream_t s);

}  // namespace fla
