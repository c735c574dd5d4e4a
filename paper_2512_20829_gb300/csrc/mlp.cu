// Learned bandwidth correction: parameter packing and the standalone forward
// (the records kernel fuses the same forward; see mlp_tc.cuh).
#include "mlp_tc.cuh"

namespace fla {
namespace {

// One thread per byte pair / float of the packed image.
__global__ void k_mlp_pack(const float* __restrict__ P, unsigned char* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // BF16 operand images: W1 (64 x 16, K zero-padded from 6), W2, W3 (64 x 64)
    if (t < kMlpH * 16) {
        const int n = t / 16, k = t % 16;
        const float w = k < kMlpIn ? P[kOffW1 + n * kMlpIn + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(out + kPkW1 + cm_offset(n, k, 16)) = __float2bfloat16_rn(w);
        return;
    }
    int u = t - kMlpH * 16;
    if (u < 2 * kMlpH * kMlpH) {
        const int layer = u / (kMlpH * kMlpH);
        const int e = u % (kMlpH * kMlpH);
        const int n = e / kMlpH, k = e % kMlpH;
        const float w = P[(layer == 0 ? kOffW2 : kOffW3) + n * kMlpH + k];
        *reinterpret_cast<__nv_bfloat16*>(out + (layer == 0 ? kPkW2 : kPkW3) + cm_offset(n, k, kMlpH)) =
            __float2bfloat16_rn(w);
        return;
    }
    u -= 2 * kMlpH * kMlpH;
    if (u < 3 * kMlpH) {   // biases stay FP32
        const int layer = u / kMlpH, k = u % kMlpH;
        const int src = layer == 0 ? kOffB1 : (layer == 1 ? kOffB2 : kOffB3);
        reinterpret_cast<float*>(out + kPkB1)[layer * kMlpH + k] = P[src + k];
        return;
    }
    u -= 3 * kMlpH;
    if (u < kMlpH) {   // last layer on the CUDA cores: BF16-rounded weights held as FP32
        reinterpret_cast<float*>(out + kPkW4)[u] = __bfloat162float(__float2bfloat16_rn(P[kOffW4 + u]));
        return;
    }
    u -= kMlpH;
    if (u < 4) reinterpret_cast<float*>(out + kPkB4)[u] = u == 0 ? P[kOffB4] : 0.0f;
}

// c = g(f) for n feature rows (row-major n x 6), 128 rows per CTA.
__global__ void __launch_bounds__(kMlpRows) k_mlp_forward(const unsigned char* __restrict__ packed,
                                                          const float* __restrict__ F, int64_t n,
                                                          float* __restrict__ out, DevStatus* st)
{
    extern __shared__ __align__(128) unsigned char smem[];
    MlpCta m = mlp_cta_layout(smem);
    mlp_cta_begin(m, packed);
    const int64_t i = blockIdx.x * (int64_t)kMlpRows + threadIdx.x;
    float f[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) f[k] = i < n ? F[i * kMlpIn + k] : 0.0f;
    bool ok = true;
    const float c = mlp_cta_forward(m, f, &ok);
    if (i < n) out[i] = c;
    if (!ok && threadIdx.x == 0) atomicOr(&st->flags, kFlagMlpTimeout);
    mlp_cta_end(m);
}

}  // namespace

cudaError_t launch_mlp_pack(const float* params, void* packed, cudaStream_t s)
{
    const int total = kMlpH * 16 + 2 * kMlpH * kMlpH + 4 * kMlpH + 4;
    k_mlp_pack<<<(total + 255) / 256, 256, 0, s>>>(params, (unsigned char*)packed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* packed, const float* feats, int64_t n, float* out, DevStatus* st,
                               cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + kMlpRows - 1) / kMlpRows);
    k_mlp_forward<<<blocks, kMlpRows, kMlpSmemBytes, s>>>((const unsigned char*)packed, feats, n, out, st);
    return cudaGetLastError();
}

}  // namespace fla
