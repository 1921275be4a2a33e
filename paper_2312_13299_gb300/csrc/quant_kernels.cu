// quant_kernels.cu -- the quantisation step after the sort (Sec. 3.4
// "Quantization & Compression" of Morgenstern et al., arXiv 2312.13299):
// every attribute channel of the sorted grid is clipped to a range and
// rounded to the nearest of q equally spaced values, giving the integer
// planes that an image codec then stores.
//
//   t = (min(max(x, lo), hi) - lo) / (hi - lo),  code = rint(t * (q - 1))
//   (FP32, IEEE division, round half to even; hi == lo gives code 0)
//   dequantised value = lo + code * ((hi - lo) / (q - 1))
//
// The channel parameters are a kernel argument, staged into shared memory at
// the start of each CTA (lanes of a warp read different channels).  A thread
// handles 4 consecutive elements per step (16-byte loads when the input is
// aligned) and advances the channel index of its elements incrementally.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "plas_host.h"

namespace plas {

constexpr int kQuantMaxC = 256;
constexpr int kQuantThreads = 256;

struct QuantParams {
    float lo[kQuantMaxC];
    float hi[kQuantMaxC];
    float qm1[kQuantMaxC];  // q - 1
};

__device__ __forceinline__ uint16_t quant_one(float x, float lo, float hi, float qm1) {
    int k = 0;
    if (hi > lo) {
        const float v = fminf(fmaxf(x, lo), hi);
        const float t = __fdiv_rn(__fsub_rn(v, lo), __fsub_rn(hi, lo));
        k = __float2int_rn(__fmul_rn(t, qm1));
    }
    return (uint16_t)k;
}

// element i of the [N][C] grid is channel i mod C; element groups [4g, 4g+4)
__global__ void __launch_bounds__(kQuantThreads) quantize_kernel(const float* __restrict__ x, long long n,
                                                                 int C, QuantParams p,
                                                                 uint16_t* __restrict__ codes) {
    __shared__ float s_lo[kQuantMaxC], s_hi[kQuantMaxC], s_qm1[kQuantMaxC];
    for (int c = threadIdx.x; c < C; c += kQuantThreads) {
        s_lo[c] = p.lo[c];
        s_hi[c] = p.hi[c];
        s_qm1[c] = p.qm1[c];
    }
    __syncthreads();
    const long long groups = (n + 3) / 4;
    const long long g0 = (long long)blockIdx.x * kQuantThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kQuantThreads;
    const int cstep = (int)((4 * gstride) % C);
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(codes)) & 15) == 0;
    int c = (int)((4 * g0) % C);
    for (long long g = g0; g < groups; g += gstride) {
        const long long i = 4 * g;
        int cc[4];
        cc[0] = c;
#pragma unroll
        for (int k = 1; k < 4; ++k) cc[k] = cc[k - 1] + 1 == C ? 0 : cc[k - 1] + 1;
        if (vec && i + 4 <= n) {
            const float4 v = *reinterpret_cast<const float4*>(x + i);
            const float f[4] = {v.x, v.y, v.z, v.w};
            ushort4 o;
            uint16_t* op = reinterpret_cast<uint16_t*>(&o);
#pragma unroll
            for (int k = 0; k < 4; ++k) op[k] = quant_one(f[k], s_lo[cc[k]], s_hi[cc[k]], s_qm1[cc[k]]);
            *reinterpret_cast<ushort4*>(codes + i) = o;
        } else {
            for (int k = 0; k < 4 && i + k < n; ++k)
                codes[i + k] = quant_one(x[i + k], s_lo[cc[k]], s_hi[cc[k]], s_qm1[cc[k]]);
        }
        c += cstep;
        if (c >= C) c -= C;
    }
}

__global__ void __launch_bounds__(kQuantThreads) dequantize_kernel(const uint16_t* __restrict__ codes,
                                                                   long long n, int C, QuantParams p,
                                                                   float* __restrict__ out) {
    __shared__ float s_lo[kQuantMaxC], s_step[kQuantMaxC];
    for (int c = threadIdx.x; c < C; c += kQuantThreads) {
        const float lo = p.lo[c], hi = p.hi[c];
        s_lo[c] = lo;
        s_step[c] = hi > lo ? __fdiv_rn(__fsub_rn(hi, lo), p.qm1[c]) : 0.0f;
    }
    __syncthreads();
    const long long groups = (n + 3) / 4;
    const long long g0 = (long long)blockIdx.x * kQuantThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kQuantThreads;
    const int cstep = (int)((4 * gstride) % C);
    const bool vec = ((reinterpret_cast<uintptr_t>(codes) & 7) | (reinterpret_cast<uintptr_t>(out) & 15)) == 0;
    int c = (int)((4 * g0) % C);
    for (long long g = g0; g < groups; g += gstride) {
        const long long i = 4 * g;
        int cc[4];
        cc[0] = c;
#pragma unroll
        for (int k = 1; k < 4; ++k) cc[k] = cc[k - 1] + 1 == C ? 0 : cc[k - 1] + 1;
        if (vec && i + 4 <= n) {
            const ushort4 q = *reinterpret_cast<const ushort4*>(codes + i);
            const uint16_t qq[4] = {q.x, q.y, q.z, q.w};
            float r[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] = __fadd_rn(s_lo[cc[k]], __fmul_rn((float)qq[k], s_step[cc[k]]));
            *reinterpret_cast<float4*>(out + i) = make_float4(r[0], r[1], r[2], r[3]);
        } else {
            for (int k = 0; k < 4 && i + k < n; ++k)
                out[i + k] = __fadd_rn(s_lo[cc[k]], __fmul_rn((float)codes[i + k], s_step[cc[k]]));
        }
        c += cstep;
        if (c >= C) c -= C;
    }
}

static int make_params(int C, const float* lo, const float* hi, const int* q, QuantParams* p) {
    if (C < 1 || C > kQuantMaxC) return fail(PLAS_ERR_INVALID_ARG, "C must be 1..%d", kQuantMaxC);
    if (!lo || !hi || !q) return fail(PLAS_ERR_INVALID_ARG, "lo, hi and q are required");
    for (int c = 0; c < C; ++c) {
        if (!(lo[c] <= hi[c]) || !std::isfinite(lo[c]) || !std::isfinite(hi[c]))
            return fail(PLAS_ERR_INVALID_ARG, "channel %d: need finite lo <= hi", c);
        if (q[c] < 2 || q[c] > 65536) return fail(PLAS_ERR_INVALID_ARG, "channel %d: q must be 2..65536", c);
        p->lo[c] = lo[c];
        p->hi[c] = hi[c];
        p->qm1[c] = (float)(q[c] - 1);
    }
    return PLAS_OK;
}

static unsigned quant_blocks(long long n) {
    const long long b = ((n + 3) / 4 + kQuantThreads - 1) / kQuantThreads;
    return (unsigned)std::min<long long>(std::max<long long>(b, 1), (long long)num_sms() * 8);
}

}  // namespace plas

using namespace plas;

extern "C" int plas_quantize(const float* x, long long N, int C, const float* lo, const float* hi,
                             const int* q, uint16_t* codes, void* stream) {
    set_last_error("");
    if (N < 0) return fail(PLAS_ERR_INVALID_ARG, "N must be >= 0");
    QuantParams p;
    if (int e = make_params(C, lo, hi, q, &p)) return e;
    if (N == 0) return PLAS_OK;
    if (!x || !codes) return fail(PLAS_ERR_INVALID_ARG, "x and codes are required");
    const long long n = N * C;
    quantize_kernel<<<quant_blocks(n), kQuantThreads, 0, (cudaStream_t)stream>>>(x, n, C, p, codes);
    return check_launch("quantize");
}

extern "C" int plas_dequantize(const uint16_t* codes, long long N, int C, const float* lo,
                               const float* hi, const int* q, float* out, void* stream) {
    set_last_error("");
    if (N < 0) return fail(PLAS_ERR_INVALID_ARG, "N must be >= 0");
    QuantParams p;
    if (int e = make_params(C, lo, hi, q, &p)) return e;
    if (N == 0) return PLAS_OK;
    if (!codes || !out) return fail(PLAS_ERR_INVALID_ARG, "codes and out are required");
    const long long n = N * C;
    dequantize_kernel<<<quant_blocks(n), kQuantThreads, 0, (cudaStream_t)stream>>>(codes, n, C, p, out);
    return check_launch("dequantize");
}
