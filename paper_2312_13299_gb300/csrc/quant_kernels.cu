// quant_kernels.cu -- the quantisation step after the sort (Sec. 3.3
// "Quantization & Compression" of Morgenstern et al., arXiv 2312.13299):
// every attribute channel of the sorted grid is clipped to a range and
// rounded to the nearest of q equally spaced values, giving the integer
// planes that an image codec then stores.
//
//   t = (min(max(x, lo), hi) - lo) / (hi - lo),  code = rint(t * (q - 1))
//   (FP32, IEEE division, round half to even; hi == lo gives code 0)
//   dequantised value = lo + code * ((hi - lo) / (q - 1))
//
// One thread per element; channel parameters are a kernel argument.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "plas_host.h"

namespace plas {

constexpr int kQuantMaxC = 256;

struct QuantParams {
    float lo[kQuantMaxC];
    float hi[kQuantMaxC];
    float qm1[kQuantMaxC];  // q - 1
};

__global__ void quantize_kernel(const float* __restrict__ x, long long n, int C, QuantParams p,
                                uint16_t* __restrict__ codes) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const float lo = p.lo[c], hi = p.hi[c];
        int k = 0;
        if (hi > lo) {
            const float v = fminf(fmaxf(x[i], lo), hi);
            const float t = __fdiv_rn(__fsub_rn(v, lo), __fsub_rn(hi, lo));
            k = __float2int_rn(__fmul_rn(t, p.qm1[c]));
        }
        codes[i] = (uint16_t)k;
    }
}

__global__ void dequantize_kernel(const uint16_t* __restrict__ codes, long long n, int C,
                                  QuantParams p, float* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const float lo = p.lo[c], hi = p.hi[c];
        const float step = hi > lo ? __fdiv_rn(__fsub_rn(hi, lo), p.qm1[c]) : 0.0f;
        out[i] = __fadd_rn(lo, __fmul_rn((float)codes[i], step));
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
    const long long b = (n + 255) / 256;
    return (unsigned)std::min<long long>(std::max<long long>(b, 1), (long long)num_sms() * 16);
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
    quantize_kernel<<<quant_blocks(n), 256, 0, (cudaStream_t)stream>>>(x, n, C, p, codes);
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
    dequantize_kernel<<<quant_blocks(n), 256, 0, (cudaStream_t)stream>>>(codes, n, C, p, out);
    return check_launch("dequantize");
}
