// prep_kernels.cu -- once-per-sort kernels of the PLAS grid sort (Sec. 3.1 of
// Morgenstern et al., arXiv 2312.13299): exact per-channel min/max,
// normalisation and weights, the keyed random initial placement, the border
// norms of the blur, and the outputs (permutation, carried-attribute gather,
// grid metrics).  Floating point uses explicit round-to-nearest intrinsics.
#include <algorithm>
#include <cstdio>

#include "plas_kernels.h"

namespace plas {

static inline unsigned ceil_div_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ============================================================================
// preparation (Sec. 3.1 "Organizing Gaussians into a 2D Grid"; random init)
// ============================================================================
__global__ void state_reset_kernel(DevState* st) {
    const int t = threadIdx.x;
    if (t < kMaxD) {
        st->lo_bits[t] = 0xFFFFFFFFu;
        st->hi_bits[t] = 0u;
    }
    if (t == 0) {
        st->S = 0ull;
        st->arrivals = 0u;
        st->nonfinite = 0;
        st->bad_index = 0;
        st->grouped = 0;
    }
}

void launch_state_reset(DevState* st, cudaStream_t s) { state_reset_kernel<<<1, 64, 0, s>>>(st); }

// Grid-stride with a stride that is a multiple of D, so every thread always
// sees the same channel and keeps one running min / max.
__global__ void minmax_kernel(const float* __restrict__ x, long long total, int D,
                              DevState* st) {
    __shared__ unsigned int slo[kMaxD], shi[kMaxD];
    __shared__ int sbad;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        slo[d] = 0xFFFFFFFFu;
        shi[d] = 0u;
    }
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long stride = (nthreads / D) * D;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt < stride) {
        unsigned int lo = 0xFFFFFFFFu, hi = 0u;
        bool bad = false;
        for (long long e = gt; e < total; e += stride) {
            const float v = x[e];
            bad |= !isfinite(v);
            const unsigned int u = float_to_ordered(__fadd_rn(v, 0.0f));  // -0 -> +0
            lo = min(lo, u);
            hi = max(hi, u);
        }
        const int d = (int)(gt % D);
        atomicMin(&slo[d], lo);
        atomicMax(&shi[d], hi);
        if (bad) sbad = 1;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        atomicMin(&st->lo_bits[d], slo[d]);
        atomicMax(&st->hi_bits[d], shi[d]);
    }
    if (threadIdx.x == 0 && sbad) st->nonfinite = 1;
}

void launch_minmax(const float* x, long long N, int D, DevState* st, int num_sms,
                   cudaStream_t s) {
    const long long total = N * D;
    int blocks = (int)std::min<long long>((total + 255) / 256, (long long)num_sms * 8);
    if (blocks < 1) blocks = 1;
    minmax_kernel<<<blocks, 256, 0, s>>>(x, total, D, st);
}

// Fixed-point exponent of the residual sum: largest k <= 32 with
// N * E * 2^k < 2^62, E = sqrt(sum_d (w_d * span_d)^2) bounding every
// grid-to-target distance (span_d = 1 after normalisation, else hi - lo).
__global__ void finalize_prep_kernel(DevState* st, long long N, int D, Weights w,
                                     int normalize) {
    if (threadIdx.x != 0) return;
    double e2 = 0.0;
    for (int d = 0; d < D; ++d) {
        double span = 1.0;
        if (!normalize) {
            span = N > 0 ? __dsub_rn((double)ordered_to_float(st->hi_bits[d]),
                                     (double)ordered_to_float(st->lo_bits[d]))
                         : 0.0;
        }
        const double sd = __dmul_rn((double)w.w[d], span);
        e2 = __dadd_rn(e2, __dmul_rn(sd, sd));
    }
    const double m = __dmul_rn((double)N, __dsqrt_rn(e2));
    int k = 32;
    while (k > 0 && ldexp(m, k) >= 4611686018427387904.0 /* 2^62 */) --k;
    st->scale_exp = k;
    // box target: fixed-point exponent s, the largest <= 40 with B 2^s <= 2^31
    // for B = max_d |w_d| (times max(|lo_d|, |hi_d|) without normalisation)
    double B = 0.0;
    for (int d = 0; d < D; ++d) {
        double b = fabs((double)w.w[d]);
        if (!normalize && N > 0)
            b = __dmul_rn(b, fmax(fabs((double)ordered_to_float(st->lo_bits[d])),
                                  fabs((double)ordered_to_float(st->hi_bits[d]))));
        B = fmax(B, b);
    }
    int s = 40;
    while (s > -60 && ldexp(B, s) > 2147483648.0 /* 2^31 */) --s;
    st->box_exp = s;
    if (st->nonfinite) {
        st->status = -5;  // PLAS_ERR_NONFINITE
        st->done = 1;
    }
}

void launch_finalize_prep(DevState* st, long long N, int D, const Weights& w, int normalize,
                          cudaStream_t s) {
    finalize_prep_kernel<<<1, 32, 0, s>>>(st, N, D, w, normalize);
}

// G[dst] = (w * (x[src] - lo) / (hi - lo), src, 0...).  A caller-supplied start
// permutation is bounds-checked: an entry outside [0, N) is not read; it marks
// the state invalid (the sort then stops and reports PLAS_ERR_INVALID_ARG).
__global__ void pack_kernel(const float* __restrict__ x, int N, int D, int gs, Weights w,
                            int normalize, DevState* __restrict__ st, int mode,
                            const int32_t* __restrict__ perm_init, uint64_t seed, uint32_t h,
                            float* __restrict__ G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int src = i, dst = i;
    if (mode == 1) dst = (int)keyed_permute((uint32_t)i, (uint32_t)N, h, seed, kTagInit, 0ull);
    if (mode == 2) {
        src = perm_init[i];
        if (src < 0 || src >= N) {
            st->bad_index = 1;
            st->status = -1;  // PLAS_ERR_INVALID_ARG
            st->done = 1;
            src = 0;
        }
    }
    float* g = G + (size_t)dst * gs;
    const float* xs = x + (size_t)src * D;
    for (int d = 0; d < D; ++d) {
        const float v = xs[d];
        float f;
        if (normalize) {
            const float lo = ordered_to_float(st->lo_bits[d]);
            const float hi = ordered_to_float(st->hi_bits[d]);
            f = (hi == lo) ? 0.0f
                           : __fmul_rn(w.w[d], __fdiv_rn(__fsub_rn(v, lo), __fsub_rn(hi, lo)));
        } else {
            f = __fmul_rn(w.w[d], v);
        }
        g[d] = f;
    }
    g[D] = __int_as_float(src);
    for (int d = D + 1; d < gs; ++d) g[d] = 0.0f;
}

void launch_pack(const float* x, int N, int D, const Weights& w, int normalize, DevState* st,
                 int mode, const int32_t* perm_init, uint64_t seed, float* G, cudaStream_t s) {
    if (N <= 0) return;
    const uint32_t h = feistel_half_bits((uint32_t)N);
    pack_kernel<<<ceil_div_u(N, 256), 256, 0, s>>>(x, N, D, grid_stride(D), w, normalize, st,
                                                    mode, perm_init, seed, h, G);
}

// Border renormalisation of the blur: in-range tap mass, ascending j, FP32.
// The level table holds every tap twice (k, k); the first copy is summed.
__global__ void norms_kernel(const LevelDesc* __restrict__ lv, int nlev, int H, int W,
                             float* __restrict__ table) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)W + H;
    if (gid >= per * nlev) return;
    const int L = (int)(gid / per);
    const int p = (int)(gid % per);
    const LevelDesc d = lv[L];
    int r, rp, len, pos;
    const float* taps;
    float* out;
    if (p < W) {
        r = d.rx; rp = d.rpx; len = W; pos = p;
        taps = table + d.off_tx; out = table + d.off_nx;
    } else {
        r = d.ry; rp = d.rpy; len = H; pos = p - W;
        taps = table + d.off_ty; out = table + d.off_ny;
    }
    const int jlo = max(-r, -pos), jhi = min(r, len - 1 - pos);
    float n = 0.0f;
    for (int j = jlo; j <= jhi; ++j) n = __fadd_rn(n, taps[2 * (rp + j)]);
    out[pos] = n;
    out[((len + 3) & ~3) + pos] = __frcp_rn(n);  // RN(1/n), for the correctly rounded division
}

void launch_norms(const LevelDesc* lv_dev, int nlev, int H, int W, float* table,
                  cudaStream_t s) {
    const long long total = (long long)nlev * (W + H);
    if (total <= 0) return;
    norms_kernel<<<ceil_div_u(total, 256), 256, 0, s>>>(lv_dev, nlev, H, W, table);
}

// ============================================================================
// standalone random sources (per-kernel parity of the grouping permutation and
// of Philox4x32-10)
// ============================================================================
__global__ void keyed_permutation_kernel(uint64_t seed, uint32_t tag, uint64_t counter,
                                         uint32_t n, uint32_t h, uint32_t* __restrict__ out) {
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
        out[m] = keyed_permute(m, n, h, seed, tag, counter);
}

void launch_keyed_permutation(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n,
                              uint32_t* out, int num_sms, cudaStream_t s) {
    const uint32_t h = feistel_half_bits(n);
    int blocks = (int)std::min<long long>(ceil_div_u(n, 256), (long long)num_sms * 8);
    keyed_permutation_kernel<<<blocks, 256, 0, s>>>(seed, tag, counter, n, h, out);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int n,
                              uint32_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = philox4x32_10(c, k0, k1);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

void launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out,
                   cudaStream_t s) {
    if (n <= 0) return;
    philox_kernel<<<ceil_div_u(n, 256), 256, 0, s>>>(ctr, k0, k1, n, out);
}

__global__ void fill_uniform_kernel(float* __restrict__ out, long long n, uint32_t k0,
                                    uint32_t k1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 o = philox4x32_10(make_uint4((uint32_t)i, 4u << 8, (uint32_t)(i >> 32), 0u), k0, k1);
    out[i] = (float)(o.x >> 8) * (1.0f / 16777216.0f);
}

void launch_fill_uniform(float* out, long long n, uint64_t seed, cudaStream_t s) {
    if (n <= 0) return;
    fill_uniform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, (uint32_t)seed,
                                                                    (uint32_t)(seed >> 32));
}

// ============================================================================
// outputs (Sec. 3: every attribute plane follows the one permutation)
// ============================================================================
__global__ void extract_perm_kernel(const float* __restrict__ G, int N, int gs, int D,
                                    int32_t* __restrict__ perm) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) perm[p] = __float_as_int(G[(size_t)p * gs + D]);
}

void launch_extract_perm(const float* G, int N, int D, int32_t* perm, cudaStream_t s) {
    if (N <= 0) return;
    extract_perm_kernel<<<ceil_div_u(N, 256), 256, 0, s>>>(G, N, grid_stride(D), D, perm);
}

// Bijection check of a permutation of [0, N) (the sort places every
// Gaussian on exactly one cell, Sec. 3.1).  Pass 1 marks each in-range value
// in 'seen' and, if it was marked already, in 'dup'; pass 2 takes the
// smallest position whose value is out of range or marked in 'dup'.  Both
// bitmaps hold ceil(N/32) words and start at zero; res[0] starts at INT_MAX.
// A value missing from perm implies an out-of-range or repeated value
// elsewhere, so res[0] == INT_MAX exactly when perm is a permutation.
__global__ void check_perm_mark_kernel(const int32_t* __restrict__ perm, int N, uint32_t* seen,
                                       uint32_t* dup) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int v = perm[p];
        if (v < 0 || v >= N) continue;
        const uint32_t bit = 1u << (v & 31);
        if (atomicOr(&seen[v >> 5], bit) & bit) atomicOr(&dup[v >> 5], bit);
    }
}

__global__ void check_perm_first_kernel(const int32_t* __restrict__ perm, int N,
                                        const uint32_t* __restrict__ dup, int* res) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int v = perm[p];
        const bool bad = v < 0 || v >= N || ((dup[v >> 5] >> (v & 31)) & 1u);
        if (bad) atomicMin(res, p);
    }
}

void launch_check_permutation(const int32_t* perm, int N, uint32_t* seen, uint32_t* dup, int* res,
                              int num_sms, cudaStream_t s) {
    if (N <= 0) return;
    const unsigned blocks = std::min<unsigned>(ceil_div_u(N, 256), (unsigned)num_sms * 8u);
    check_perm_mark_kernel<<<blocks, 256, 0, s>>>(perm, N, seen, dup);
    check_perm_first_kernel<<<blocks, 256, 0, s>>>(perm, N, dup, res);
}

// dst[p, c] = src[perm[p], c]; consecutive threads write consecutive floats.
__global__ void gather_rows_kernel(const float* __restrict__ src, long long N, long long Nsrc, int C,
                                   const int32_t* __restrict__ perm, float* __restrict__ dst) {
    const long long total = N * C;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long p = o / C;
        const int c = (int)(o - p * C);
        const int q = __ldg(perm + p);
        dst[o] = (q >= 0 && q < Nsrc) ? __ldg(src + (size_t)q * C + c) : 0.0f;
    }
}

__global__ void gather_rows4_kernel(const float4* __restrict__ src, long long N, long long Nsrc, int C4,
                                    const int32_t* __restrict__ perm, float4* __restrict__ dst) {
    const long long total = N * C4;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long p = o / C4;
        const int c = (int)(o - p * C4);
        const int q = __ldg(perm + p);
        dst[o] = (q >= 0 && q < Nsrc) ? __ldg(src + (size_t)q * C4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

void launch_gather_rows(const float* src, long long N, int C, const int32_t* perm, float* dst,
                        cudaStream_t s, long long Nsrc) {
    if (N <= 0 || C <= 0) return;
    if (Nsrc < 0) Nsrc = N;
    const bool vec = (C % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 16 == 0);
    const long long total = vec ? N * (C / 4) : N * C;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    if (vec)
        gather_rows4_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(src), N, Nsrc,
                                                   C / 4, perm, reinterpret_cast<float4*>(dst));
    else
        gather_rows_kernel<<<blocks, 256, 0, s>>>(src, N, Nsrc, C, perm, dst);
}

__global__ void copy_features_kernel(const float* __restrict__ T, long long N, int D, int ts,
                                     float* __restrict__ out) {
    const long long total = N * D;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long p = o / D;
        out[o] = T[p * ts + (o - p * D)];
    }
}

void launch_copy_features(const float* T, int N, int D, int ts, float* out, cudaStream_t s) {
    if (N <= 0) return;
    const long long total = (long long)N * D;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    copy_features_kernel<<<blocks, 256, 0, s>>>(T, N, D, ts, out);
}

// Grid quality: neighbour L2 and the moments of |diff| for VAD (FP64).
__global__ void neighbour_metrics_kernel(const float* __restrict__ g, int stride, int H, int W,
                                         int D, double scale, double* __restrict__ acc) {
    double s_l2 = 0.0, s1 = 0.0, s2 = 0.0;
    const long long N = (long long)H * W;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        const float* a = g + (size_t)p * stride;
        for (int dir = 0; dir < 2; ++dir) {
            const int y2 = y + (dir == 1), x2 = x + (dir == 0);
            if (y2 >= H || x2 >= W) continue;
            const float* b = g + ((size_t)y2 * W + x2) * stride;
            double q = 0.0;
            for (int d = 0; d < D; ++d) {
                const double diff = (double)a[d] - (double)b[d];
                q += diff * diff;
                const double ad = fabs(diff * scale);
                s1 += ad;
                s2 += ad * ad;
            }
            s_l2 += sqrt(q);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        s_l2 += __shfl_down_sync(0xFFFFFFFFu, s_l2, off);
        s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
        s2 += __shfl_down_sync(0xFFFFFFFFu, s2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, s_l2);
        atomicAdd(acc + 1, s1);
        atomicAdd(acc + 2, s2);
    }
}

void launch_neighbour_metrics(const float* g, int stride, int H, int W, int D, double scale,
                              double* acc, int num_sms, cudaStream_t s) {
    const long long N = (long long)H * W;
    if (N <= 0) return;
    const int blocks = (int)std::min<long long>((N + 255) / 256, (long long)num_sms * 8);
    neighbour_metrics_kernel<<<blocks, 256, 0, s>>>(g, stride, H, W, D, scale, acc);
}

// ---- checked runs: guard bands between workspace regions ---------------------
__global__ void fill_guards_kernel(Guards g) {
    for (int k = blockIdx.x; k < g.n; k += gridDim.x)
        for (int b = threadIdx.x; b < kGuardBytes; b += blockDim.x) g.at[k][b] = kGuardByte;
}

__global__ void check_guards_kernel(Guards g, unsigned int* bad) {
    for (int k = blockIdx.x; k < g.n; k += gridDim.x)
        for (int b = threadIdx.x; b < kGuardBytes; b += blockDim.x)
            if (g.at[k][b] != kGuardByte) atomicAdd(bad, 1u);
}

void launch_fill_guards(const Guards& g, cudaStream_t s) {
    if (g.n > 0) fill_guards_kernel<<<g.n, 256, 0, s>>>(g);
}

void launch_check_guards(const Guards& g, unsigned int* bad, cudaStream_t s) {
    if (g.n > 0) check_guards_kernel<<<g.n, 256, 0, s>>>(g, bad);
}

}  // namespace plas
