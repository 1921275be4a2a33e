// sort_kernels.cu -- sm_103a kernels of the PLAS grid sort (Sec. 3.1 of
// Morgenstern et al., arXiv 2312.13299).
//
// Floating-point contract (shared with the CPU oracle by specification, not by
// code): every multiply-add is an explicit __fmaf_rn, every other operation an
// explicit round-to-nearest intrinsic, sums run in ascending tap / channel
// order, and the only reduction that feeds a decision (the mean L2 distance of
// the schedule) is an exact integer sum.  The library is built with
// -fmad=false so the compiler cannot contract anything on its own.
#include <algorithm>
#include <cstdio>

#include "plas_kernels.h"

namespace plas {

static inline unsigned ceil_div_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ============================================================================
// preparation: exact per-channel min/max, normalisation + weights, placement
// (Sec. 3.1 "Organizing Gaussians into a 2D Grid"; random init, Sec. 3.1)
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

void launch_pack(const float* x, int N, int D, const Weights& w, int normalize,
                 DevState* st, int mode, const int32_t* perm_init, uint64_t seed,
                 float* G, cudaStream_t s) {
    if (N <= 0) return;
    const uint32_t h = feistel_half_bits((uint32_t)N);
    pack_kernel<<<ceil_div_u(N, 256), 256, 0, s>>>(x, N, D, grid_stride(D), w, normalize, st,
                                                    mode, perm_init, seed, h, G);
}

// ============================================================================
// blur geometry: border renormalisation (in-range tap mass, ascending j)
// ============================================================================
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
    for (int j = jlo; j <= jhi; ++j) n = __fadd_rn(n, taps[rp + j]);
    out[pos] = n;
}

void launch_norms(const LevelDesc* lv_dev, int nlev, int H, int W, float* table,
                  cudaStream_t s) {
    const long long total = (long long)nlev * (W + H);
    if (total <= 0) return;
    norms_kernel<<<ceil_div_u(total, 256), 256, 0, s>>>(lv_dev, nlev, H, W, table);
}

// ============================================================================
// target, pass along x.  One CTA per (row, channel chunk); warp w owns channel
// d0 + w and every lane X consecutive outputs.  The row sits in shared memory
// planar per channel with one padding float after every X floats, which makes
// the stride-X accesses of a warp bank-conflict free.  Each output is the
// ascending-tap fmaf chain over the zero-padded row (a zero tap or a zero
// sample leaves the chain bit-for-bit unchanged), divided by the in-range tap
// mass.
// ============================================================================
template <int X>
__device__ __forceinline__ int swz(int t) { return t + t / X; }

template <int X>
__global__ void __launch_bounds__(1024) blur_rows_kernel(
    const float* __restrict__ G, int gs, int W, int D, float* __restrict__ H1,
    const DevState* __restrict__ st, int level, int r, int rp, int ntp,
    const float* __restrict__ taps, const float* __restrict__ norm, int dc) {
    if (state_idle(st, level)) return;
    extern __shared__ __align__(16) float smem[];
    const int y = blockIdx.x;
    const int d0 = blockIdx.y * dc;
    const int dcnt = min(dc, D - d0);
    const int Wr = (W + X - 1) / X * X;
    const int Ls = Wr + ntp + X;
    const int P = swz<X>(Ls) + 1;
    const int ntp4 = (ntp + 3) & ~3;
    float* tp = smem;                    // ntp taps (16-byte aligned)
    float* s = smem + ntp4;              // dcnt rows of P floats
    float* stage = s + (size_t)dc * P;   // (32 * X) cells x dcnt
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int t = tid; t < ntp; t += nt) tp[t] = taps[t];
    const float* grow = G + (size_t)y * W * gs + d0;
    for (int e = tid; e < Ls * dcnt; e += nt) {
        const int t = e / dcnt, d = e - t * dcnt;
        const int x = t - rp;
        const float v = (x >= 0 && x < W) ? grow[(size_t)x * gs + d] : 0.0f;
        s[d * P + swz<X>(t)] = v;
    }
    __syncthreads();

    const int lane = tid & 31, w = tid >> 5;
    const float* srow = s + w * P;
    float* hrow = H1 + (size_t)y * W * D;
    for (int cb = 0; cb < Wr; cb += 32 * X) {
        const int x0 = cb + lane * X;
        if (w < dcnt && x0 < Wr) {
            // warp-uniform trimmed step range: steps where some output of the
            // warp meets a non-zero tap and an in-range sample
            const int wend = min(cb + 32 * X, W);
            int jlo = max(rp - r, rp - (wend - 1));
            int jhi = min(rp + r, rp + W - 1 - cb);
            jlo = max(0, jlo / X * X);
            const int jend = min(ntp, (jhi + X) / X * X);
            float acc[X], win[X];
#pragma unroll
            for (int i = 0; i < X; ++i) acc[i] = 0.0f;
#pragma unroll
            for (int u = 0; u < X; ++u) win[u] = srow[swz<X>(x0 + jlo + u)];
            for (int jb = jlo; jb < jend; jb += X) {
                const int nb = swz<X>(x0 + jb + X);
                const float4 ka = *reinterpret_cast<const float4*>(tp + jb);
                const float4 kb = *reinterpret_cast<const float4*>(tp + jb + 4);
                const float kk[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
#pragma unroll
                for (int u = 0; u < X; ++u) {
#pragma unroll
                    for (int i = 0; i < X; ++i) acc[i] = __fmaf_rn(kk[u], win[(u + i) % X], acc[i]);
                    win[u] = srow[nb + u];
                }
            }
#pragma unroll
            for (int i = 0; i < X; ++i) {
                const int x = x0 + i;
                if (x < W) stage[(lane * X + i) * dcnt + w] = __fdiv_rn(acc[i], norm[x]);
            }
        }
        __syncthreads();
        const int ncell = min(32 * X, W - cb);
        if (dcnt == D) {
            float* dst = hrow + (size_t)cb * D;
            for (int e = tid; e < ncell * D; e += nt) dst[e] = stage[e];
        } else {
            for (int e = tid; e < ncell * dcnt; e += nt) {
                const int c = e / dcnt, d = e - c * dcnt;
                hrow[(size_t)(cb + c) * D + d0 + d] = stage[e];
            }
        }
        __syncthreads();
    }
}

RowPlan plan_rows(int W, int D, int ntpx) {
    const int X = kFirX;
    const int Wr = (W + X - 1) / X * X;
    const int Ls = Wr + ntpx + X;
    const int P = (Ls + Ls / X) + 1;
    const int ntp4 = (ntpx + 3) & ~3;
    const size_t budget = 227 * 1024;
    int dc = D < 32 ? D : 32;
    while (dc > 1) {
        const size_t bytes = sizeof(float) * ((size_t)ntp4 + (size_t)dc * P + (size_t)32 * X * dc);
        if (bytes <= budget) break;
        dc = (dc + 1) / 2;
    }
    RowPlan p;
    p.dc = dc;
    p.threads = 32 * dc;
    p.smem = sizeof(float) * ((size_t)ntp4 + (size_t)dc * P + (size_t)32 * X * dc);
    return p;
}

template <int X>
__global__ void blur_cols_kernel(const float* __restrict__ H1, int H, int W, int D, int ts,
                                 float* __restrict__ T, const DevState* __restrict__ st,
                                 int level, int r, int rp, int ntp,
                                 const float* __restrict__ taps, const float* __restrict__ norm,
                                 int TY);

// Opt every large-shared-memory kernel in to the full 227 KB, once per device.
static void smem_opt_in() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    const int max_smem = 227 * 1024;
    cudaFuncSetAttribute(blur_rows_kernel<kFirX>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    cudaFuncSetAttribute(blur_cols_kernel<kFirX>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    done[dev] = true;
}

void launch_blur_rows(const float* G, int gs, int H, int W, int D, float* H1,
                      const DevState* st, int level, const LevelDesc& lv, const float* table,
                      const RowPlan& plan, cudaStream_t s) {
    smem_opt_in();
    dim3 grid(H, (D + plan.dc - 1) / plan.dc);
    blur_rows_kernel<kFirX><<<grid, plan.threads, plan.smem, s>>>(
        G, gs, W, D, H1, st, level, lv.rx, lv.rpx, lv.ntpx, table + lv.off_tx, table + lv.off_nx,
        plan.dc);
}

// ============================================================================
// target, pass along y.  H1 is a [H][W*D] matrix; a CTA owns 32 consecutive
// columns (lane = column) and TY output rows (warp q = rows qX..qX+X-1).  The
// input rows stream through a 512-row ring in shared memory ([row][lane], so a
// warp reads one 128-byte row) in chunks of 64 tap steps: cp.async fetches the
// next chunk's rows while the current chunk is computed, so shared memory does
// not grow with the radius.  Out-of-grid rows are zero-filled by the copy.
// ============================================================================
constexpr int kColRing = 512;  // ring rows (power of two)
constexpr int kColChunk = 64;  // tap steps per chunk

__device__ __forceinline__ void cp_async_f32(float* sdst, const float* gsrc, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int X>
__global__ void __launch_bounds__(1024) blur_cols_kernel(
    const float* __restrict__ H1, int H, int W, int D, int ts, float* __restrict__ T,
    const DevState* __restrict__ st, int level, int r, int rp, int ntp,
    const float* __restrict__ taps, const float* __restrict__ norm, int TY) {
    if (state_idle(st, level)) return;
    extern __shared__ __align__(16) float ring[];
    const int Wc = W * D;
    const int c0 = blockIdx.x * 32;
    const int y0 = blockIdx.y * TY;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = c0 + lane;
    const bool cok = c < Wc;
    const float* gcol = H1 + (cok ? c : 0);

    // CTA-uniform step range: non-zero taps that reach an in-range row
    int jlo = max(rp - r, rp - y0 - TY + 1);
    const int jhi = min(rp + r, rp - y0 + H - 1);
    jlo = max(0, jlo / X * X);
    const int jend = min(ntp, (jhi + X) / X * X);

    const int span = TY + X;  // rows read beyond the last step of a chunk
    auto fetch = [&](int t) {
        const int yy = y0 - rp + t;
        const bool ok = cok && yy >= 0 && yy < H;
        cp_async_f32(ring + (t & (kColRing - 1)) * 32 + lane, ok ? gcol + (size_t)yy * Wc : gcol,
                     ok);
    };
    int loaded_end = min(jlo + kColChunk, jend) + span;
    for (int t = jlo + q; t < loaded_end; t += nw) fetch(t);
    cp_async_wait_all();
    __syncthreads();

    float acc[X], win[X];
#pragma unroll
    for (int i = 0; i < X; ++i) acc[i] = 0.0f;
    const int rbase = q * X;
#pragma unroll
    for (int u = 0; u < X; ++u) win[u] = ring[((rbase + jlo + u) & (kColRing - 1)) * 32 + lane];

    for (int jc = jlo; jc < jend; jc += kColChunk) {
        const int cend = min(jc + kColChunk, jend);
        // the ring holds >= 2*chunk + TY + X rows, so the next chunk's rows
        // never alias a row that the current chunk still reads
        const int next_end = min(cend + kColChunk, jend) + span;
        for (int t = loaded_end + q; t < next_end; t += nw) fetch(t);
        loaded_end = max(loaded_end, next_end);
        for (int jb = jc; jb < cend; jb += X) {
            const int nb = (rbase + jb + X) & (kColRing - 1);
            const float4 ka = __ldg(reinterpret_cast<const float4*>(taps + jb));
            const float4 kb = __ldg(reinterpret_cast<const float4*>(taps + jb + 4));
            const float kk[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
#pragma unroll
            for (int u = 0; u < X; ++u) {
#pragma unroll
                for (int i = 0; i < X; ++i) acc[i] = __fmaf_rn(kk[u], win[(u + i) % X], acc[i]);
                win[u] = ring[(nb + u) * 32 + lane];
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    if (cok) {
        const int x = c / D, d = c - x * D;
#pragma unroll
        for (int i = 0; i < X; ++i) {
            const int y = y0 + rbase + i;
            if (y < H) T[((size_t)y * W + x) * ts + d] = __fdiv_rn(acc[i], norm[y]);
        }
    }
}

ColPlan plan_cols(int H) {
    int ty = 256;
    while (ty > kFirX && ty / 2 >= H) ty /= 2;
    ColPlan p;
    p.ty = ty;
    p.threads = 32 * ty / kFirX;
    if (p.threads < 32) p.threads = 32;
    p.smem = sizeof(float) * (size_t)32 * kColRing;
    return p;
}

void launch_blur_cols(const float* H1, int H, int W, int D, int ts, float* T,
                      const DevState* st, int level, const LevelDesc& lv, const float* table,
                      const ColPlan& plan, cudaStream_t s) {
    smem_opt_in();
    dim3 grid(ceil_div_u((long long)W * D, 32), ceil_div_u(H, plan.ty));
    blur_cols_kernel<kFirX><<<grid, plan.threads, plan.smem, s>>>(
        H1, H, W, D, ts, T, st, level, lv.ry, lv.rpy, lv.ntpy, table + lv.off_ty,
        table + lv.off_ny, plan.ty);
}

// ============================================================================
// grouping permutation of the block cells (Sec. 3.1, "Blockwise Linear
// Assignment"): pi[m] for m < beta^2, fresh every iteration, shared by all
// blocks.
// ============================================================================
__global__ void group_table_kernel(uint64_t seed, const DevState* __restrict__ st, int level,
                                   uint32_t n, uint32_t h, uint32_t* __restrict__ pi) {
    if (state_idle(st, level)) return;
    const uint64_t it = (uint64_t)st->it;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
        pi[m] = keyed_permute(m, n, h, seed, kTagGroup, it);
}

void launch_group_table(uint64_t seed, const DevState* st, int level, int beta, uint32_t* pi,
                        int num_sms, cudaStream_t s) {
    const uint32_t n = (uint32_t)beta * (uint32_t)beta;
    const uint32_t h = feistel_half_bits(n);
    int blocks = (int)std::min<long long>(ceil_div_u(n, 256), (long long)num_sms * 8);
    group_table_kernel<<<blocks, 256, 0, s>>>(seed, st, level, n, h, pi);
}

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

// ============================================================================
// assignment (Sec. 3.1 "Blockwise Linear Assignment", Fig. "swapping_pixels"):
// a quad of lanes per group of four cells.  Lane i loads the feature row of
// cell p_i and the four target rows, forms row i of the 4x4 cost matrix
// C[i][j] = sum_d (G[p_i]_d - T[p_j]_d)^2, scores the six permutations whose
// first entry is i (lexicographic positions 6i..6i+5), and the quad agrees on
// the first strict minimum.  Lane i then writes its row to p_sigma(i).  The
// distance of every cell to the target after the swap is added to an exact
// fixed-point sum; the last CTA to finish runs the schedule step (Sec. 3.1).
// ============================================================================
template <int D>
struct Row {
    static constexpr int GS = (D + 1 + 3) & ~3;
    static constexpr int TS = (D + 3) & ~3;
};

template <int N4>
__device__ __forceinline__ void load_row4(const float* __restrict__ p, float* v) {
#pragma unroll
    for (int k = 0; k < N4; ++k) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p) + k);
        v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
    }
}

// The working grid is written by the same kernel (other cells), so it is read
// with ordinary coherent loads, not the read-only path.
template <int N4>
__device__ __forceinline__ void load_row4_rw(const float* p, float* v) {
#pragma unroll
    for (int k = 0; k < N4; ++k) {
        const float4 a = reinterpret_cast<const float4*>(p)[k];
        v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
    }
}

template <int D>
__device__ __forceinline__ float sqdist(const float* g, const float* t) {
    float acc = 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float delta = __fsub_rn(g[d], t[d]);
        acc = __fmaf_rn(delta, delta, acc);
    }
    return acc;
}

__device__ __forceinline__ unsigned long long fixed_point(float e, double scale) {
    return (unsigned long long)__double2ll_rn(__dmul_rn((double)e, scale));
}

// The 24 permutations of four positions in lexicographic order, generated at
// compile time (Fig. "swapping_pixels": brute force over all 24).
struct Perm24 {
    int p[24][4];
};
__host__ __device__ constexpr Perm24 make_perm24() {
    Perm24 t{};
    int n = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d)
                    if (a != b && a != c && a != d && b != c && b != d && c != d) {
                        t.p[n][0] = a; t.p[n][1] = b; t.p[n][2] = c; t.p[n][3] = d;
                        ++n;
                    }
    return t;
}

__device__ __forceinline__ float pick4(const float (&v)[4], int j) {
    return j == 0 ? v[0] : (j == 1 ? v[1] : (j == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ int pick4i(const int (&v)[4], int j) {
    return j == 0 ? v[0] : (j == 1 ? v[1] : (j == 2 ? v[2] : v[3]));
}

__device__ void schedule_step(DevState* st, long long N, int nby, int nbx, int ngroups,
                              int nlevels, double tol, long long* trace_S, int* trace_level,
                              long long trace_cap) {
    const unsigned long long S = atomicAdd(&st->S, 0ull);
    const double denom = ldexp((double)N, st->scale_exp);
    const double d = __ddiv_rn(__ull2double_rn(S), denom);
    const long long it = st->it;
    if (trace_S && it < trace_cap) trace_S[it] = (long long)S;
    if (trace_level && it < trace_cap) trace_level[it] = st->level;
    const bool improved =
        !st->has_prev ||
        (d < st->d_prev && __dsub_rn(st->d_prev, d) >= __dmul_rn(tol, st->d_prev));
    if (improved) {
        st->stall = 0;
        st->d_prev = d;
        st->has_prev = 1;
    } else if (st->stall == 0) {
        st->stall = 1;
        st->epoch += 1;
        st->redraws += 1;
        st->d_prev = d;
        st->has_prev = 1;
    } else {
        st->level += 1;
        st->stall = 0;
        st->epoch += 1;
        st->has_prev = 0;
        st->d_prev = 0.0;
    }
    st->d_last = d;
    st->it = it + 1;
    st->grouped += (long long)nby * nbx * ngroups * 4;
    if (st->level >= nlevels) st->done = 1;
    st->S = 0ull;
    st->arrivals = 0u;
    __threadfence();
}

template <int D>
__global__ void __launch_bounds__(256) assign_kernel(AssignArgs a) {
    using R = Row<D>;
    constexpr int GS = R::GS, TS = R::TS;
    __shared__ int s_idle, s_dy, s_dx;
    __shared__ unsigned long long s_part[8];
    DevState* st = a.st;
    if (threadIdx.x == 0) {
        const int idle = state_idle(st, a.level);
        s_idle = idle;
        if (!idle) {
            int dy, dx;
            block_shift(a.seed, st->epoch, a.beta, a.H, a.W, &dy, &dx);
            s_dy = dy;
            s_dx = dx;
        }
    }
    __syncthreads();
    if (s_idle) return;
    const int dy = s_dy, dx = s_dx, beta = a.beta, H = a.H, W = a.W;
    const int nby = (H - dy) / beta, nbx = (W - dx) / beta;
    const int ngroups = a.ngroups;
    const long long ngt = (long long)nby * nbx * ngroups;
    const double scale = ldexp(1.0, st->scale_exp);
    float* __restrict__ G = a.G;
    const float* __restrict__ T = a.T;
    unsigned long long part = 0ull;

    const int lane = threadIdx.x & 31, qi = lane & 3, qbase = lane & ~3;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // ---- groups: 8 per warp ----
    for (long long base = gwarp * 8; base < ngt; base += nwarps * 8) {
        const long long task0 = base + (lane >> 2);
        const bool active = task0 < ngt;
        const long long task = active ? task0 : 0;
        const long long blk = task / ngroups;
        const int g = (int)(task - blk * ngroups);
        const int by = (int)(blk / nbx), bx = (int)(blk - (long long)by * nbx);
        const int oy = dy + by * beta, ox = dx + bx * beta;
        const uint4 l4 = __ldg(reinterpret_cast<const uint4*>(a.pi) + g);
        const uint32_t ls[4] = {l4.x, l4.y, l4.z, l4.w};
        int pos[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ly = (int)(ls[k] / (uint32_t)beta);
            const int lx = (int)(ls[k] - (uint32_t)ly * (uint32_t)beta);
            pos[k] = (oy + ly) * W + (ox + lx);
        }
        float grow[GS];
        load_row4_rw<GS / 4>(G + (size_t)pick4i(pos, qi) * GS, grow);
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float trow[TS];
            load_row4<TS / 4>(T + (size_t)pos[j] * TS, trow);
            c[j] = sqdist<D>(grow, trow);
        }
        // all-gather the cost matrix inside the quad; every lane then scores
        // all 24 permutations (identical result in the four lanes)
        float C[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) C[i][j] = __shfl_sync(0xFFFFFFFFu, c[j], qbase | i);
        constexpr Perm24 kPerm24 = make_perm24();
        float best = 0.0f;
        int bidx = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            const float cost = __fadd_rn(
                __fadd_rn(__fadd_rn(C[0][kPerm24.p[k][0]], C[1][kPerm24.p[k][1]]), C[2][kPerm24.p[k][2]]),
                C[3][kPerm24.p[k][3]]);
            if (k == 0 || cost < best) {
                best = cost;
                bidx = k;
            }
        }
        int sg[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int v = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) v = (bidx == k) ? kPerm24.p[k][i] : v;
            sg[i] = v;
        }
        const int my_dst = pick4i(sg, qi);
        if (active) {
            float4* dst = reinterpret_cast<float4*>(G + (size_t)pick4i(pos, my_dst) * GS);
#pragma unroll
            for (int k = 0; k < GS / 4; ++k)
                dst[k] = make_float4(grow[4 * k], grow[4 * k + 1], grow[4 * k + 2], grow[4 * k + 3]);
            part += fixed_point(__fsqrt_rn(pick4(c, my_dst)), scale);
        }
    }

    // ---- cells outside the full blocks ----
    const int cy0 = dy, cy1 = dy + nby * beta, cx0 = dx, cx1 = dx + nbx * beta;
    const long long N = (long long)H * W;
    const long long gthread = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    for (long long p = gthread; p < N; p += nthreads) {
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        if (y >= cy0 && y < cy1 && x >= cx0 && x < cx1) continue;
        float grow[GS], trow[TS];
        load_row4_rw<GS / 4>(G + (size_t)p * GS, grow);
        load_row4<TS / 4>(T + (size_t)p * TS, trow);
        part += fixed_point(__fsqrt_rn(sqdist<D>(grow, trow)), scale);
    }
    // ---- leftover cells of each block (beta^2 mod 4 of them) ----
    const int nleft = beta * beta - 4 * ngroups;
    const long long nl = (long long)nby * nbx * nleft;
    for (long long e = gthread; e < nl; e += nthreads) {
        const long long blk = e / nleft;
        const int m = 4 * ngroups + (int)(e - blk * nleft);
        const int by = (int)(blk / nbx), bx = (int)(blk - (long long)by * nbx);
        const uint32_t l = a.pi[m];
        const int ly = (int)(l / (uint32_t)beta), lx = (int)(l - (uint32_t)ly * (uint32_t)beta);
        const long long p = (long long)(dy + by * beta + ly) * W + (dx + bx * beta + lx);
        float grow[GS], trow[TS];
        load_row4_rw<GS / 4>(G + (size_t)p * GS, grow);
        load_row4<TS / 4>(T + (size_t)p * TS, trow);
        part += fixed_point(__fsqrt_rn(sqdist<D>(grow, trow)), scale);
    }

    // ---- exact reduction, last CTA runs the schedule ----
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
    if (lane == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_part[w];
        atomicAdd(&st->S, tot);
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->arrivals, 1u);
        if (ticket == gridDim.x - 1) {
            __threadfence();
            schedule_step(st, N, nby, nbx, ngroups, a.nlevels, a.tol, a.trace_S, a.trace_level,
                          a.trace_cap);
        }
    }
}

int assign_grid_size(int H, int W, int beta, int num_sms) {
    const long long N = (long long)H * W;
    long long need = (N / 4 + 63) / 64;  // one quad per group, 64 groups per CTA
    const long long cap = (long long)num_sms * 8;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    (void)beta;
    return (int)need;
}

template <int D>
static void launch_assign_t(const AssignArgs& a, int grid, cudaStream_t s) {
    assign_kernel<D><<<grid, 256, 0, s>>>(a);
}

void launch_assign(const AssignArgs& a, int grid, cudaStream_t s) {
    switch (a.D) {
#define PLAS_CASE(d) \
    case d: launch_assign_t<d>(a, grid, s); break;
        PLAS_CASE(1) PLAS_CASE(2) PLAS_CASE(3) PLAS_CASE(4) PLAS_CASE(5) PLAS_CASE(6)
        PLAS_CASE(7) PLAS_CASE(8) PLAS_CASE(9) PLAS_CASE(10) PLAS_CASE(11) PLAS_CASE(12)
        PLAS_CASE(13) PLAS_CASE(14) PLAS_CASE(15) PLAS_CASE(16) PLAS_CASE(20) PLAS_CASE(24)
        PLAS_CASE(32) PLAS_CASE(48) PLAS_CASE(64)
#undef PLAS_CASE
        default: break;  // the API only admits the instantiated channel counts
    }
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

// dst[p, c] = src[perm[p], c]; consecutive threads write consecutive floats.
__global__ void gather_rows_kernel(const float* __restrict__ src, long long N, int C,
                                   const int32_t* __restrict__ perm, float* __restrict__ dst) {
    const long long total = N * C;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long p = o / C;
        const int c = (int)(o - p * C);
        const int q = __ldg(perm + p);
        dst[o] = (q >= 0 && q < N) ? __ldg(src + (size_t)q * C + c) : 0.0f;
    }
}

__global__ void gather_rows4_kernel(const float4* __restrict__ src, long long N, int C4,
                                    const int32_t* __restrict__ perm, float4* __restrict__ dst) {
    const long long total = N * C4;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long p = o / C4;
        const int c = (int)(o - p * C4);
        const int q = __ldg(perm + p);
        dst[o] = (q >= 0 && q < N) ? __ldg(src + (size_t)q * C4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

void launch_gather_rows(const float* src, long long N, int C, const int32_t* perm, float* dst,
                        cudaStream_t s) {
    if (N <= 0 || C <= 0) return;
    const bool vec = (C % 4 == 0) && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 16 == 0);
    const long long total = vec ? N * (C / 4) : N * C;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    if (vec)
        gather_rows4_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(src), N, C / 4,
                                                   perm, reinterpret_cast<float4*>(dst));
    else
        gather_rows_kernel<<<blocks, 256, 0, s>>>(src, N, C, perm, dst);
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

}  // namespace plas
