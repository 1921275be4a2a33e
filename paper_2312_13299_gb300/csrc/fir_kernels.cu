// fir_kernels.cu -- the low-pass target of the PLAS sort (Sec. 3.1 of
// Morgenstern et al., arXiv 2312.13299: the grid is low-pass filtered into an
// idealised target whose kernel shrinks with the radius), one separable pass
// per launch, over every grid of a sweep.
//
// A pass filters the columns of a logical R x NC matrix along its rows (the
// blur axis).  Pass 0 runs along y on the working grid (columns = (x, d);
// output written as [x][y][d]); pass 1 runs along x on that output (columns =
// (y, d); output = the target [y][x][d]).  The pass-0 launch also writes the
// iteration's grouping table (one launch fewer per iteration).
//
// The ring kernel: a CTA owns 128 columns and TY output rows (128 or 64, see
// FirTiling); small radii use fir_direct_kernel (no ring, 32 rows x 64
// columns per CTA).  Lane l handles the four
// columns c0+l, c0+32+l, c0+64+l, c0+96+l as two packed pairs, so each tap step
// is 16 fma.rn.f32x2 (two independent IEEE round-to-nearest FMAs each) fed by
// one 16-byte shared-memory load; warp q owns output rows 8q..8q+7 and keeps
// them in registers.  Input rows stream through a ring in shared memory
// ([row][lane][4 columns]) in chunks of tap steps: cp.async fetches
// the next chunk's rows and taps while the current one is computed, and
// out-of-grid rows are zero-filled by the copy.  Each output is the ascending-tap FMA chain
// over the zero-padded column: a zero tap or a zero sample leaves the chain
// bit-for-bit unchanged (the accumulator starts at +0 and never becomes -0),
// so padded and per-warp trimmed step ranges give exactly the in-range sum.
// It is then divided by the in-range tap mass (correctly rounded, as the
// IEEE division).
#include <algorithm>

#include "plas_kernels.h"

namespace plas {

static_assert(kFirCols == 128, "four columns per lane");

// Two tilings of the ring kernel (identical results): rows per CTA, ring
// rows, tap steps per chunk, CTAs per SM.  The large one keeps 16 warps per
// CTA busy at large radii; the medium one (2 CTAs per SM) overlaps one CTA's
// first fetch and epilogue with the other's taps at middle radii.  Small
// radii take fir_direct_kernel below (no ring).
template <int TY_, int RING_, int CH_, int MINB_>
struct FirTiling {
    static constexpr int TY = TY_, RING = RING_, CH = CH_, MINB = MINB_;
    static constexpr int THREADS = 32 * TY / kFirX;
    static_assert(RING >= 2 * CH + TY + kFirX, "ring must hold two chunks + span");
    static_assert(RING % kFirX == 0 && CH % kFirX == 0, "ring and chunk in whole steps of 8");
    // ring slot of input row t (t >= 0)
    __device__ static __forceinline__ int slot(int t) {
        return (RING & (RING - 1)) == 0 ? (t & (RING - 1)) : (t % RING);
    }
};
using FirLarge = FirTiling<128, 256, 56, 1>;
using FirMedium = FirTiling<64, 128, 24, 2>;

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// a / b correctly rounded, from y = RN(1/b): q = RN(a*y) is within one ulp of
// a/b, the remainder r = a - b*q is exact (one FMA), and RN(q + r*y) is the
// correctly rounded quotient (Markstein's theorem, IBM J. Res. Dev. 34(1),
// 1990) as long as nothing underflows or overflows.  Magnitudes outside
// [2^-60, 2^60] (and zero, NaN, Inf) take the IEEE division itself.
__device__ __forceinline__ float div_rn(float a, float b, float y) {
    const float m = fabsf(a);
    if (!(m >= 0x1p-60f && m <= 0x1p60f)) return __fdiv_rn(a, b);
    const float q = __fmul_rn(a, y);
    const float r = __fmaf_rn(-q, b, a);
    return __fmaf_rn(r, y, q);
}

// 4-byte copy to shared address sa + OFF (n = 4: copy, n = 0: zero-fill)
template <int OFF>
__device__ __forceinline__ void cp_async_f32_at(unsigned sa, const float* gsrc, int n) {
    asm volatile("cp.async.ca.shared.global [%0+%3], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n),
                 "n"(OFF)
                 : "memory");
}
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <class TL>
__global__ void __launch_bounds__(TL::THREADS, TL::MINB) fir_kernel(
    int pass, const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, int D, int gs,
    int ts) {
    constexpr int X = kFirX;
    constexpr int kFirTY = TL::TY, kFirChunk = TL::CH;
    constexpr int kFirThreads = TL::THREADS;
    constexpr int NW = kFirThreads / 32;
    const CtaRef cr = resolve_cta(map);
    const GridRef& gr = grids[cr.g];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];

    const float* in;
    long long in_row, in_cell;
    int R, NC, r, rp, ntp;
    const float* taps;
    if (pass == 0) {  // along y: G -> H1 ([x][y][d])
        in = gr.G; in_row = (long long)gr.W * gs; in_cell = gs;
        R = gr.H; NC = gr.W * D;
        r = lv.ry; rp = lv.rpy; ntp = lv.ntpy;
        taps = gr.table + lv.off_ty;
    } else {          // along x: H1 -> T ([y][x][d], cell stride ts)
        in = gr.H1; in_row = (long long)gr.H * D; in_cell = D;
        R = gr.W; NC = gr.H * D;
        r = lv.rx; rp = lv.rpx; ntp = lv.ntpx;
        taps = gr.table + lv.off_tx;
    }
    const int ncol = (NC + kFirCols - 1) / kFirCols;
    const int c0 = (cr.local % ncol) * kFirCols;
    const int t0 = (cr.local / ncol) * kFirTY;

    extern __shared__ __align__(16) ulonglong2 ring[];  // kFirRing x 32 lanes x 4 columns
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    // column c = (cell, channel): c / D by multiply-high with ceil(2^32 / D),
    // exact for c < 2^26 and 2 <= D <= 64 (the host keeps max(H, W) * D <=
    // 2^26); D = 1 is the identity
    const unsigned dinv = D > 1 ? (unsigned)((0x100000000ull + (unsigned)D - 1) / (unsigned)D) : 0u;
    long long inoff[4];
    int ccell[4], cch[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = c0 + 32 * k + lane;
        ok[k] = c < NC;
        ccell[k] = D > 1 ? (int)__umulhi((unsigned)c, dinv) : c;
        cch[k] = c - ccell[k] * D;
        inoff[k] = ok[k] ? (long long)ccell[k] * in_cell + cch[k] : 0;
    }

    // CTA step range: non-zero taps that reach an in-range row for some output
    int jlo = max(rp - r, rp - (t0 + kFirTY - 1));
    jlo = jlo / X * X;
    const int jhi = min(rp + r, rp + R - 1 - t0);
    const int jend = min(ntp, (jhi + X) / X * X);
    // warp step range: the same for this warp's 8 output rows
    const int rbase = q * X;
    const int ylo = t0 + rbase;
    const bool wact = ylo < R;
    const int yhi = min(ylo + X, R) - 1;
    int wlo = max(rp - r, rp - yhi);
    wlo = max(jlo, wlo / X * X);
    const int whi = min(rp + r, rp + R - 1 - ylo);
    const int wend = min(jend, (whi + X) / X * X);

    const int span = kFirTY + X;  // rows read past the last step of a chunk
    // row fetch: ring row t holds input row t0 - rp + t (zero outside [0, R));
    // per lane the four column pointers, copy sizes and the ring address are
    // set up once, so a row costs one multiply, four 64-bit adds and four copies
    const float* colp[4];
    int csz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        colp[k] = in + inoff[k];
        csz[k] = ok[k] ? 4 : 0;
    }
    const int tlo = rp - t0, thi = rp - t0 + R;  // ring rows holding grid rows
    const unsigned ring_sa = (unsigned)__cvta_generic_to_shared(ring) + 16u * (unsigned)lane;
    auto fetch = [&](int t) {
        const unsigned sa = ring_sa + 512u * (unsigned)TL::slot(t);
        if (t >= tlo && t < thi) {  // warp-uniform
            const long long off = (long long)(t - tlo) * in_row;
            cp_async_f32_at<0>(sa, colp[0] + off, csz[0]);
            cp_async_f32_at<4>(sa, colp[1] + off, csz[1]);
            cp_async_f32_at<8>(sa, colp[2] + off, csz[2]);
            cp_async_f32_at<12>(sa, colp[3] + off, csz[3]);
        } else {
            cp_async_f32_at<0>(sa, colp[0], 0);
            cp_async_f32_at<4>(sa, colp[1], 0);
            cp_async_f32_at<8>(sa, colp[2], 0);
            cp_async_f32_at<12>(sa, colp[3], 0);
        }
    };
    // taps of a chunk, (k, k) pairs, double-buffered next to the ring
    __shared__ __align__(16) unsigned long long tapbuf[2][kFirChunk];
    const unsigned long long* tp = reinterpret_cast<const unsigned long long*>(taps);
    auto fetch_taps = [&](int from, int to, int b) {  // steps [from, to), multiples of 8
        for (int p = threadIdx.x; 2 * p < to - from; p += kFirThreads)
            cp_async_16(&tapbuf[b][2 * p], tp + from + 2 * p);
    };
    int loaded_end = min(jlo + kFirChunk, jend) + span;
    fetch_taps(jlo, min(jlo + kFirChunk, jend), 0);
    for (int t = jlo + q; t < loaded_end; t += NW) fetch(t);
    cp_async_wait_all();
    __syncthreads();

    float2 acc[X][2];
    float4 win[X];
#pragma unroll
    for (int i = 0; i < X; ++i) acc[i][0] = acc[i][1] = make_float2(0.0f, 0.0f);
    const float4* fring = reinterpret_cast<const float4*>(ring);
    bool started = false;
    int ci = 0;
    for (int jc = jlo; jc < jend; jc += kFirChunk, ++ci) {
        const int cend = min(jc + kFirChunk, jend);
        // the ring holds >= 2 chunks + kFirTY + X rows, so the next chunk's rows
        // never land on a row that the current chunk still reads; the other tap
        // buffer was last read by the previous chunk, before its barrier
        const int next_end = min(cend + kFirChunk, jend) + span;
        if (cend < jend) fetch_taps(cend, min(cend + kFirChunk, jend), (ci + 1) & 1);
        for (int t = loaded_end + q; t < next_end; t += NW) fetch(t);
        loaded_end = max(loaded_end, next_end);
        const unsigned long long* tb = tapbuf[ci & 1];
        if (wact) {
            const int s0 = max(jc, wlo), s1 = min(cend, wend);
            if (s0 < s1) {
                if (!started) {
#pragma unroll
                    for (int u = 0; u < X; ++u) win[u] = fring[TL::slot(rbase + s0 + u) * 32 + lane];
                    started = true;
                }
                for (int jb = s0; jb < s1; jb += X) {
                    const int nb = TL::slot(rbase + jb + X);  // a multiple of 8: nb + 7 < RING
#pragma unroll
                    for (int u = 0; u < X; u += 2) {
                        // taps of steps jb+u and jb+u+1 as two (k, k) pairs
                        const float4 k4 = *reinterpret_cast<const float4*>(tb + (jb - jc + u));
                        const float2 ka = make_float2(k4.x, k4.y), kb = make_float2(k4.z, k4.w);
#pragma unroll
                        for (int i = 0; i < X; ++i) {
                            const float4 w = win[(u + i) % X];
                            acc[i][0] = __ffma2_rn(ka, make_float2(w.x, w.y), acc[i][0]);
                            acc[i][1] = __ffma2_rn(ka, make_float2(w.z, w.w), acc[i][1]);
                        }
                        win[u] = fring[(nb + u) * 32 + lane];
#pragma unroll
                        for (int i = 0; i < X; ++i) {
                            const float4 w = win[(u + 1 + i) % X];
                            acc[i][0] = __ffma2_rn(kb, make_float2(w.x, w.y), acc[i][0]);
                            acc[i][1] = __ffma2_rn(kb, make_float2(w.z, w.w), acc[i][1]);
                        }
                        win[u + 1] = fring[(nb + u + 1) * 32 + lane];
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    if (wact) {
        float* out;
        long long out_row, out_cell;
        const float* norm;
        if (pass == 0) {
            out = gr.H1; out_row = D; out_cell = (long long)gr.H * D;
            norm = gr.table + lv.off_ny;
        } else {
            out = gr.T; out_row = ts; out_cell = (long long)gr.W * ts;
            norm = gr.table + lv.off_nx;
        }
        const float* rnorm = norm + ((R + 3) & ~3);  // RN(1/n) per position
        long long ooff[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ooff[k] = ok[k] ? (long long)ccell[k] * out_cell + cch[k] : 0;
#pragma unroll
        for (int i = 0; i < X; ++i) {
            const int y = ylo + i;
            if (y < R) {
                const float nrm = norm[y];
                const float rcp = rnorm[y];
                float* orow = out + (long long)y * out_row;
                const float v[4] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (ok[k]) orow[ooff[k]] = div_rn(v[k], nrm, rcp);
            }
        }
    }

    // the iteration's grouping table (the state is not written before the
    // assignment launch's schedule step)
    if (pass == 0) write_group_table(gr, lv, st, cr.local, cr.count, kFirThreads);
}

// Small radii: a kernel without shared memory or barriers.  A CTA of 4 warps
// owns 32 output rows x 64 columns; warp q owns rows 8q..8q+7 and lane l the
// columns c0+l and c0+32+l as one packed pair.  The warp loads every input row
// that its tap steps reach straight into registers with read-only loads (L2
// serves the rows that neighbouring warps share) and then runs the same
// ascending FMA chains as the ring kernel: step s of output row i is input
// row base + s + i.  Up to three 8-step blocks are unrolled with all loads
// issued first; longer step ranges run block by block, in the same order.
constexpr int kDirTY = 32, kDirCols = 64, kDirThreads = 128;

template <int NB>
__device__ __forceinline__ void dir_chains(const float* __restrict__ in, long long in_row,
                                           const long long (&inoff)[2], const bool (&ok)[2], int R,
                                           int base, const float2* __restrict__ tp,
                                           float2 (&acc)[kFirX]) {
    constexpr int X = kFirX, NR = NB * X + X - 1;
    float2 w[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        const int yy = base + m;
        float2 v = make_float2(0.0f, 0.0f);
        if (yy >= 0 && yy < R) {  // warp-uniform
            const float* p = in + (long long)yy * in_row;
            if (ok[0]) v.x = __ldg(p + inoff[0]);
            if (ok[1]) v.y = __ldg(p + inoff[1]);
        }
        w[m] = v;
    }
#pragma unroll
    for (int s = 0; s < NB * X; ++s) {
        const float2 k = __ldg(tp + s);
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i] = __ffma2_rn(k, w[s + i], acc[i]);
    }
}

__global__ void __launch_bounds__(kDirThreads) fir_direct_kernel(
    int pass, const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, int D, int gs,
    int ts) {
    constexpr int X = kFirX;
    const CtaRef cr = resolve_cta(map);
    const GridRef& gr = grids[cr.g];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];

    const float* in;
    long long in_row, in_cell;
    int R, NC, r, rp, ntp;
    const float* taps;
    if (pass == 0) {  // along y: G -> H1 ([x][y][d])
        in = gr.G; in_row = (long long)gr.W * gs; in_cell = gs;
        R = gr.H; NC = gr.W * D;
        r = lv.ry; rp = lv.rpy; ntp = lv.ntpy;
        taps = gr.table + lv.off_ty;
    } else {          // along x: H1 -> T ([y][x][d], cell stride ts)
        in = gr.H1; in_row = (long long)gr.H * D; in_cell = D;
        R = gr.W; NC = gr.H * D;
        r = lv.rx; rp = lv.rpx; ntp = lv.ntpx;
        taps = gr.table + lv.off_tx;
    }
    const int ncol = (NC + kDirCols - 1) / kDirCols;
    const int c0 = (cr.local % ncol) * kDirCols;
    const int t0 = (cr.local / ncol) * kDirTY;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const unsigned dinv = D > 1 ? (unsigned)((0x100000000ull + (unsigned)D - 1) / (unsigned)D) : 0u;
    long long inoff[2];
    int ccell[2], cch[2];
    bool ok[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c = c0 + 32 * k + lane;
        ok[k] = c < NC;
        ccell[k] = D > 1 ? (int)__umulhi((unsigned)c, dinv) : c;
        cch[k] = c - ccell[k] * D;
        inoff[k] = ok[k] ? (long long)ccell[k] * in_cell + cch[k] : 0;
    }
    const int ylo = t0 + q * X;
    if (ylo < R) {
        // the warp's step range: non-zero taps that reach an in-range row
        const int yhi = min(ylo + X, R) - 1;
        int wlo = max(rp - r, rp - yhi);
        wlo = wlo / X * X;
        const int whi = min(rp + r, rp + R - 1 - ylo);
        const int wend = min(ntp, (whi + X) / X * X);
        float2 acc[X];
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i] = make_float2(0.0f, 0.0f);
        const float2* tp = reinterpret_cast<const float2*>(taps) + wlo;
        const int base = ylo - rp + wlo;
        const int nb = (wend - wlo) / X;
        if (nb == 1) {
            dir_chains<1>(in, in_row, inoff, ok, R, base, tp, acc);
        } else if (nb == 2) {
            dir_chains<2>(in, in_row, inoff, ok, R, base, tp, acc);
        } else if (nb == 3) {
            dir_chains<3>(in, in_row, inoff, ok, R, base, tp, acc);
        } else {
            for (int b = 0; b < nb; ++b) dir_chains<1>(in, in_row, inoff, ok, R, base + X * b, tp + X * b, acc);
        }
        float* out;
        long long out_row, out_cell;
        const float* norm;
        if (pass == 0) {
            out = gr.H1; out_row = D; out_cell = (long long)gr.H * D;
            norm = gr.table + lv.off_ny;
        } else {
            out = gr.T; out_row = ts; out_cell = (long long)gr.W * ts;
            norm = gr.table + lv.off_nx;
        }
        const float* rnorm = norm + ((R + 3) & ~3);  // RN(1/n) per position
        long long ooff[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) ooff[k] = ok[k] ? (long long)ccell[k] * out_cell + cch[k] : 0;
#pragma unroll
        for (int i = 0; i < X; ++i) {
            const int y = ylo + i;
            if (y < R) {
                const float nrm = norm[y];
                const float rcp = rnorm[y];
                float* orow = out + (long long)y * out_row;
                const float v[2] = {acc[i].x, acc[i].y};
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (ok[k]) orow[ooff[k]] = div_rn(v[k], nrm, rcp);
            }
        }
    }
    if (pass == 0) write_group_table(gr, lv, st, cr.local, cr.count, kDirThreads);
}

int fir_ctas(int rows, int cols, int variant) {
    if (variant == kFirSmallRadius) return ((cols + kDirCols - 1) / kDirCols) * ((rows + kDirTY - 1) / kDirTY);
    const int ty = variant == kFirMediumRadius ? FirMedium::TY : FirLarge::TY;
    return ((cols + kFirCols - 1) / kFirCols) * ((rows + ty - 1) / ty);
}

template <class TL>
static size_t fir_smem() { return sizeof(ulonglong2) * TL::RING * 32; }

static void fir_opt_in() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(fir_kernel<FirLarge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fir_smem<FirLarge>());
    cudaFuncSetAttribute(fir_kernel<FirMedium>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fir_smem<FirMedium>());
    done[dev] = true;
}

void prepare_fir_launches() { fir_opt_in(); }

void launch_fir(int pass, const GridRef* grids, const CtaMap* map, int ctas, int D, int variant,
                cudaStream_t s) {
    if (ctas <= 0) return;
    fir_opt_in();
    if (variant == kFirSmallRadius)
        fir_direct_kernel<<<ctas, kDirThreads, 0, s>>>(pass, grids, map, D, grid_stride(D),
                                                        target_stride(D));
    else if (variant == kFirMediumRadius)
        fir_kernel<FirMedium><<<ctas, FirMedium::THREADS, fir_smem<FirMedium>(), s>>>(
            pass, grids, map, D, grid_stride(D), target_stride(D));
    else
        fir_kernel<FirLarge><<<ctas, FirLarge::THREADS, fir_smem<FirLarge>(), s>>>(
            pass, grids, map, D, grid_stride(D), target_stride(D));
}

}  // namespace plas
