// sweep_bodies.cuh -- the per-work-item bodies of the chunked ring target
// pass and of the assignment step of the PLAS sort (Sec. 3.1 of Morgenstern
// et al., arXiv 2312.13299), shared by their one-launch-per-class kernels
// (fir_kernels.cu, sort_kernels.cu) and by the persistent sweep kernel
// (persist_kernels.cu), which runs many iterations of many grids in one
// cooperative launch.  A body processes one work item (a tile of a target
// pass, or a slice of a grid's groups) with the whole CTA.
#pragma once

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
// 16-byte copy global -> shared through L2 only (data read once); with
// take = false the destination is zero-filled and nothing is read
__device__ __forceinline__ void cp_async_cg16(float4* sdst, const float* gsrc, bool take) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc),
                 "r"(take ? 16 : 0)
                 : "memory");
}


template <class TL>
__device__ __forceinline__ void fir_ring_body(int pass, const GridRef* __restrict__ grids,
                                              const CtaRef cr, int D, int gs, int ts,
                                              ulonglong2* __restrict__ ring) {
    constexpr int X = kFirX;
    constexpr int kFirTY = TL::TY, kFirChunk = TL::CH;
    constexpr int kFirThreads = TL::THREADS;
    constexpr int NW = kFirThreads / 32;
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
        in = gr.H1; in_row = h1_stride(gr.H, D); in_cell = D;
        R = gr.W; NC = gr.H * D;
        r = lv.rx; rp = lv.rpx; ntp = lv.ntpx;
        taps = gr.table + lv.off_tx;
    }
    const int ncol = (NC + kFirCols - 1) / kFirCols;
    const int c0 = (cr.local % ncol) * kFirCols;
    const int t0 = (cr.local / ncol) * kFirTY;

    // ring: TL::RING rows x 32 lanes x 4 columns of shared memory
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
            out = gr.H1; out_row = D; out_cell = h1_stride(gr.H, D);
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

// RO: through the read-only data path (data not written during the launch);
// otherwise ordinary loads (a persistent launch rewrites the target).
template <int N4, bool RO = true>
__device__ __forceinline__ void load_row4(const float* __restrict__ p, float* v) {
#pragma unroll
    for (int k = 0; k < N4; ++k) {
        const float4 a = RO ? __ldg(reinterpret_cast<const float4*>(p) + k)
                            : reinterpret_cast<const float4*>(p)[k];
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

// rint(e * 2^k) as an integer.  Scaling by a power of two is exact in FP32
// (e * 2^k < 2^62 here), so this equals rint((double)e * 2^k) without the
// FP64 pipe.
__device__ __forceinline__ unsigned long long fixed_point(float e, float scale) {
    return (unsigned long long)__float2ll_rn(__fmul_rn(e, scale));
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

// The six permutations that send cell 0 to target a are numbers 6a..6a+5 of
// the lexicographic order; with r0 < r1 < r2 the other three targets they
// send cells 1, 2, 3 to (r0 r1 r2), (r0 r2 r1), (r1 r0 r2), (r1 r2 r0),
// (r2 r0 r1), (r2 r1 r0): kRest6[w] indexes (r0, r1, r2) for permutation
// 6a + w.  kKeys[a] packs the lexicographic keys (targets of cells 0..3 as
// base-4 digits, cell 0 most significant) of those six permutations, eight
// bits each.
__device__ constexpr int kRest6[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                         {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
struct PermKeys {
    unsigned long long k[4];
};
__host__ __device__ constexpr PermKeys make_perm_keys() {
    PermKeys t{};
    const Perm24 p = make_perm24();
    for (int a = 0; a < 4; ++a)
        for (int w = 0; w < 6; ++w) {
            const int* q = p.p[6 * a + w];
            const unsigned long long key =
                (unsigned long long)((q[0] << 6) | (q[1] << 4) | (q[2] << 2) | q[3]);
            t.k[a] |= key << (8 * w);
        }
    return t;
}
// compile-time check of the layout above against the lexicographic table
__host__ __device__ constexpr bool perm_split_ok() {
    const Perm24 p = make_perm24();
    constexpr int rest6[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int a = 0; a < 4; ++a) {
        const int r[3] = {a == 0 ? 1 : 0, a <= 1 ? 2 : 1, a <= 2 ? 3 : 2};
        for (int w = 0; w < 6; ++w) {
            if (p.p[6 * a + w][0] != a) return false;
            for (int m = 0; m < 3; ++m)
                if (p.p[6 * a + w][m + 1] != r[rest6[w][m]]) return false;
        }
    }
    return true;
}
static_assert(perm_split_ok(), "permutations 6a..6a+5 are (a, rest in lexicographic order)");

// Schedule step (Sec. 3.1): d = mean L2 distance to the target; an assignment
// that improves d by less than tol (relative) is a stall; one stall draws a
// new block shift, a second in a row shrinks the radius; the sort ends when
// the radius falls below phi_min (no levels left).
static __device__ void schedule_step(DevState* st, long long N, int nby, int nbx, int ngroups,
                              int nlevels, double tol, long long* trace_S, int* trace_level,
                              long long trace_cap, double fmas_y, double fmas_x, double beta2) {
    st->fmas_y += fmas_y;
    if (st->fused_pending) {  // both passes ran in the pass-0 launch
        st->fmas_xf += fmas_x;
        st->fused_its += 1;
        st->fused_pending = 0;
    } else {
        st->fmas_x += fmas_x;
    }
    st->beta2_sum += beta2;
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
    // cells of the groups (with cut blocks an upper bound, capped at N)
    st->grouped += std::min<long long>((long long)nby * nbx * ngroups * 4, N);
    if (st->level >= nlevels) st->done = 1;
    st->S = 0ull;
    st->arrivals = 0u;
    __threadfence();
}

template <bool RO, class T>
__device__ __forceinline__ T ldg_ro(const T* p) {
    return RO ? __ldg(p) : *p;
}

// One work item of the assignment with the whole CTA (kAssignThreads
// threads): slice cr.local of cr.count of grid cr.g's groups and cells.  RO:
// the target and the grouping table are read through the read-only path
// (they are not written during the launch).  CHECKED: every grouping entry
// and cell position is checked against the block and the grid first.
template <int D, bool RO, bool CHECKED = false>
__device__ __forceinline__ void assign_body(const GridRef* __restrict__ grids, const CtaRef cr,
                                            double tol) {
    constexpr int GS = (D + 1 + 3) & ~3, TS = (D + 3) & ~3;
    __shared__ unsigned long long s_part[kAssignThreads / 32];
    const GridRef& gr = grids[cr.g];
    DevState* st = gr.st;
    const int H = gr.H, W = gr.W;
    // Every thread reads the state and derives the block shift itself: the
    // state changes only in the schedule step, after every CTA of this launch
    // has passed its final barrier and arrived.
    if (sweep_idle(st)) return;
    const int beta = gr.lv[st->level].beta;
    int dy, dx;
    block_shift(gr.seed, st->epoch, beta, H, W, &dy, &dx);
    // block origins (Sec. 3.1): every block that meets the grid, the ones cut
    // by the top/left border included (edge reading, the default), or the
    // whole blocks from (dy, dx) on
    const bool edge = gr.edge_blocks != 0;
    const int oy0 = edge && dy > 0 ? dy - beta : dy, ox0 = edge && dx > 0 ? dx - beta : dx;
    const int nby = edge ? (H - oy0 + beta - 1) / beta : (H - dy) / beta;
    const int nbx = edge ? (W - ox0 + beta - 1) / beta : (W - dx) / beta;
    const int ngroups = (beta * beta) / 4;
    // N <= 2^26 (checked on the host), so every cell and group index fits 32 bits
    const int ngt = nby * nbx * ngroups;
    const float scale = ldexpf(1.0f, st->scale_exp);  // 2^k, 0 <= k <= 32
    float* __restrict__ G = gr.G;
    const float* __restrict__ T = gr.T;
    const uint32_t* __restrict__ pi = gr.pi;
    unsigned long long part = 0ull;

    const int lane = threadIdx.x & 31, qi = lane & 3, qbase = lane & ~3, q = lane >> 2;
    // Row staging (up to 16 channels): per warp, the 32 grid rows of its 8
    // quads at an odd stride of SG float4s, and the 32 target rows at an odd
    // stride ST with one float4 between quads, so that the shared-memory reads
    // below (lane i: grid row i of its quad; the quad: one target row) are
    // free of bank conflicts.
    constexpr bool kStaged = D <= 16;
    constexpr int NG = GS / 4, NT = TS / 4, SG = NG | 1, ST = NT | 1, QT = 4 * ST + 1;
    constexpr int kWarpStage = 32 * SG + 8 * QT;
    __shared__ float4 s_stage[kStaged ? (kAssignThreads / 32) * kWarpStage : 1];
    float4* const sg = s_stage + (kStaged ? (int)(threadIdx.x >> 5) * kWarpStage : 0);
    float4* const stt = sg + 32 * SG;
    const int gwarp = (cr.local * kAssignThreads + (int)threadIdx.x) >> 5;
    const int nwarps = (cr.count * kAssignThreads) >> 5;
    constexpr PermKeys kPermKeys = make_perm_keys();
    // ---- groups: 8 per warp ----
    // Lane cursor: the lane's group task = (by * nbx + bx) * ngroups + g is
    // advanced by S = 8 * nwarps per step without dividing: S splits once
    // into whole blocks and a remainder.  The grouping-table entries of the
    // next step are read one step ahead, so each step waits for one memory
    // round trip, not two.
    const uint32_t ug = (uint32_t)ngroups, unbx = (uint32_t)nbx;
    const uint32_t S = (uint32_t)nwarps * 8u;
    const uint32_t Sg = S % ug, Sb = S / ug, Sbx = Sb % unbx, Sby = Sb / unbx;
    uint32_t cg, cbx, cby;
    {
        const uint32_t t = (uint32_t)(gwarp * 8 + (lane >> 2)), b = t / ug;
        cg = t - b * ug;
        cby = b / unbx;
        cbx = b - cby * unbx;
    }
    const uint4* __restrict__ pi4 = reinterpret_cast<const uint4*>(pi);
    uint4 l4_next = make_uint4(0u, 0u, 0u, 0u);
    if (gwarp * 8 < ngt) l4_next = ldg_ro<RO>(pi4 + cg);  // cg < ngroups always
#pragma unroll 1
    for (int base = gwarp * 8; base < ngt; base += nwarps * 8) {
        const bool active = base + (lane >> 2) < ngt;
        const int oy = oy0 + (int)cby * beta, ox = ox0 + (int)cbx * beta;
        const uint4 l4 = l4_next;
        {
            cg += Sg;
            const uint32_t carry = cg >= ug ? 1u : 0u;
            cg -= carry ? ug : 0u;
            cbx += Sbx + carry;
            if (cbx >= unbx) {
                cbx -= unbx;
                cby += 1u;
            }
            cby += Sby;
        }
        if (base + nwarps * 8 < ngt) l4_next = ldg_ro<RO>(pi4 + cg);
        const uint32_t ls[4] = {l4.x, l4.y, l4.z, l4.w};
        // cells of the group; a cell beyond the grid border (edge reading)
        // reads cell 0 and takes no part: its group stays put
        int pos[4];
        unsigned inmask = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int yy = oy + (int)(ls[k] >> 16), xx = ox + (int)(ls[k] & 0xFFFFu);
            const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
            inmask |= (unsigned)in << k;
            pos[k] = in ? yy * W + xx : 0;
        }
        const bool inside = inmask == 15u;
        if (CHECKED) {
            // checked run: every grouping entry must lie in the block and every
            // cell position in the grid; a violation is recorded and the
            // warp's groups skipped
            bool inb = edge || inside;
#pragma unroll
            for (int k = 0; k < 4; ++k) inb = inb && (ls[k] >> 16) < (uint32_t)beta && (ls[k] & 0xFFFFu) < (uint32_t)beta && pos[k] >= 0 && pos[k] < H * W;
            if (!__all_sync(0xFFFFFFFFu, !active || inb)) {
                if (active && !inb) atomicCAS(&st->status, 0, -7);  // PLAS_ERR_INTERNAL
                continue;
            }
        }
        float c[4];
        float grow[GS];  // the lane's own grid row (all of it without staging)
        if (kStaged) {
            // the quad copies its four grid rows and four target rows into the
            // warp's staging area, lane qi taking float4s qi, qi + 4, ... of
            // the rows laid end to end, so every copy instruction moves whole
            // 64-byte rows (one memory transaction per row, not per lane).
            // Rows of cells beyond the border (and of idle quads) are
            // zero-filled without a read: their costs are never used.
#pragma unroll
            for (int m = 0; m < NG; ++m) {
                const int e = qi + 4 * m, row = e / NG, col = e - row * NG;
                cp_async_cg16(sg + (4 * q + row) * SG + col,
                              G + (size_t)pick4i(pos, row) * GS + 4 * col,
                              active && ((inmask >> row) & 1u));
            }
#pragma unroll
            for (int m = 0; m < NT; ++m) {
                const int e = qi + 4 * m, row = e / NT, col = e - row * NT;
                cp_async_cg16(stt + q * QT + row * ST + col,
                              T + (size_t)pick4i(pos, row) * TS + 4 * col,
                              active && ((inmask >> row) & 1u));
            }
            cp_async_wait_all();
            __syncwarp();
            // cost row qi, ascending channels: c[j] = sum_d (g_d - t_j,d)^2
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                const float4 v = sg[(4 * q + qi) * SG + k];
                grow[4 * k] = v.x; grow[4 * k + 1] = v.y; grow[4 * k + 2] = v.z; grow[4 * k + 3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float trow[TS];
#pragma unroll
                for (int k = 0; k < NT; ++k) {
                    const float4 v = stt[q * QT + j * ST + k];
                    trow[4 * k] = v.x; trow[4 * k + 1] = v.y; trow[4 * k + 2] = v.z; trow[4 * k + 3] = v.w;
                }
                c[j] = sqdist<D>(grow, trow);
            }
        } else {
            // lane qi loads the grid row and the target row of its own cell;
            // the quad passes the target rows around with shuffles
            float trow[TS];
            const int mypos = pick4i(pos, qi);
            load_row4_rw<GS / 4>(G + (size_t)mypos * GS, grow);
            load_row4<TS / 4, RO>(T + (size_t)mypos * TS, trow);
            // cost row qi, ascending channels: cr[m] = sum_d (g_d - t_d)^2
            // against the target row of lane (qi + m) & 3 of the quad
            float cr[4];
            cr[0] = sqdist<D>(grow, trow);
#pragma unroll
            for (int m = 1; m < 4; ++m) {
                const int src = qbase | ((qi + m) & 3);
                float acc = 0.0f;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float delta = __fsub_rn(grow[d], __shfl_sync(0xFFFFFFFFu, trow[d], src));
                    acc = __fmaf_rn(delta, delta, acc);
                }
                cr[m] = acc;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) c[j] = pick4(cr, (j - qi) & 3);
        }
        // all-gather the cost matrix inside the quad
        float C[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) C[i][j] = __shfl_sync(0xFFFFFFFFu, c[j], qbase | i);
        // lane qi scores the six permutations that send cell 0 to target qi
        // (kRest6), keeping the first strict minimum; the quad then takes the
        // lowest cost, on equal costs the lowest lexicographic key, which is
        // the first strict minimum over all 24 in lexicographic order
        float x[4][3];  // x[i][m] = C[i][r_m], the targets other than qi in order
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            x[i][0] = qi == 0 ? C[i][1] : C[i][0];
            x[i][1] = qi <= 1 ? C[i][2] : C[i][1];
            x[i][2] = qi <= 2 ? C[i][3] : C[i][2];
        }
        const float c0 = pick4(C[0], qi);
        float best = 0.0f;
        int bw = 0;
#pragma unroll
        for (int w = 0; w < 6; ++w) {
            const float sc = __fadd_rn(
                __fadd_rn(__fadd_rn(c0, x[1][kRest6[w][0]]), x[2][kRest6[w][1]]),
                x[3][kRest6[w][2]]);
            if (w == 0 || sc < best) {
                best = sc;
                bw = w;
            }
        }
        const unsigned long long keys =
            qi == 0 ? kPermKeys.k[0] : (qi == 1 ? kPermKeys.k[1] : (qi == 2 ? kPermKeys.k[2] : kPermKeys.k[3]));
        unsigned key = (unsigned)(keys >> (8 * bw)) & 0xFFu;
#pragma unroll
        for (int off = 1; off < 4; off <<= 1) {
            const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
            const unsigned okey = __shfl_xor_sync(0xFFFFFFFFu, key, off);
            if (ob < best || (ob == best && okey < key)) {
                best = ob;
                key = okey;
            }
        }
        // a group with a cell beyond the border keeps its arrangement; each of
        // its cells inside the grid adds its own distance
        const int my_dst = inside ? (int)(key >> (6 - 2 * qi)) & 3 : qi;
        if (kStaged) {
            // the quad writes its staged rows back whole: row j moves to cell
            // pos[sigma(j)], lane qi taking the same float4s as in the copy
            if (active && inside) {
#pragma unroll
                for (int m = 0; m < NG; ++m) {
                    const int e = qi + 4 * m, row = e / NG, col = e - row * NG;
                    const int dst = pick4i(pos, (int)(key >> (6 - 2 * row)) & 3);
                    reinterpret_cast<float4*>(G + (size_t)dst * GS)[col] = sg[(4 * q + row) * SG + col];
                }
            }
            __syncwarp();  // the stage is refilled by the next iteration
        } else if (active && inside) {
            float4* dst = reinterpret_cast<float4*>(G + (size_t)pick4i(pos, my_dst) * GS);
#pragma unroll
            for (int k = 0; k < GS / 4; ++k)
                dst[k] = make_float4(grow[4 * k], grow[4 * k + 1], grow[4 * k + 2], grow[4 * k + 3]);
        }
        if (active && ((inmask >> qi) & 1u)) part += fixed_point(__fsqrt_rn(pick4(c, my_dst)), scale);
    }

    // ---- cells outside the full blocks (enumerated directly: the rows above
    // and below the covered band, then the left and right margins of it) ----
    // (none under the edge reading: the blocks cover the grid)
    const int cy0 = dy, cy1 = dy + nby * beta, cx0 = dx, cx1 = dx + nbx * beta;
    const int gthread = cr.local * kAssignThreads + (int)threadIdx.x;
    const int nthreads = cr.count * kAssignThreads;
    const int n_top = cy0 * W, n_bot = (H - cy1) * W, margin = W - (cx1 - cx0);
    const int n_unc = edge ? 0 : n_top + n_bot + (cy1 - cy0) * margin;
#pragma unroll 1
    for (int e = gthread; e < n_unc; e += nthreads) {
        int y, x;
        if (e < n_top + n_bot) {
            const int f = e < n_top ? e : e - n_top + cy1 * W;
            y = (int)((uint32_t)f / (uint32_t)W);
            x = f - y * W;
        } else {
            const int f = e - n_top - n_bot;
            const int row = (int)((uint32_t)f / (uint32_t)margin), c = f - row * margin;
            y = cy0 + row;
            x = c < cx0 ? c : cx1 + (c - cx0);
        }
        const int p = y * W + x;
        float grow[GS], trow[TS];
        load_row4_rw<GS / 4>(G + (size_t)p * GS, grow);
        load_row4<TS / 4, RO>(T + (size_t)p * TS, trow);
        part += fixed_point(__fsqrt_rn(sqdist<D>(grow, trow)), scale);
    }
    // ---- leftover cells of each block (beta^2 mod 4 of them) ----
    const int nleft = beta * beta - 4 * ngroups;
    const int nl = nby * nbx * nleft;
#pragma unroll 1
    for (int e = gthread; e < nl; e += nthreads) {
        const int blk = (int)((uint32_t)e / (uint32_t)nleft);
        const int m = 4 * ngroups + (e - blk * nleft);
        const int by = (int)((uint32_t)blk / (uint32_t)nbx), bx = blk - by * nbx;
        const uint32_t l = pi[m];
        const int ly = (int)(l >> 16), lx = (int)(l & 0xFFFFu);
        const int yy = oy0 + by * beta + ly, xx = ox0 + bx * beta + lx;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;  // (edge reading)
        const int p = yy * W + xx;
        float grow[GS], trow[TS];
        load_row4_rw<GS / 4>(G + (size_t)p * GS, grow);
        load_row4<TS / 4, RO>(T + (size_t)p * TS, trow);
        part += fixed_point(__fsqrt_rn(sqdist<D>(grow, trow)), scale);
    }

    // ---- exact reduction; the grid's last CTA runs the schedule ----
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
    if (lane == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0ull;
        for (int w = 0; w < kAssignThreads / 32; ++w) tot += s_part[w];
        atomicAdd(&st->S, tot);
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->arrivals, 1u);
        if (ticket == (unsigned)cr.count - 1u) {
            __threadfence();
            const LevelDesc& lv = gr.lv[st->level];
            // in-range tap FMAs of the Gaussian passes (none for the box target)
            const double fy = gr.target_mode == 1 ? 0.0 : pass_taps(H, lv.ry) * (double)W * D;
            const double fx = gr.target_mode == 1 ? 0.0 : pass_taps(W, lv.rx) * (double)H * D;
            schedule_step(st, (long long)H * W, nby, nbx, ngroups, gr.nlev, tol, gr.trace_S, gr.trace_level,
                          gr.trace_cap, fy, fx, (double)beta * beta);
        }
    }
}


}  // namespace plas
