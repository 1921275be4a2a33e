// box_kernels.cu -- the box target (schedule.target_mode = 1), a fast
// low-pass variant of the idealised target of Sec. 3.1 (Morgenstern et al.,
// arXiv 2312.13299): the mean of the in-range cells of the (2r+1) x (2r+1)
// window around each cell, on fixed-point features q = rint(F 2^s).
//
// The window sums are exact int64 arithmetic, so any order of summation gives
// the same sums, and the cost does not depend on r.  Two launches:
//   1. column prefix sums P(y, x) = sum_{y' <= y} q(y', x), read straight
//      from the working grid (one CTA per cell column);
//   2. per (row, channel pair): the window's column sums
//      V(x) = P(y+r, x) - P(y-r-1, x) (rows clipped to the grid), their
//      prefix along x in shared memory, S(x) = R(x+r) - R(x-r-1) and
//      T = ((float)S / (float)n) * 2^-s   (FP32, IEEE division);
//      this launch also writes the iteration's grouping table.
// The same bits as the oracle's sliding window sums.  Rows wider than
// kRowsMaxW cells (whose prefix does not fit in shared memory) take a
// three-launch path over a full summed-area table I(y, x) instead: a scan
// along x, a scan along y, four corner reads per output.
#include <algorithm>

#include "plas_kernels.h"

namespace plas {

namespace {

constexpr int kScanThreads = 256;
constexpr int kEvalThreads = 256;
constexpr int kRowThreads = 256;
constexpr int kRowsMaxW = 6144;  // prefix of one channel pair of a row: 16 B per cell, <= 96 KB

__device__ __forceinline__ float pow2f(int e) { return ldexpf(1.0f, e); }  // exact for |e| <= 126

// The summed-area table holds DP = D rounded up to even int64 channels per
// cell (the pad channel stays 0), so every channel pair is one aligned
// 16-byte access.
__host__ __device__ constexpr int sat_channels(int D) { return (D + 1) & ~1; }

__device__ __forceinline__ long long shfl_up64(long long v, int delta) {
    return (long long)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)v, delta);
}

// prefix sums along x of q = rint(F 2^s): one CTA per row; thread t owns the
// cells [t*cpt, (t+1)*cpt) and all D channels (float4 loads of the cell's
// features, 16-byte stores of channel pairs).  The per-thread channel totals
// are scanned across the CTA with warp shuffles.  Exact int64.
template <int D>
__global__ void __launch_bounds__(kScanThreads) box_rowscan_kernel(const GridRef* __restrict__ grids) {
    constexpr int GS = (D + 1 + 3) & ~3, DP = sat_channels(D);
    __shared__ long long wtot[kScanThreads / 32][DP];
    const GridRef& gr = grids[0];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const int W = gr.W, y = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int cpt = (W + kScanThreads - 1) / kScanThreads;
    const int c0 = min(t * cpt, W), c1 = min(c0 + cpt, W);
    const float scale = pow2f(st->box_exp);
    const float* g = gr.G + (long long)y * W * GS;
    auto load_q = [&](int x, long long* q) {
        const float4* c = reinterpret_cast<const float4*>(g + (long long)x * GS);
#pragma unroll
        for (int k = 0; k < GS / 4; ++k) {
            const float4 v = c[k];
            const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * k + j < D) q[4 * k + j] = __float2ll_rn(__fmul_rn(f[j], scale));
        }
    };
    long long tot[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) tot[d] = 0;
    for (int x = c0; x < c1; ++x) {
        long long q[D];
        load_q(x, q);
#pragma unroll
        for (int d = 0; d < D; ++d) tot[d] += q[d];
    }
    // exclusive prefix of the thread totals, per channel, across the CTA
#pragma unroll
    for (int d = 0; d < D; ++d) {
        long long v = tot[d];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = shfl_up64(v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wtot[warp][d] = v;
        tot[d] = v - tot[d];  // exclusive within the warp
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < D; ++d) {
        long long off = 0;
        for (int w = 0; w < warp; ++w) off += wtot[w][d];
        tot[d] += off;
    }
    long long* out = gr.sat + (long long)y * W * DP;
    for (int x = c0; x < c1; ++x) {
        long long q[D];
        load_q(x, q);
#pragma unroll
        for (int d = 0; d < D; ++d) tot[d] += q[d];
        longlong2* o = reinterpret_cast<longlong2*>(out + (long long)x * DP);
#pragma unroll
        for (int k = 0; k < DP / 2; ++k)
            o[k] = make_longlong2(tot[2 * k], 2 * k + 1 < D ? tot[2 * k + 1] : 0LL);
    }
}

// prefix sums along y of the row sums, in place: one CTA per cell column;
// thread (k, j) owns row segment k of channel pair j (16-byte accesses).
// Phase 1 sums the segments, phase 2 scans the segment totals per pair,
// phase 3 walks the segments again (L1-resident: one cell column is
// H x DP x 8 bytes) and writes the prefix sums.
__global__ void __launch_bounds__(kScanThreads) box_colscan_kernel(const GridRef* __restrict__ grids, int DP) {
    __shared__ longlong2 tot[kScanThreads];
    const GridRef& gr = grids[0];
    if (sweep_idle(gr.st)) return;
    const int H = gr.H, W = gr.W, x = blockIdx.x;
    const int pairs = DP / 2;
    const int K = kScanThreads / pairs;
    const int L = (H + K - 1) / K;
    const int t = threadIdx.x, k = t / pairs, j = t - (t / pairs) * pairs;
    const bool act = k < K;
    const int y0 = min(k * L, H), y1 = min(y0 + L, H);
    const long long row = (long long)W * DP / 2;  // longlong2 per row
    longlong2* p = reinterpret_cast<longlong2*>(gr.sat) + (long long)x * pairs + j;
    long long s0 = 0, s1 = 0;
    if (act) {
        int y = y0;
        for (; y + 4 <= y1; y += 4) {
            const longlong2 a = p[(long long)y * row], b = p[(long long)(y + 1) * row];
            const longlong2 c = p[(long long)(y + 2) * row], e = p[(long long)(y + 3) * row];
            s0 += a.x + b.x + c.x + e.x;
            s1 += a.y + b.y + c.y + e.y;
        }
        for (; y < y1; ++y) {
            const longlong2 a = p[(long long)y * row];
            s0 += a.x;
            s1 += a.y;
        }
    }
    tot[t] = make_longlong2(s0, s1);
    __syncthreads();
    if (t < pairs) {
        long long r0 = 0, r1 = 0;
        for (int kk = 0; kk < K; ++kk) {
            const longlong2 v = tot[kk * pairs + t];
            tot[kk * pairs + t] = make_longlong2(r0, r1);
            r0 += v.x;
            r1 += v.y;
        }
    }
    __syncthreads();
    if (act) {
        long long r0 = tot[t].x, r1 = tot[t].y;
        for (int y = y0; y < y1; ++y) {
            const longlong2 a = p[(long long)y * row];
            r0 += a.x;
            r1 += a.y;
            p[(long long)y * row] = make_longlong2(r0, r1);
        }
    }
}

// window mean from four corners of the summed-area table, a channel pair per
// thread; writes T and the grouping table
__global__ void __launch_bounds__(kEvalThreads) box_eval_kernel(const GridRef* __restrict__ grids, int D,
                                                                int ts) {
    const GridRef& gr = grids[0];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int H = gr.H, W = gr.W, r = lv.r;
    const int DP = sat_channels(D), pairs = DP / 2;
    const float inv_scale = pow2f(-st->box_exp);
    const long long total = (long long)H * W * pairs;
    const long long rowp = (long long)W * pairs;
    const longlong2* I = reinterpret_cast<const longlong2*>(gr.sat);
    for (long long e = (long long)blockIdx.x * kEvalThreads + threadIdx.x; e < total;
         e += (long long)gridDim.x * kEvalThreads) {
        const long long cell = e / pairs;
        const int j = (int)(e - cell * pairs);
        const int y = (int)(cell / W), x = (int)(cell - (long long)y * W);
        const int y0 = max(y - r, 0) - 1, y1 = min(y + r, H - 1);
        const int x0 = max(x - r, 0) - 1, x1 = min(x + r, W - 1);
        longlong2 S = I[(long long)y1 * rowp + (long long)x1 * pairs + j];
        if (y0 >= 0) {
            const longlong2 v = I[(long long)y0 * rowp + (long long)x1 * pairs + j];
            S.x -= v.x;
            S.y -= v.y;
        }
        if (x0 >= 0) {
            const longlong2 v = I[(long long)y1 * rowp + (long long)x0 * pairs + j];
            S.x -= v.x;
            S.y -= v.y;
        }
        if (y0 >= 0 && x0 >= 0) {
            const longlong2 v = I[(long long)y0 * rowp + (long long)x0 * pairs + j];
            S.x += v.x;
            S.y += v.y;
        }
        const float n = (float)((y1 - y0) * (x1 - x0));
        float* o = gr.T + cell * ts + 2 * j;
        o[0] = __fmul_rn(__fdiv_rn(__ll2float_rn(S.x), n), inv_scale);
        if (2 * j + 1 < D) o[1] = __fmul_rn(__fdiv_rn(__ll2float_rn(S.y), n), inv_scale);
    }
    write_group_table(gr, lv, st, blockIdx.x, gridDim.x, kEvalThreads);
}

// column prefix sums of q = rint(F 2^s), read from the working grid: one CTA
// per cell column; thread (k, j) owns row segment k of channel pair j (8-byte
// loads of the pair's features, 16-byte stores of the pair's sums).  Phase 1
// sums the segments, phase 2 scans the segment totals per pair, phase 3
// walks the segments again (one cell column is H x 4 gs bytes, mostly cache-
// resident) and writes P(y, x) = sum_{y' <= y} q(y', x).
__global__ void __launch_bounds__(kScanThreads) box_colprefix_kernel(const GridRef* __restrict__ grids, int D,
                                                                     int gs) {
    __shared__ longlong2 tot[kScanThreads];
    const GridRef& gr = grids[0];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const int H = gr.H, W = gr.W, x = blockIdx.x;
    const int pairs = sat_channels(D) / 2;
    const int K = kScanThreads / pairs;
    const int L = (H + K - 1) / K;
    const int t = threadIdx.x, k = t / pairs, j = t - (t / pairs) * pairs;
    const bool act = k < K;
    const bool two = 2 * j + 1 < D;  // else the pair's second channel is the zero pad
    const int y0 = min(k * L, H), y1 = min(y0 + L, H);
    const float scale = pow2f(st->box_exp);
    const long long grow = (long long)W * gs;  // floats per grid row
    const float* g = gr.G + (long long)x * gs + 2 * j;
    // read-only loads (the grid is not written by this launch), so they can
    // be issued ahead of the stores of phase 3
    auto q2 = [&](int y) {
        const float2 f = __ldg(reinterpret_cast<const float2*>(g + (long long)y * grow));
        return make_longlong2(__float2ll_rn(__fmul_rn(f.x, scale)),
                              two ? __float2ll_rn(__fmul_rn(f.y, scale)) : 0LL);
    };
    long long s0 = 0, s1 = 0;
    if (act) {
        int y = y0;
        for (; y + 4 <= y1; y += 4) {
            const longlong2 a = q2(y), b = q2(y + 1), c = q2(y + 2), e = q2(y + 3);
            s0 += a.x + b.x + c.x + e.x;
            s1 += a.y + b.y + c.y + e.y;
        }
        for (; y < y1; ++y) {
            const longlong2 a = q2(y);
            s0 += a.x;
            s1 += a.y;
        }
    }
    tot[t] = make_longlong2(s0, s1);
    __syncthreads();
    if (t < pairs) {
        long long r0 = 0, r1 = 0;
        for (int kk = 0; kk < K; ++kk) {
            const longlong2 v = tot[kk * pairs + t];
            tot[kk * pairs + t] = make_longlong2(r0, r1);
            r0 += v.x;
            r1 += v.y;
        }
    }
    __syncthreads();
    if (act) {
        long long r0 = tot[t].x, r1 = tot[t].y;
        longlong2* p = reinterpret_cast<longlong2*>(gr.sat) + (long long)x * pairs + j;
        const long long row = (long long)W * pairs;  // longlong2 per row
        int y = y0;
        for (; y + 4 <= y1; y += 4) {
            longlong2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = q2(y + u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                r0 += v[u].x;
                r1 += v[u].y;
                p[(long long)(y + u) * row] = make_longlong2(r0, r1);
            }
        }
        for (; y < y1; ++y) {
            const longlong2 a = q2(y);
            r0 += a.x;
            r1 += a.y;
            p[(long long)y * row] = make_longlong2(r0, r1);
        }
    }
}

// one CTA per (row y, channel pair j): the window's column sums
// V(x) = P(min(y+r, H-1), x) - P(y-r-1, x), their inclusive prefix R along x
// in shared memory (thread t owns cells [t*cpt, (t+1)*cpt); the thread totals
// are scanned with warp shuffles), then per cell S = R(min(x+r, W-1)) -
// R(x-r-1) and the target.  The CTAs of one row's channel pairs are adjacent,
// so the 16-byte loads of one pair share their lines with the others in L2.
__global__ void __launch_bounds__(kRowThreads) box_rows_kernel(const GridRef* __restrict__ grids, int D, int ts) {
    extern __shared__ longlong2 R[];  // W entries
    __shared__ longlong2 wsum[kRowThreads / 32];
    const GridRef& gr = grids[0];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int H = gr.H, W = gr.W, r = lv.r;
    const int pairs = sat_channels(D) / 2;
    const int y = blockIdx.x / pairs, j = blockIdx.x - (blockIdx.x / pairs) * pairs;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int yb = min(y + r, H - 1), ya = y - r - 1;
    const longlong2* P = reinterpret_cast<const longlong2*>(gr.sat);
    const longlong2* pb = P + (long long)yb * W * pairs + j;
    const longlong2* pa = P + (long long)max(ya, 0) * W * pairs + j;
    const int cpt = (W + kRowThreads - 1) / kRowThreads;
    const int c0 = min(t * cpt, W), c1 = min(c0 + cpt, W);
    long long s0 = 0, s1 = 0;
    // four cells at a time: read-only loads first (P is not written by this
    // launch), then the prefix into shared memory
    for (int xb = c0; xb < c1; xb += 4) {
        longlong2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v[u] = make_longlong2(0, 0);
            if (xb + u < c1) {
                v[u] = __ldg(pb + (long long)(xb + u) * pairs);
                if (ya >= 0) {
                    const longlong2 a = __ldg(pa + (long long)(xb + u) * pairs);
                    v[u].x -= a.x;
                    v[u].y -= a.y;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (xb + u < c1) {
                s0 += v[u].x;
                s1 += v[u].y;
                R[xb + u] = make_longlong2(s0, s1);
            }
        }
    }
    // exclusive prefix of the thread totals across the CTA
    long long e0 = s0, e1 = s1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u0 = shfl_up64(e0, o), u1 = shfl_up64(e1, o);
        if (lane >= o) {
            e0 += u0;
            e1 += u1;
        }
    }
    if (lane == 31) wsum[warp] = make_longlong2(e0, e1);
    e0 -= s0;
    e1 -= s1;
    __syncthreads();
    for (int w = 0; w < warp; ++w) {
        e0 += wsum[w].x;
        e1 += wsum[w].y;
    }
    for (int x = c0; x < c1; ++x) {
        longlong2 v = R[x];
        v.x += e0;
        v.y += e1;
        R[x] = v;
    }
    __syncthreads();
    const int ny = yb - max(y - r, 0) + 1;
    const float inv_scale = pow2f(-st->box_exp);
    const bool two = 2 * j + 1 < D;
    // the last pair's CTA also zero-fills the target's pad channels, so that
    // every 32-byte sector of a target line is written in full
    const int pad0 = 2 * pairs, pad1 = j == pairs - 1 ? ts : pad0;
    float* out = gr.T + (long long)y * W * ts;
    for (int x = t; x < W; x += kRowThreads) {
        const int xb = min(x + r, W - 1), xa = x - r - 1;
        longlong2 S = R[xb];
        if (xa >= 0) {
            const longlong2 a = R[xa];
            S.x -= a.x;
            S.y -= a.y;
        }
        const float n = (float)(ny * (xb - max(x - r, 0) + 1));
        float* o = out + (long long)x * ts;
        const float v0 = __fmul_rn(__fdiv_rn(__ll2float_rn(S.x), n), inv_scale);
        const float v1 = two ? __fmul_rn(__fdiv_rn(__ll2float_rn(S.y), n), inv_scale) : 0.0f;
        *reinterpret_cast<float2*>(o + 2 * j) = make_float2(v0, v1);
        for (int c = pad0; c < pad1; c += 2) *reinterpret_cast<float2*>(o + c) = make_float2(0.0f, 0.0f);
    }
    write_group_table(gr, lv, st, blockIdx.x, gridDim.x, kRowThreads);
}

// One CTA per row with all channel pairs (rows whose prefix fits in shared
// memory, D <= 16): thread t owns cells [t*cpt, (t+1)*cpt).  It loads the
// cells' P lines (16 B per pair, contiguous per cell, so a warp reads whole
// lines), forms V = P(yb) - P(ya) and its running prefix per channel, the
// CTA scans the thread totals (warp shuffles, then one warp over the warp
// totals), and the prefix R goes to shared memory.  Each cell then reads
// R(min(x+r, W-1)) - R(x-r-1) for every pair and writes its whole target
// line, pad channels included, as 16-byte stores.
constexpr int kRowCtaThreads = 512;
constexpr int kRowCtaMaxBytes = 200 * 1024;  // the row prefix of every pair

template <int PAIRS>
__global__ void __launch_bounds__(kRowCtaThreads, 1) box_rowcta_kernel(const GridRef* __restrict__ grids, int D,
                                                                       int ts) {
    extern __shared__ longlong2 R[];  // W x PAIRS
    __shared__ long long wtot[kRowCtaThreads / 32][2 * PAIRS];
    const GridRef& gr = grids[0];
    const DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int H = gr.H, W = gr.W, r = lv.r;
    const int y = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int yb = min(y + r, H - 1), ya = y - r - 1;
    const longlong2* P = reinterpret_cast<const longlong2*>(gr.sat);
    const longlong2* pb = P + (long long)yb * W * PAIRS;
    const longlong2* pa = P + (long long)max(ya, 0) * W * PAIRS;
    const int cpt = (W + kRowCtaThreads - 1) / kRowCtaThreads;
    const int c0 = min(t * cpt, W), c1 = min(c0 + cpt, W);
    long long s[2 * PAIRS];
#pragma unroll
    for (int c = 0; c < 2 * PAIRS; ++c) s[c] = 0;
    for (int x = c0; x < c1; ++x) {
        longlong2 v[PAIRS];
#pragma unroll
        for (int j = 0; j < PAIRS; ++j) v[j] = __ldg(pb + (long long)x * PAIRS + j);
        if (ya >= 0) {
#pragma unroll
            for (int j = 0; j < PAIRS; ++j) {
                const longlong2 a = __ldg(pa + (long long)x * PAIRS + j);
                v[j].x -= a.x;
                v[j].y -= a.y;
            }
        }
#pragma unroll
        for (int j = 0; j < PAIRS; ++j) {
            s[2 * j] += v[j].x;
            s[2 * j + 1] += v[j].y;
            R[(long long)x * PAIRS + j] = make_longlong2(s[2 * j], s[2 * j + 1]);
        }
    }
    // exclusive prefix of the thread totals: within the warp, then over warps
    long long e[2 * PAIRS];
#pragma unroll
    for (int c = 0; c < 2 * PAIRS; ++c) {
        long long v = s[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = shfl_up64(v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wtot[warp][c] = v;
        e[c] = v - s[c];
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = kRowCtaThreads / 32;
#pragma unroll
        for (int c = 0; c < 2 * PAIRS; ++c) {
            const long long w0 = lane < NW ? wtot[lane][c] : 0LL;
            long long v = w0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = shfl_up64(v, o);
                if (lane >= o) v += u;
            }
            if (lane < NW) wtot[lane][c] = v - w0;  // exclusive over the warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 2 * PAIRS; ++c) e[c] += wtot[warp][c];
    for (int x = c0; x < c1; ++x) {
#pragma unroll
        for (int j = 0; j < PAIRS; ++j) {
            longlong2 v = R[(long long)x * PAIRS + j];
            v.x += e[2 * j];
            v.y += e[2 * j + 1];
            R[(long long)x * PAIRS + j] = v;
        }
    }
    __syncthreads();
    const int ny = yb - max(y - r, 0) + 1;
    const float inv_scale = pow2f(-st->box_exp);
    float* out = gr.T + (long long)y * W * ts;
    for (int x = t; x < W; x += kRowCtaThreads) {
        const int xb = min(x + r, W - 1), xa = x - r - 1;
        const float n = (float)(ny * (xb - max(x - r, 0) + 1));
        // the target line: TSP = round_up(D, 4) floats for D = 2 PAIRS - 1 or
        // 2 PAIRS (ts == TSP, checked by the launcher)
        constexpr int TSP = (2 * PAIRS + 3) & ~3;
        float v[TSP];
#pragma unroll
        for (int c = 0; c < TSP; ++c) v[c] = 0.0f;
#pragma unroll
        for (int j = 0; j < PAIRS; ++j) {
            longlong2 S = R[(long long)xb * PAIRS + j];
            if (xa >= 0) {
                const longlong2 a = R[(long long)xa * PAIRS + j];
                S.x -= a.x;
                S.y -= a.y;
            }
            v[2 * j] = __fmul_rn(__fdiv_rn(__ll2float_rn(S.x), n), inv_scale);
            if (2 * j + 1 < D) v[2 * j + 1] = __fmul_rn(__fdiv_rn(__ll2float_rn(S.y), n), inv_scale);
        }
        float4* o = reinterpret_cast<float4*>(out + (long long)x * TSP);
#pragma unroll
        for (int k = 0; k < TSP / 4; ++k) o[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    write_group_table(gr, lv, st, blockIdx.x, gridDim.x, kRowCtaThreads);
}

template <int PAIRS>
void launch_rowcta_t(const GridRef* grid, int H, int W, int D, cudaStream_t s) {
    const size_t smem = sizeof(longlong2) * (size_t)W * PAIRS;
    box_rowcta_kernel<PAIRS><<<(unsigned)H, kRowCtaThreads, smem, s>>>(grid, D, target_stride(D));
}

// true if a row-per-CTA launch was made (D <= 16 and the row prefix fits)
bool launch_rowcta(const GridRef* grid, int H, int W, int D, cudaStream_t s) {
    const int pairs = sat_channels(D) / 2;
    if (pairs > 8 || (size_t)W * pairs * sizeof(longlong2) > (size_t)kRowCtaMaxBytes) return false;
    if (target_stride(D) != ((2 * pairs + 3) & ~3)) return false;  // holds for every D
    switch (pairs) {
        case 1: launch_rowcta_t<1>(grid, H, W, D, s); break;
        case 2: launch_rowcta_t<2>(grid, H, W, D, s); break;
        case 3: launch_rowcta_t<3>(grid, H, W, D, s); break;
        case 4: launch_rowcta_t<4>(grid, H, W, D, s); break;
        case 5: launch_rowcta_t<5>(grid, H, W, D, s); break;
        case 6: launch_rowcta_t<6>(grid, H, W, D, s); break;
        case 7: launch_rowcta_t<7>(grid, H, W, D, s); break;
        default: launch_rowcta_t<8>(grid, H, W, D, s); break;
    }
    return true;
}

template <int D>
void launch_rowscan_t(const GridRef* grid, int H, cudaStream_t s) {
    box_rowscan_kernel<D><<<(unsigned)H, kScanThreads, 0, s>>>(grid);
}

void launch_rowscan(const GridRef* grid, int H, int D, cudaStream_t s) {
    switch (D) {
        case 1: launch_rowscan_t<1>(grid, H, s); break;
        case 2: launch_rowscan_t<2>(grid, H, s); break;
        case 3: launch_rowscan_t<3>(grid, H, s); break;
        case 4: launch_rowscan_t<4>(grid, H, s); break;
        case 5: launch_rowscan_t<5>(grid, H, s); break;
        case 6: launch_rowscan_t<6>(grid, H, s); break;
        case 7: launch_rowscan_t<7>(grid, H, s); break;
        case 8: launch_rowscan_t<8>(grid, H, s); break;
        case 9: launch_rowscan_t<9>(grid, H, s); break;
        case 10: launch_rowscan_t<10>(grid, H, s); break;
        case 11: launch_rowscan_t<11>(grid, H, s); break;
        case 12: launch_rowscan_t<12>(grid, H, s); break;
        case 13: launch_rowscan_t<13>(grid, H, s); break;
        case 14: launch_rowscan_t<14>(grid, H, s); break;
        case 15: launch_rowscan_t<15>(grid, H, s); break;
        case 16: launch_rowscan_t<16>(grid, H, s); break;
        case 20: launch_rowscan_t<20>(grid, H, s); break;
        case 24: launch_rowscan_t<24>(grid, H, s); break;
        case 32: launch_rowscan_t<32>(grid, H, s); break;
        case 48: launch_rowscan_t<48>(grid, H, s); break;
        default: launch_rowscan_t<64>(grid, H, s); break;
    }
}

}  // namespace

void prepare_box_launches() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(box_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(longlong2) * kRowsMaxW));
    cudaFuncSetAttribute(box_rowcta_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    cudaFuncSetAttribute(box_rowcta_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowCtaMaxBytes);
    done[dev] = true;
}

void launch_box_target(const GridRef* grid, int H, int W, int D, int num_sms, cudaStream_t s) {
    const int pairs = sat_channels(D) / 2;
    if (W <= kRowsMaxW) {
        prepare_box_launches();
        box_colprefix_kernel<<<(unsigned)W, kScanThreads, 0, s>>>(grid, D, grid_stride(D));
        if (!launch_rowcta(grid, H, W, D, s))
            box_rows_kernel<<<(unsigned)((long long)H * pairs), kRowThreads, sizeof(longlong2) * (size_t)W, s>>>(
                grid, D, target_stride(D));
        return;
    }
    launch_rowscan(grid, H, D, s);                                          // one CTA per row
    box_colscan_kernel<<<(unsigned)W, kScanThreads, 0, s>>>(grid, sat_channels(D));  // per cell column
    const long long total = (long long)H * W * pairs;
    const unsigned blocks = (unsigned)std::min<long long>((total + kEvalThreads - 1) / kEvalThreads,
                                                          (long long)num_sms * 8);
    box_eval_kernel<<<blocks, kEvalThreads, 0, s>>>(grid, D, target_stride(D));
}

}  // namespace plas
