// sort_kernels.cu -- the per-iteration kernels of the PLAS grid sort (Sec. 3.1
// of Morgenstern et al., arXiv 2312.13299): grouping permutation, the two
// passes of the low-pass target, and the 24-permutation assignment with the
// convergence test.  Each launch is a sweep over a list of grids: a CTA looks
// up its grid (and that grid's current radius level in device memory), so one
// grid or many are advanced by the same kernels.
//
// Floating-point contract (shared with the CPU oracle by specification, not by
// code): every multiply-add is a round-to-nearest FMA (scalar __fmaf_rn or the
// packed fma.rn.f32x2, which performs two independent IEEE FMAs), every other
// operation an explicit round-to-nearest intrinsic, sums run in ascending tap
// / channel order, and the only reduction that feeds a decision (the mean L2
// distance of the schedule) is an exact integer sum.  The library is built
// with -fmad=false so the compiler contracts nothing on its own.
#include <algorithm>
#include <cstdio>

#include "plas_kernels.h"

namespace plas {

// ============================================================================
// assignment (Sec. 3.1 "Blockwise Linear Assignment", Fig. "swapping_pixels"):
// a quad of lanes per group of four cells.  Lane i loads the feature row of
// cell p_i and the four target rows (the four lanes of a quad load the same
// target rows in one instruction) and forms row i of the 4x4 cost matrix
// C[i][j] = sum_d (G[p_i]_d - T[p_j]_d)^2; the quad all-gathers the matrix and
// every lane scores all 24 permutations in lexicographic order, keeping the
// first strict minimum.  Lane i then writes its row to p_sigma(i) (groups are
// disjoint, so the swap is in place).  The distance of every cell to the
// target after the swap is added to an exact fixed-point sum; the last CTA of
// the grid to finish runs the schedule step (Sec. 3.1).
// ============================================================================
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

// Schedule step (Sec. 3.1): d = mean L2 distance to the target; an assignment
// that improves d by less than tol (relative) is a stall; one stall draws a
// new block shift, a second in a row shrinks the radius; the sort ends when
// the radius falls below phi_min (no levels left).
__device__ void schedule_step(DevState* st, long long N, int nby, int nbx, int ngroups,
                              int nlevels, double tol, long long* trace_S, int* trace_level,
                              long long trace_cap, double fmas_y, double fmas_x, double beta2) {
    st->fmas_y += fmas_y;
    st->fmas_x += fmas_x;
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
    st->grouped += (long long)nby * nbx * ngroups * 4;
    if (st->level >= nlevels) st->done = 1;
    st->S = 0ull;
    st->arrivals = 0u;
    __threadfence();
}

template <int D>
__global__ void __launch_bounds__(kAssignThreads, 4) assign_kernel(
    const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, double tol) {
    constexpr int GS = (D + 1 + 3) & ~3, TS = (D + 3) & ~3;
    __shared__ unsigned long long s_part[kAssignThreads / 32];
    const CtaRef cr = resolve_cta(map);
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
    const int nby = (H - dy) / beta, nbx = (W - dx) / beta;
    const int ngroups = (beta * beta) / 4;
    // N <= 2^26 (checked on the host), so every cell and group index fits 32 bits
    const int ngt = nby * nbx * ngroups;
    const float scale = ldexpf(1.0f, st->scale_exp);  // 2^k, 0 <= k <= 32
    float* __restrict__ G = gr.G;
    const float* __restrict__ T = gr.T;
    const uint32_t* __restrict__ pi = gr.pi;
    unsigned long long part = 0ull;

    const int lane = threadIdx.x & 31, qi = lane & 3, qbase = lane & ~3;
    const int gwarp = (cr.local * kAssignThreads + (int)threadIdx.x) >> 5;
    const int nwarps = (cr.count * kAssignThreads) >> 5;
    constexpr Perm24 kPerm24 = make_perm24();
    // ---- groups: 8 per warp ----
    // the grouping-table entries of the next iteration are read one iteration
    // ahead, so each iteration waits for one memory round trip, not two
    auto group_of = [&](int b) -> int {
        const int t = b + (lane >> 2);
        return t < ngt ? (int)((uint32_t)t % (uint32_t)ngroups) : 0;
    };
    uint4 l4_next = make_uint4(0u, 0u, 0u, 0u);
    if (gwarp * 8 < ngt) l4_next = __ldg(reinterpret_cast<const uint4*>(pi) + group_of(gwarp * 8));
    for (int base = gwarp * 8; base < ngt; base += nwarps * 8) {
        const int task0 = base + (lane >> 2);
        const bool active = task0 < ngt;
        const uint32_t task = active ? (uint32_t)task0 : 0u;
        const uint32_t blk = task / (uint32_t)ngroups;
        const int by = (int)(blk / (uint32_t)nbx), bx = (int)(blk - (uint32_t)by * (uint32_t)nbx);
        const int oy = dy + by * beta, ox = dx + bx * beta;
        const uint4 l4 = l4_next;
        if (base + nwarps * 8 < ngt)
            l4_next = __ldg(reinterpret_cast<const uint4*>(pi) + group_of(base + nwarps * 8));
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
        // first strict minimum in lexicographic order, as a pairwise tree:
        // the left operand always holds the earlier permutations and wins
        // ties, so the tree picks the same permutation as a sequential scan.
        // Each node carries its permutation packed as four 2-bit targets.
        float bc[24];
        int bp[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            bc[k] = __fadd_rn(__fadd_rn(__fadd_rn(C[0][kPerm24.p[k][0]], C[1][kPerm24.p[k][1]]),
                                        C[2][kPerm24.p[k][2]]),
                              C[3][kPerm24.p[k][3]]);
            bp[k] = kPerm24.p[k][0] | (kPerm24.p[k][1] << 2) | (kPerm24.p[k][2] << 4) |
                    (kPerm24.p[k][3] << 6);
        }
#pragma unroll
        for (int n = 24; n > 1; n = (n + 1) / 2) {
#pragma unroll
            for (int m = 0; m < n / 2; ++m) {
                const bool right = bc[2 * m + 1] < bc[2 * m];
                bc[m] = right ? bc[2 * m + 1] : bc[2 * m];
                bp[m] = right ? bp[2 * m + 1] : bp[2 * m];
            }
            if (n & 1) {
                bc[n / 2] = bc[n - 1];
                bp[n / 2] = bp[n - 1];
            }
        }
        const int my_dst = (bp[0] >> (2 * qi)) & 3;
        if (active) {
            float4* dst = reinterpret_cast<float4*>(G + (size_t)pick4i(pos, my_dst) * GS);
#pragma unroll
            for (int k = 0; k < GS / 4; ++k)
                dst[k] = make_float4(grow[4 * k], grow[4 * k + 1], grow[4 * k + 2], grow[4 * k + 3]);
            part += fixed_point(__fsqrt_rn(pick4(c, my_dst)), scale);
        }
    }

    // ---- cells outside the full blocks (enumerated directly: the rows above
    // and below the covered band, then the left and right margins of it) ----
    const int cy0 = dy, cy1 = dy + nby * beta, cx0 = dx, cx1 = dx + nbx * beta;
    const int gthread = cr.local * kAssignThreads + (int)threadIdx.x;
    const int nthreads = cr.count * kAssignThreads;
    const int n_top = cy0 * W, n_bot = (H - cy1) * W, margin = W - (cx1 - cx0);
    const int n_unc = n_top + n_bot + (cy1 - cy0) * margin;
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
        load_row4<TS / 4>(T + (size_t)p * TS, trow);
        part += fixed_point(__fsqrt_rn(sqdist<D>(grow, trow)), scale);
    }
    // ---- leftover cells of each block (beta^2 mod 4 of them) ----
    const int nleft = beta * beta - 4 * ngroups;
    const int nl = nby * nbx * nleft;
    for (int e = gthread; e < nl; e += nthreads) {
        const int blk = (int)((uint32_t)e / (uint32_t)nleft);
        const int m = 4 * ngroups + (e - blk * nleft);
        const int by = (int)((uint32_t)blk / (uint32_t)nbx), bx = blk - by * nbx;
        const uint32_t l = pi[m];
        const int ly = (int)(l / (uint32_t)beta), lx = (int)(l - (uint32_t)ly * (uint32_t)beta);
        const int p = (dy + by * beta + ly) * W + (dx + bx * beta + lx);
        float grow[GS], trow[TS];
        load_row4_rw<GS / 4>(G + (size_t)p * GS, grow);
        load_row4<TS / 4>(T + (size_t)p * TS, trow);
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

int assign_ctas(int H, int W, int num_sms, int per_sm) {
    const long long N = (long long)H * W;
    long long need = (N / 4 + 63) / 64;  // one quad per group, 64 groups per CTA
    per_sm = std::min(std::max(per_sm, 1), kAssignMaxPerSm);
    need = std::min<long long>(need, (long long)num_sms * per_sm);
    return (int)std::max<long long>(need, 1);
}

template <int D>
static void launch_assign_t(const GridRef* grids, const CtaMap* map, int ctas, double tol,
                            cudaStream_t s) {
    assign_kernel<D><<<ctas, kAssignThreads, 0, s>>>(grids, map, tol);
}

void launch_assign(const GridRef* grids, const CtaMap* map, int ctas, int D, double tol,
                   cudaStream_t s) {
    if (ctas <= 0) return;
    switch (D) {
#define PLAS_CASE(d) \
    case d: launch_assign_t<d>(grids, map, ctas, tol, s); break;
        PLAS_CASE(1) PLAS_CASE(2) PLAS_CASE(3) PLAS_CASE(4) PLAS_CASE(5) PLAS_CASE(6)
        PLAS_CASE(7) PLAS_CASE(8) PLAS_CASE(9) PLAS_CASE(10) PLAS_CASE(11) PLAS_CASE(12)
        PLAS_CASE(13) PLAS_CASE(14) PLAS_CASE(15) PLAS_CASE(16) PLAS_CASE(20) PLAS_CASE(24)
        PLAS_CASE(32) PLAS_CASE(48) PLAS_CASE(64)
#undef PLAS_CASE
        default: break;  // the API only admits the instantiated channel counts
    }
}

}  // namespace plas
