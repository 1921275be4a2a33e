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

#include "sweep_bodies.cuh"

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
template <int D, bool CHECKED>
__global__ void __launch_bounds__(kAssignThreads, 4) assign_kernel(
    const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, double tol) {
    assign_body<D, true, CHECKED>(grids, resolve_cta(map), tol);
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
                            bool checked, cudaStream_t s) {
    if (checked)
        assign_kernel<D, true><<<ctas, kAssignThreads, 0, s>>>(grids, map, tol);
    else
        assign_kernel<D, false><<<ctas, kAssignThreads, 0, s>>>(grids, map, tol);
}

void launch_assign(const GridRef* grids, const CtaMap* map, int ctas, int D, double tol,
                   cudaStream_t s, bool checked) {
    if (ctas <= 0) return;
    switch (D) {
#define PLAS_CASE(d) \
    case d: launch_assign_t<d>(grids, map, ctas, tol, checked, s); break;
        PLAS_CASE(1) PLAS_CASE(2) PLAS_CASE(3) PLAS_CASE(4) PLAS_CASE(5) PLAS_CASE(6)
        PLAS_CASE(7) PLAS_CASE(8) PLAS_CASE(9) PLAS_CASE(10) PLAS_CASE(11) PLAS_CASE(12)
        PLAS_CASE(13) PLAS_CASE(14) PLAS_CASE(15) PLAS_CASE(16) PLAS_CASE(20) PLAS_CASE(24)
        PLAS_CASE(32) PLAS_CASE(48) PLAS_CASE(64)
#undef PLAS_CASE
        default: break;  // the API only admits the instantiated channel counts
    }
}

}  // namespace plas
