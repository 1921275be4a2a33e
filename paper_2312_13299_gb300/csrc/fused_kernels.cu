// fused_kernels.cu -- both passes of the low-pass target of the PLAS sort
// (Sec. 3.1 of Morgenstern et al., arXiv 2312.13299: a separable Gaussian
// blur of the grid, renormalised at the border) in one launch, for small
// radii (r <= kFusedMaxR) and up to 16 channels.
//
// A CTA owns a tile of 16 x 32 cells of the target.  Phase 1 runs the pass
// along y for the tile's rows and for its cells widened by the radius on
// both sides (the halo the pass along x needs), reading the working grid
// straight from global memory, and keeps the result (H1) in shared memory;
// phase 2 runs the pass along x out of shared memory and writes the target.
// H1 never goes to global memory.
//
// Each output's FMA chain runs over the taps k_{-r} .. k_r in ascending
// order, as in the oracle; inputs beyond the border enter as zeros, which
// leave the chain unchanged, so the in-range terms are the oracle's terms in
// the oracle's order.  Each pass ends with the correctly rounded division by
// the border tap mass (div_rn), as in the two-pass kernels, so the target is
// bit-identical to them and to the oracle.  The radius is a compile-time
// constant of the chains: the kernel for radii up to RMAX switches on the
// level's radius (which only shrinks during a sort) to the matching chain.
// Lanes work on channel pairs (packed fma.rn.f32x2, two independent IEEE
// FMAs); with an odd D the second channel of the last pair is the grid's
// index column, which is computed alongside and never stored.
#include "sweep_bodies.cuh"

namespace plas {

constexpr int kFusedTY = 16, kFusedTX = 32, kFusedThreads = 256;

int fused_ctas(int H, int W) {
    return ((W + kFusedTX - 1) / kFusedTX) * ((H + kFusedTY - 1) / kFusedTY);
}

static size_t fused_smem(int D, int rmax) {
    const int P = (D + 1) / 2;
    return sizeof(float2) * (size_t)kFusedTY * (size_t)(kFusedTX + 2 * rmax) * (size_t)P;
}

// Phase 1 for radius R along y: H1 of the tile's rows for every halo cell and
// channel pair, into shared memory ([row][cell][pair], nch * P float2 a row).
template <int R>
__device__ __forceinline__ void fused_pass_y(const GridRef& gr, const LevelDesc& lv, int x0, int y0,
                                             int rx, int P, int nch, int gs, float2* h1s) {
    constexpr int X = kFirX, NR = X + 2 * R;
    const int H = gr.H, W = gr.W;
    const int rs = nch * P;
    const float2* __restrict__ tp = reinterpret_cast<const float2*>(gr.table + lv.off_ty);
    const float* __restrict__ nrm = gr.table + lv.off_ny;
    const float* __restrict__ rcp = nrm + ((H + 3) & ~3);
    const long long in_row = (long long)W * gs;
    const int nu = (kFusedTY / X) * rs;
    for (int u = threadIdx.x; u < nu; u += kFusedThreads) {
        const int b = u / rs, cp = u - b * rs;  // cp = cell * P + pair
        const int ch = cp / P, p = cp - ch * P;
        const int x = x0 - rx + ch, ylo = y0 + X * b;
        float2* dst = h1s + (X * b) * rs + cp;
        if (x < 0 || x >= W || ylo >= H) {  // halo beyond the grid: zeros
#pragma unroll
            for (int i = 0; i < X; ++i) dst[i * rs] = make_float2(0.0f, 0.0f);
            continue;
        }
        const float* col = gr.G + (long long)x * gs + 2 * p;
        float2 w[NR];
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            const int yy = ylo - R + m;
            w[m] = (yy >= 0 && yy < H) ? __ldg(reinterpret_cast<const float2*>(col + (long long)yy * in_row))
                                       : make_float2(0.0f, 0.0f);
        }
        float2 acc[X];
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) {  // tap j - R, stored at pair index j
            const float2 k = __ldg(tp + j);
#pragma unroll
            for (int i = 0; i < X; ++i) acc[i] = __ffma2_rn(k, w[i + j], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < X; ++i) {
            const int y = ylo + i;
            if (y < H) {
                const float n = nrm[y], q = rcp[y];
                dst[i * rs] = make_float2(div_rn(acc[i].x, n, q), div_rn(acc[i].y, n, q));
            }
        }
    }
}

// Phase 2 for radius R along x: the target of the tile from shared H1.
template <int R>
__device__ __forceinline__ void fused_pass_x(const GridRef& gr, const LevelDesc& lv, int x0, int y0,
                                             int P, int nch, int D, int ts, const float2* h1s) {
    constexpr int X = kFirX, NR = X + 2 * R;
    const int H = gr.H, W = gr.W;
    const int rs = nch * P;
    const float2* __restrict__ tp = reinterpret_cast<const float2*>(gr.table + lv.off_tx);
    const float* __restrict__ nrm = gr.table + lv.off_nx;
    const float* __restrict__ rcp = nrm + ((W + 3) & ~3);
    const int per_block = kFusedTY * P;
    const int nu = (kFusedTX / X) * per_block;
    const bool even_d = (D & 1) == 0;
    for (int v = threadIdx.x; v < nu; v += kFusedThreads) {
        const int cb = v / per_block, ip = v - cb * per_block;
        const int i = ip / P, p = ip - i * P;
        const int y = y0 + i, xlo = x0 + X * cb;
        if (y >= H || xlo >= W) continue;
        // window cell m is x = xlo - R + m: halo index X * cb + m (in the halo)
        const float2* row = h1s + i * rs + (X * cb) * P + p;
        float2 w[NR];
#pragma unroll
        for (int m = 0; m < NR; ++m) w[m] = row[m * P];
        float2 acc[X];
#pragma unroll
        for (int k = 0; k < X; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) {
            const float2 k2 = __ldg(tp + j);
#pragma unroll
            for (int k = 0; k < X; ++k) acc[k] = __ffma2_rn(k2, w[k + j], acc[k]);
        }
        float* out = gr.T + ((long long)y * W + xlo) * ts + 2 * p;
        const bool pair = even_d || p + 1 < P;
#pragma unroll
        for (int k = 0; k < X; ++k) {
            const int x = xlo + k;
            if (x < W) {
                const float n = nrm[x], q = rcp[x];
                const float a = div_rn(acc[k].x, n, q);
                if (pair)
                    *reinterpret_cast<float2*>(out + k * ts) = make_float2(a, div_rn(acc[k].y, n, q));
                else
                    out[k * ts] = a;
            }
        }
    }
}

// The chains for the level's radius r (0 .. RMAX; the host plans the launch
// for a radius <= RMAX, and radii only shrink during a sort).
template <int R, int RMAX>
__device__ __forceinline__ void fused_y_at(int r, const GridRef& gr, const LevelDesc& lv, int x0, int y0,
                                           int rx, int P, int nch, int gs, float2* h1s) {
    if constexpr (R <= RMAX) {
        if (r == R)
            fused_pass_y<R>(gr, lv, x0, y0, rx, P, nch, gs, h1s);
        else
            fused_y_at<R + 1, RMAX>(r, gr, lv, x0, y0, rx, P, nch, gs, h1s);
    }
}
template <int R, int RMAX>
__device__ __forceinline__ void fused_x_at(int r, const GridRef& gr, const LevelDesc& lv, int x0, int y0,
                                           int P, int nch, int D, int ts, const float2* h1s) {
    if constexpr (R <= RMAX) {
        if (r == R)
            fused_pass_x<R>(gr, lv, x0, y0, P, nch, D, ts, h1s);
        else
            fused_x_at<R + 1, RMAX>(r, gr, lv, x0, y0, P, nch, D, ts, h1s);
    }
}

// Registers per thread budget: the radius group's window (8 + 2 RMAX channel
// pairs) plus 8 accumulator pairs.
template <int RMAX>
__global__ void __launch_bounds__(kFusedThreads, RMAX <= 3 ? 3 : 2) fir_fused_kernel(
    const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, int D, int gs, int ts) {
    extern __shared__ __align__(16) float2 h1s[];  // [kFusedTY][nch][P]
    const CtaRef cr = resolve_cta(map);
    const GridRef& gr = grids[cr.g];
    DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int ry = lv.ry, rx = lv.rx;
    if (ry > RMAX || rx > RMAX) {  // planned for smaller radii only: record, touch nothing
        if (threadIdx.x == 0) atomicCAS(&st->status, 0, -7);  // PLAS_ERR_INTERNAL
        return;
    }
    const int P = (D + 1) >> 1;
    const int ntx = (gr.W + kFusedTX - 1) / kFusedTX;
    const int x0 = (cr.local % ntx) * kFusedTX, y0 = (cr.local / ntx) * kFusedTY;
    const int nch = kFusedTX + 2 * rx;  // tile cells plus the halo along x
    fused_y_at<0, RMAX>(ry, gr, lv, x0, y0, rx, P, nch, gs, h1s);
    __syncthreads();
    fused_x_at<0, RMAX>(rx, gr, lv, x0, y0, P, nch, D, ts, h1s);
    // the iteration's grouping table (the pass along y writes it in the
    // two-pass path)
    write_group_table(gr, lv, st, cr.local, cr.count, kFusedThreads);
    // tell the schedule step which launch ran the pass along x (work counts)
    if (cr.local == 0 && threadIdx.x == 0) st->fused_pending = 1;
}

void prepare_fused_launches() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(fir_fused_kernel<kFusedGroupMaxR[0]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem(kFusedMaxD, kFusedGroupMaxR[0]));
    cudaFuncSetAttribute(fir_fused_kernel<kFusedGroupMaxR[1]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem(kFusedMaxD, kFusedGroupMaxR[1]));
    cudaFuncSetAttribute(fir_fused_kernel<kFusedGroupMaxR[2]>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem(kFusedMaxD, kFusedGroupMaxR[2]));
    done[dev] = true;
}

void launch_fir_fused(const GridRef* grids, const CtaMap* map, int ctas, int D, int group,
                      cudaStream_t s) {
    if (ctas <= 0 || D > kFusedMaxD || group < 0 || group >= kFusedGroups) return;
    prepare_fused_launches();
    const int gs = grid_stride(D), ts = target_stride(D);
    const size_t sm = fused_smem(D, kFusedGroupMaxR[group]);
    if (group == 0)
        fir_fused_kernel<kFusedGroupMaxR[0]><<<ctas, kFusedThreads, sm, s>>>(grids, map, D, gs, ts);
    else if (group == 1)
        fir_fused_kernel<kFusedGroupMaxR[1]><<<ctas, kFusedThreads, sm, s>>>(grids, map, D, gs, ts);
    else
        fir_fused_kernel<kFusedGroupMaxR[2]><<<ctas, kFusedThreads, sm, s>>>(grids, map, D, gs, ts);
}

}  // namespace plas
