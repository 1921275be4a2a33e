// fused_kernels.cu -- both passes of the low-pass target of the PLAS sort
// (Sec. 3.1 of Morgenstern et al., arXiv 2312.13299: a separable Gaussian
// blur of the grid, renormalised at the border) in one launch, for small
// radii (r <= kFusedMaxR) and up to 16 channels.
//
// A CTA owns a tile of 32 x 32 cells of the target.  Phase 1 runs the pass
// along y for the tile's rows and for its cells widened by the radius on
// both sides (the halo the pass along x needs), reading the working grid
// straight from global memory, and keeps the result (H1) in shared memory;
// phase 2 runs the pass along x out of shared memory and writes the target.
// H1 never goes to global memory, and the grid is read once per tile.
//
// The chains are those of the two-pass kernels: every output's FMA chain
// runs over the same tap steps (the step range of its aligned block of 8
// outputs, zero taps and zero rows beyond the border included, in ascending
// order), and each pass ends with the same correctly rounded division by the
// border tap mass, so the target is bit-identical to the two-pass path.
// Lanes work on channel pairs (packed fma.rn.f32x2, two independent IEEE
// FMAs); with an odd D the second channel of the last pair is the grid's
// index column, which is computed alongside and never stored.
#include "sweep_bodies.cuh"

namespace plas {

constexpr int kFusedTY = 32, kFusedTX = 32, kFusedThreads = 256;

size_t fused_smem_bytes(int D) {
    const int P = (D + 1) / 2;
    return sizeof(float2) * (size_t)kFusedTY * (size_t)(kFusedTX + 2 * kFusedMaxR) * (size_t)P;
}

int fused_ctas(int H, int W) {
    return ((W + kFusedTX - 1) / kFusedTX) * ((H + kFusedTY - 1) / kFusedTY);
}

// Pass along y for one channel pair of one cell and 8 output rows: NR window
// rows of the grid (column pointer col, row stride in_row; zero outside
// [0, H)), NB blocks of 8 tap steps from tp.
template <int NB>
__device__ __forceinline__ void chain_grid(const float* __restrict__ col, long long in_row, int H,
                                           int base, const float2* __restrict__ tp,
                                           float2 (&acc)[kFirX]) {
    constexpr int X = kFirX, NR = NB * X + X - 1;
    float2 w[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        const int yy = base + m;
        w[m] = (yy >= 0 && yy < H) ? __ldg(reinterpret_cast<const float2*>(col + (long long)yy * in_row))
                                   : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int s = 0; s < NB * X; ++s) {
        const float2 k = __ldg(tp + s);
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i] = __ffma2_rn(k, w[s + i], acc[i]);
    }
}

// Pass along x for one channel pair of one row and 8 output cells: NR window
// cells of the shared H1 row (stride P float2 per cell; zero outside
// [0, nch)).
template <int NB>
__device__ __forceinline__ void chain_shared(const float2* row, int P, int nch, int base,
                                             const float2* __restrict__ tp, float2 (&acc)[kFirX]) {
    constexpr int X = kFirX, NR = NB * X + X - 1;
    float2 w[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        const int c = base + m;
        w[m] = (c >= 0 && c < nch) ? row[c * P] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int s = 0; s < NB * X; ++s) {
        const float2 k = __ldg(tp + s);
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i] = __ffma2_rn(k, w[s + i], acc[i]);
    }
}

// Tap-step range [wlo, wend) of the aligned block of 8 outputs starting at
// position lo on an axis of length len (the same rule as the two-pass
// kernels): steps with a non-zero tap that reach an in-range input for some
// output of the block, widened to whole blocks of 8.
__device__ __forceinline__ void block_steps(int lo, int len, int r, int rp, int ntp, int* wlo,
                                            int* nb) {
    const int hi = min(lo + kFirX, len) - 1;
    int a = max(rp - r, rp - hi);
    a = a / kFirX * kFirX;
    const int b = min(rp + r, rp + len - 1 - lo);
    const int e = min(ntp, (b + kFirX) / kFirX * kFirX);
    *wlo = a;
    *nb = (e - a) / kFirX;
}

__global__ void __launch_bounds__(kFusedThreads, 2) fir_fused_kernel(
    const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, int D, int gs, int ts) {
    constexpr int X = kFirX;
    extern __shared__ __align__(16) float2 h1s[];  // [kFusedTY][nch][P]
    const CtaRef cr = resolve_cta(map);
    const GridRef& gr = grids[cr.g];
    DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int H = gr.H, W = gr.W;
    const int ry = lv.ry, rpy = lv.rpy, ntpy = lv.ntpy;
    const int rx = lv.rx, rpx = lv.rpx, ntpx = lv.ntpx;
    if (ry > kFusedMaxR || rx > kFusedMaxR) {  // the host plans this launch for small radii only
        if (threadIdx.x == 0) atomicCAS(&st->status, 0, -7);  // PLAS_ERR_INTERNAL
        return;
    }
    const int P = (D + 1) >> 1;
    const int ntx = (W + kFusedTX - 1) / kFusedTX;
    const int x0 = (cr.local % ntx) * kFusedTX, y0 = (cr.local / ntx) * kFusedTY;
    const int nch = kFusedTX + 2 * rx;  // tile cells plus the halo along x
    const int rs = nch * P;             // float2 per H1 row in shared memory

    // ---- phase 1: pass along y into shared memory ----
    {
        const float2* tp = reinterpret_cast<const float2*>(gr.table + lv.off_ty);
        const float* nrm = gr.table + lv.off_ny;
        const float* rcp = nrm + ((H + 3) & ~3);
        const long long in_row = (long long)W * gs;
        const int nu = (kFusedTY / X) * rs;
        for (int u = threadIdx.x; u < nu; u += kFusedThreads) {
            const int b = u / rs, cp = u - b * rs;  // cp = ch * P + p
            const int ch = cp / P, p = cp - ch * P;
            const int x = x0 - rx + ch, ylo = y0 + X * b;
            float2* dst = h1s + (X * b) * rs + cp;
            if (x < 0 || x >= W || ylo >= H) {  // halo beyond the grid: zeros
#pragma unroll
                for (int i = 0; i < X; ++i) dst[i * rs] = make_float2(0.0f, 0.0f);
                continue;
            }
            int wlo, nb;
            block_steps(ylo, H, ry, rpy, ntpy, &wlo, &nb);
            float2 acc[X];
#pragma unroll
            for (int i = 0; i < X; ++i) acc[i] = make_float2(0.0f, 0.0f);
            const float* col = gr.G + (long long)x * gs + 2 * p;
            const int base = ylo - rpy + wlo;
            if (nb == 1) chain_grid<1>(col, in_row, H, base, tp + wlo, acc);
            else if (nb == 2) chain_grid<2>(col, in_row, H, base, tp + wlo, acc);
            else chain_grid<3>(col, in_row, H, base, tp + wlo, acc);
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
    __syncthreads();

    // ---- phase 2: pass along x from shared memory into the target ----
    {
        const float2* tp = reinterpret_cast<const float2*>(gr.table + lv.off_tx);
        const float* nrm = gr.table + lv.off_nx;
        const float* rcp = nrm + ((W + 3) & ~3);
        const int per_block = kFusedTY * P;  // units of one block of 8 cells (whole warps)
        const int nu = (kFusedTX / X) * per_block;
        for (int v = threadIdx.x; v < nu; v += kFusedThreads) {
            const int cb = v / per_block, ip = v - cb * per_block;
            const int i = ip / P, p = ip - i * P;
            const int y = y0 + i, xlo = x0 + X * cb;
            if (y >= H || xlo >= W) continue;
            int wlo, nb;
            block_steps(xlo, W, rx, rpx, ntpx, &wlo, &nb);
            float2 acc[X];
#pragma unroll
            for (int k = 0; k < X; ++k) acc[k] = make_float2(0.0f, 0.0f);
            // window cell m is x = xlo - rpx + wlo + m, halo index x - (x0 - rx)
            const float2* row = h1s + i * rs + p;
            const int base = X * cb - rpx + wlo + rx;
            if (nb == 1) chain_shared<1>(row, P, nch, base, tp + wlo, acc);
            else if (nb == 2) chain_shared<2>(row, P, nch, base, tp + wlo, acc);
            else chain_shared<3>(row, P, nch, base, tp + wlo, acc);
            float* out = gr.T + ((long long)y * W + xlo) * ts + 2 * p;
            const bool pair = 2 * p + 1 < D;
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
    cudaFuncSetAttribute(fir_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem_bytes(kFusedMaxD));
    done[dev] = true;
}

void launch_fir_fused(const GridRef* grids, const CtaMap* map, int ctas, int D, cudaStream_t s) {
    if (ctas <= 0 || D > kFusedMaxD) return;
    prepare_fused_launches();
    fir_fused_kernel<<<ctas, kFusedThreads, fused_smem_bytes(D), s>>>(grids, map, D, grid_stride(D),
                                                                       target_stride(D));
}

}  // namespace plas
