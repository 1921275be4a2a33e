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
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "sweep_bodies.cuh"

namespace plas {

int num_sms();  // plas_api.cu

template <class TL>
__global__ void __launch_bounds__(TL::THREADS, TL::MINB) fir_kernel(
    int pass, const GridRef* __restrict__ grids, const CtaMap* __restrict__ map, int D, int gs,
    int ts) {
    extern __shared__ __align__(16) ulonglong2 ring[];  // TL::RING x 32 lanes x 4 columns
    fir_ring_body<TL>(pass, grids, resolve_cta(map), D, gs, ts, ring);
}

// ============================================================================
// Persistent tensor-copy ring kernel (the large tiling for single grids of an
// even number of channels).
//
// A CTA of 16 warps walks tiles tile = blockIdx.x, +gridDim.x, ... (128 output
// rows x 128 columns, the same tiles and FMA chains as the chunked kernel).
// Input rows stream through a ring of kTmaStages stages of 8 rows, each stage
// one tensor copy (cp.async.bulk.tensor): along y the box is 8 rows x ncell
// whole cells of G (index and padding included, features picked out by
// offset), along x it is 8 rows x 128 values of H1.  Rows and cells outside
// the grid arrive as zeros.  Each stage completes an mbarrier ("full") by its
// byte count.  Lane l owns the column pairs l and l + 32 (columns
// c0 + 2(l + 32k) and the next; D is even, so a pair never straddles a cell)
// and reads each as one 8-byte shared load; warp q owns output rows
// 8q..8q+7.  At 8-step block b warp q reads stages q+b and q+b+1 of the tile,
// so every warp walks the tile's nb+16 stages in order, waiting for each to
// be full and releasing it ("empty", one arrival per warp) once it no longer
// reads it.  Warp 0 reads each stage last; after each of its releases, its
// lane 0 issues the copy that refills the freed slot 32 stages further on
// (waiting for the other warps' releases of that slot first), so the ring
// runs into the next tile while the warps finish the current one, and no
// CTA-wide barrier interrupts the FMA chains.  The level's taps stay in
// shared memory for the whole launch.
//
// Every wait is bounded: after kWsTimeoutNs without progress the CTA gives
// up, records PLAS_ERR_TIMEOUT in the grid's status word, waits (bounded) for
// its copies in flight and leaves.
// ============================================================================
constexpr int kTmaTY = 128;
constexpr int kTmaWarps = kTmaTY / kFirX;  // 16
constexpr int kTmaThreads = 32 * kTmaWarps;
constexpr int kTmaStages = 32;
constexpr int kTmaSmemMax = 232448;  // dynamic shared memory opt-in per CTA
constexpr unsigned long long kWsTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for phase 'parity' of the mbarrier at shared address bar;
// false once the CTA gives up (after kWsTimeoutNs, or another warp gave up).
__device__ __noinline__ bool tma_wait_slow(unsigned bar, unsigned parity, volatile int* abort) {
    const unsigned long long t0 = global_ns();
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 63u) == 0u) {
            if (*abort) return false;
            if (global_ns() - t0 > kWsTimeoutNs) {
                *abort = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ bool tma_wait(unsigned bar, unsigned parity, volatile int* abort) {
    return mbar_try_wait(bar, parity) || tma_wait_slow(bar, parity, abort);
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void* map, unsigned bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void* map, unsigned bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}

struct TmaParams {
    CUtensorMap map;  // the pass's tensor map
    int pass, ntiles, D, ts, rowf, ncell;
};

// Geometry of a tile: first column, first output row, CTA step range.
struct TmaTile {
    int c0, t0, jlo, jend, nb;
};
__device__ __forceinline__ TmaTile tma_tile(int tile, int ncol, int R, int r, int rp, int ntp) {
    TmaTile t;
    t.c0 = (tile % ncol) * kFirCols;
    t.t0 = (tile / ncol) * kTmaTY;
    const int jlo = max(rp - r, rp - (t.t0 + kTmaTY - 1));
    t.jlo = jlo / kFirX * kFirX;
    const int jhi = min(rp + r, rp + R - 1 - t.t0);
    t.jend = min(ntp, (jhi + kFirX) / kFirX * kFirX);
    t.nb = (t.jend - t.jlo) / kFirX;
    return t;
}

// PASS 1 reads whole 128-value rows of H1: lane l owns columns c0+4l..c0+4l+3
// (one 16-byte shared load per row).  PASS 0 reads rows of ncell whole cells
// of G (ROWF = ncell * gs floats): lane l owns the column pairs l and l+32 of
// the tile (two 8-byte shared loads per row).  Either way acc[i][0] and
// acc[i][1] hold two pairs of adjacent columns of one cell, stored as float2.
template <int PASS, int ROWF>
__global__ void __launch_bounds__(kTmaThreads, 1) fir_tma_kernel(const GridRef* __restrict__ grids,
                                                                 const __grid_constant__ TmaParams P) {
    constexpr int X = kFirX;
    constexpr unsigned kRowBytes = ROWF * 4u, kStageBytes = kRowBytes * X;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const GridRef& gr = grids[0];
    DevState* st = gr.st;
    if (sweep_idle(st)) return;
    const LevelDesc& lv = gr.lv[st->level];
    const int D = P.D, hd = D >> 1;
    const int R = PASS == 0 ? gr.H : gr.W;
    const int NC = PASS == 0 ? gr.W * D : gr.H * D;
    const int r = PASS == 0 ? lv.ry : lv.rx, rp = PASS == 0 ? lv.rpy : lv.rpx;
    const int ntp = PASS == 0 ? lv.ntpy : lv.ntpx;
    const float* taps_g = gr.table + (PASS == 0 ? lv.off_ty : lv.off_tx);
    const int ncol = (NC + kFirCols - 1) / kFirCols;
    // shared memory: ring, taps, barriers, abort flag
    const unsigned ring0 = smem_u32(tsm);
    unsigned long long* taps = reinterpret_cast<unsigned long long*>(tsm + kTmaStages * kStageBytes);
    unsigned char* tail = tsm + kTmaStages * kStageBytes + (((unsigned)ntp * 8u + 127u) & ~127u);
    const unsigned full0 = smem_u32(tail), empty0 = full0 + 8u * kTmaStages;
    volatile int* abort = reinterpret_cast<volatile int*>(tail + 16 * kTmaStages);
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;

    // producer state (thread 0): the next stage to issue
    int p_tile = blockIdx.x, p_k = 0, p_nst = 0, p_x = 0, p_y = 0;
    unsigned pz = 0;
    auto p_begin_tile = [&]() {
        if (p_tile >= P.ntiles) return;
        const TmaTile t = tma_tile(p_tile, ncol, R, r, rp, ntp);
        p_nst = t.nb + kTmaWarps;
        p_k = 0;
        p_x = PASS == 0 ? (t.c0 >> 1) / hd : t.c0;  // first cell (pass 0) or column (pass 1)
        p_y = t.jlo - rp + t.t0;                     // input row of stream row 0
    };
    // issue the next stage (thread 0); false: gave up waiting
    auto issue = [&]() -> bool {
        if (p_tile >= P.ntiles) return true;
        const unsigned slot = pz & (kTmaStages - 1), use = pz / kTmaStages;
        if (use > 0 && !tma_wait(empty0 + 8u * slot, (use - 1) & 1u, abort)) return false;
        const unsigned fb = full0 + 8u * slot, dst = ring0 + slot * kStageBytes;
        mbar_expect_tx(fb, kStageBytes);
        if (PASS == 0)
            tma_load_3d(dst, &P.map, fb, 0, p_x, p_y + X * p_k);
        else
            tma_load_2d(dst, &P.map, fb, p_x, p_y + X * p_k);
        ++pz;
        if (++p_k == p_nst) {
            p_tile += gridDim.x;
            p_begin_tile();
        }
        return true;
    };

    if (threadIdx.x == 0) {
        for (int k = 0; k < kTmaStages; ++k) {
            mbar_init(full0 + 8u * k, 1u);
            mbar_init(empty0 + 8u * k, (unsigned)kTmaWarps);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        p_begin_tile();
        for (int k = 0; k < kTmaStages; ++k) issue();  // no waits: first use of every slot
    }
    // the level's taps, resident for the launch
    {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(taps_g);
        for (int p = threadIdx.x; p < ntp; p += kTmaThreads) taps[p] = src[p];
    }
    __syncthreads();

    const unsigned char* ring = tsm;
    const unsigned dinv = hd > 1 ? (unsigned)((0x100000000ull + (unsigned)hd - 1) / (unsigned)hd) : 0u;
    unsigned z = 0;  // running stage counter, the same sequence as the producer's
    bool ok = true;
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
        const TmaTile t = tma_tile(tile, ncol, R, r, rp, ntp);
        // byte offsets of this lane's columns within a ring row
        unsigned off0, off1;
        if (PASS == 0) {
            const int P0 = t.c0 >> 1;
            const int x0 = hd > 1 ? (int)__umulhi((unsigned)P0, dinv) : P0;
            const int g0 = P0 + lane, g1 = g0 + 32;
            const int c0 = hd > 1 ? (int)__umulhi((unsigned)g0, dinv) : g0;
            const int c1 = hd > 1 ? (int)__umulhi((unsigned)g1, dinv) : g1;
            const int gs = P.rowf / P.ncell;
            off0 = 4u * (unsigned)((c0 - x0) * gs + 2 * (g0 - c0 * hd));
            off1 = 4u * (unsigned)((c1 - x0) * gs + 2 * (g1 - c1 * hd));
        } else {
            off0 = 16u * (unsigned)lane;
            off1 = off0 + 8u;
        }
        const int ylo = t.t0 + q * X;
        int wlo = 0, wend = 0;
        if (ylo < R) {
            const int yhi = min(ylo + X, R) - 1;
            wlo = max(rp - r, rp - yhi);
            wlo = max(t.jlo, wlo / X * X);
            const int whi = min(rp + r, rp + R - 1 - ylo);
            wend = min(t.jend, (whi + X) / X * X);
        }
        const int nb = t.nb;
        auto full_of = [&](int k) { return full0 + 8u * ((z + (unsigned)k) & (kTmaStages - 1)); };
        auto par_of = [&](int k) { return ((z + (unsigned)k) / kTmaStages) & 1u; };
        // release stage k of the tile; warp 0 (the last reader) then refills
        // the freed slot's next stage
        auto release = [&](int k) -> bool {
            __syncwarp();
            bool good = true;
            if (lane == 0) {
                mbar_arrive(empty0 + 8u * ((z + (unsigned)k) & (kTmaStages - 1)));
                if (q == 0) good = issue();
            }
            if (q == 0) good = __shfl_sync(0xFFFFFFFFu, (int)good, 0) != 0;
            return good;
        };
        for (int k = 0; k < q && ok; ++k) {
            ok = tma_wait(full_of(k), par_of(k), abort);
            if (ok) ok = release(k);
        }
        if (ok) ok = tma_wait(full_of(q), par_of(q), abort);
        float2 acc[X][2];
        float4 win[X];
#pragma unroll
        for (int i = 0; i < X; ++i) acc[i][0] = acc[i][1] = make_float2(0.0f, 0.0f);
        bool started = false;
        // byte address of ring row 0 of this warp's current block (stage q + b)
        unsigned rowb = (z * X + (unsigned)(q * X)) & (X * kTmaStages - 1);
        for (int b = 0; b < nb && ok; ++b, rowb = (rowb + X) & (X * kTmaStages - 1)) {
            ok = tma_wait(full_of(q + b + 1), par_of(q + b + 1), abort);
            if (!ok) break;
            const int jb = t.jlo + X * b;
            if (jb >= wlo && jb < wend) {
                // the block's rows and the next block's (no wrap inside a block)
                const unsigned char* cur = ring + rowb * kRowBytes;
                const unsigned char* nxt = ring + ((rowb + X) & (X * kTmaStages - 1)) * kRowBytes;
                const unsigned char* c0p = cur + off0;
                const unsigned char* c1p = cur + off1;
                const unsigned char* n0p = nxt + off0;
                const unsigned char* n1p = nxt + off1;
                if (!started) {
#pragma unroll
                    for (int u = 0; u < X; ++u) {
                        if (PASS == 1) {
                            win[u] = *reinterpret_cast<const float4*>(c0p + u * kRowBytes);
                        } else {
                            const float2 a = *reinterpret_cast<const float2*>(c0p + u * kRowBytes);
                            const float2 c = *reinterpret_cast<const float2*>(c1p + u * kRowBytes);
                            win[u] = make_float4(a.x, a.y, c.x, c.y);
                        }
                    }
                    started = true;
                }
                const unsigned long long* tb = taps + jb;
#pragma unroll
                for (int u = 0; u < X; u += 2) {
                    const float4 k4 = *reinterpret_cast<const float4*>(tb + u);
                    const float2 ka = make_float2(k4.x, k4.y), kb = make_float2(k4.z, k4.w);
#pragma unroll
                    for (int i = 0; i < X; ++i) {
                        const float4 w = win[(u + i) % X];
                        acc[i][0] = __ffma2_rn(ka, make_float2(w.x, w.y), acc[i][0]);
                        acc[i][1] = __ffma2_rn(ka, make_float2(w.z, w.w), acc[i][1]);
                    }
                    if (PASS == 1) {
                        win[u] = *reinterpret_cast<const float4*>(n0p + u * kRowBytes);
                    } else {
                        const float2 a = *reinterpret_cast<const float2*>(n0p + u * kRowBytes);
                        const float2 c = *reinterpret_cast<const float2*>(n1p + u * kRowBytes);
                        win[u] = make_float4(a.x, a.y, c.x, c.y);
                    }
#pragma unroll
                    for (int i = 0; i < X; ++i) {
                        const float4 w = win[(u + 1 + i) % X];
                        acc[i][0] = __ffma2_rn(kb, make_float2(w.x, w.y), acc[i][0]);
                        acc[i][1] = __ffma2_rn(kb, make_float2(w.z, w.w), acc[i][1]);
                    }
                    if (PASS == 1) {
                        win[u + 1] = *reinterpret_cast<const float4*>(n0p + (u + 1) * kRowBytes);
                    } else {
                        const float2 a = *reinterpret_cast<const float2*>(n0p + (u + 1) * kRowBytes);
                        const float2 c = *reinterpret_cast<const float2*>(n1p + (u + 1) * kRowBytes);
                        win[u + 1] = make_float4(a.x, a.y, c.x, c.y);
                    }
                }
            }
            ok = release(q + b);  // stage q + b is no longer read by this warp
        }
        if (ok) ok = release(q + nb);
        for (int k = q + nb + 1; k < nb + kTmaWarps && ok; ++k) {
            ok = tma_wait(full_of(k), par_of(k), abort);
            if (ok) ok = release(k);
        }
        if (!ok) break;
        z += (unsigned)(nb + kTmaWarps);

        // epilogue: divide by the in-range tap mass, store the column pairs
        if (ylo < R) {
            float* out;
            long long out_row, out_cell;
            const float* norm;
            if (PASS == 0) {
                out = gr.H1; out_row = D; out_cell = h1_stride(gr.H, D);
                norm = gr.table + lv.off_ny;
            } else {
                out = gr.T; out_row = P.ts; out_cell = (long long)gr.W * P.ts;
                norm = gr.table + lv.off_nx;
            }
            const float* rnorm = norm + ((R + 3) & ~3);  // RN(1/n) per position
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                // column pair of acc[.][k]: pass 0 pairs l and l + 32; pass 1
                // columns 4l + 2k and 4l + 2k + 1
                const int gp = PASS == 0 ? (t.c0 >> 1) + lane + 32 * k : (t.c0 >> 1) + 2 * lane + k;
                if (2 * gp < NC) {
                    const int cell = hd > 1 ? (int)__umulhi((unsigned)gp, dinv) : gp;
                    float* o = out + (long long)cell * out_cell + 2 * (gp - cell * hd) + (long long)ylo * out_row;
#pragma unroll
                    for (int i = 0; i < X; ++i) {
                        const int y = ylo + i;
                        if (y < R) {
                            const float nrm = norm[y], rcp = rnorm[y];
                            *reinterpret_cast<float2*>(o + (long long)i * out_row) =
                                make_float2(div_rn(acc[i][k].x, nrm, rcp), div_rn(acc[i][k].y, nrm, rcp));
                        }
                    }
                }
            }
        }
        // the iteration's grouping table, spread over the grid's tiles (the
        // state is not written before the assignment launch's schedule step)
        if (PASS == 0) write_group_table(gr, lv, st, tile, P.ntiles, kTmaThreads);
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicCAS(&st->status, 0, -4);  // PLAS_ERR_TIMEOUT
            // copies still in flight land before the CTA leaves (bounded)
            for (unsigned zz = pz > kTmaStages ? pz - kTmaStages : 0; zz < pz; ++zz) {
                const unsigned fb = full0 + 8u * (zz & (kTmaStages - 1));
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(fb, (zz / kTmaStages) & 1u) && global_ns() - t0 < kWsTimeoutNs) {
                }
            }
        }
    }
}

// Row sizes (floats) of pass-0 boxes with an instantiated kernel: ncell * gs
// for D = 6 (176), 10 (168), 12 (192), 14 (160), 16 (180).
#define PLAS_TMA_ROWS(X_) X_(160) X_(168) X_(176) X_(180) X_(192)

// Tensor maps and shared-memory shape of the tensor-copy kernel for one grid.
bool make_fir_tma(const float* G, const float* H1, int H, int W, int D, int max_steps, FirTma* t) {
    t->ok = false;
    if (D < 2 || (D & 1) || H < 1 || W < 1) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q{};
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int gs = grid_stride(D), hd = D / 2;
    const int ncell = (hd + 62) / hd + 1;  // cells that 64 column pairs can touch
    t->ncell = ncell;
    t->rowf[0] = ncell * gs;
    t->rowf[1] = kFirCols;
    t->steps = (max_steps + 7) & ~7;
    for (int pass = 0; pass < 2; ++pass) {
        const size_t smem = (size_t)kTmaStages * kFirX * t->rowf[pass] * 4 +
                            (((size_t)t->steps * 8 + 127) & ~(size_t)127) + 16 * kTmaStages + 16;
        if (smem > (size_t)kTmaSmemMax) return false;
    }
    if (ncell > 256) return false;
    bool inst = false;
#define PLAS_TMA_IS(n) inst = inst || t->rowf[0] == n;
    PLAS_TMA_ROWS(PLAS_TMA_IS)
#undef PLAS_TMA_IS
    if (!inst) return false;
    CUtensorMap* m0 = reinterpret_cast<CUtensorMap*>(t->map[0]);
    CUtensorMap* m1 = reinterpret_cast<CUtensorMap*>(t->map[1]);
    {   // G: [H rows][W cells][gs floats]; boxes of 8 rows x ncell cells
        const cuuint64_t dims[3] = {(cuuint64_t)gs, (cuuint64_t)W, (cuuint64_t)H};
        const cuuint64_t strides[2] = {(cuuint64_t)gs * 4, (cuuint64_t)W * gs * 4};
        const cuuint32_t box[3] = {(cuuint32_t)gs, (cuuint32_t)ncell, (cuuint32_t)kFirX};
        const cuuint32_t es[3] = {1, 1, 1};
        if (encode(m0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)G, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    {   // H1: [W rows][H*D values, row stride h1_stride]; boxes of 8 rows x 128 values
        const cuuint64_t dims[2] = {(cuuint64_t)H * D, (cuuint64_t)W};
        const cuuint64_t strides[1] = {(cuuint64_t)h1_stride(H, D) * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kFirCols, (cuuint32_t)kFirX};
        const cuuint32_t es[2] = {1, 1};
        if (encode(m1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)H1, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    t->ok = true;
    return true;
}

static size_t tma_smem(const FirTma& t, int pass) {
    return (size_t)kTmaStages * kFirX * t.rowf[pass] * 4 + (((size_t)t.steps * 8 + 127) & ~(size_t)127) +
           16 * kTmaStages + 16;
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
        in = gr.H1; in_row = h1_stride(gr.H, D); in_cell = D;
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
            out = gr.H1; out_row = D; out_cell = h1_stride(gr.H, D);
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
    cudaFuncSetAttribute(fir_tma_kernel<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemMax);
#define PLAS_TMA_ATTR(n) \
    cudaFuncSetAttribute(fir_tma_kernel<0, n>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemMax);
    PLAS_TMA_ROWS(PLAS_TMA_ATTR)
#undef PLAS_TMA_ATTR
    done[dev] = true;
}

void prepare_fir_launches() {
    fir_opt_in();
    prepare_fused_launches();
}

void launch_fir(int pass, const GridRef* grids, const CtaMap* map, int ctas, int D, int variant,
                cudaStream_t s, const FirTma* tma) {
    if (ctas <= 0) return;
    if (variant >= kFirFused) {  // both passes in the pass-0 launch
        if (pass == 0) launch_fir_fused(grids, map, ctas, D, variant - kFirFused, s);
        return;
    }
    fir_opt_in();
    if (variant == kFirLargeRadius && map == nullptr && tma && tma->ok) {
        // persistent: at most one CTA per SM walks the tiles
        TmaParams P;
        memcpy(&P.map, tma->map[pass], sizeof(CUtensorMap));
        P.pass = pass; P.ntiles = ctas; P.D = D; P.ts = target_stride(D);
        P.rowf = tma->rowf[pass]; P.ncell = tma->ncell;
        const int g = std::min(ctas, num_sms());
        const size_t sm = tma_smem(*tma, pass);
        if (pass == 1) {
            fir_tma_kernel<1, 128><<<g, kTmaThreads, sm, s>>>(grids, P);
        } else {
            switch (P.rowf) {
#define PLAS_TMA_CASE(n) \
    case n: fir_tma_kernel<0, n><<<g, kTmaThreads, sm, s>>>(grids, P); break;
                PLAS_TMA_ROWS(PLAS_TMA_CASE)
#undef PLAS_TMA_CASE
                default: break;
            }
        }
        return;
    }
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
