// loss_kernels.cu -- the grid smoothness loss of Sec. 3.2 (Morgenstern et
// al., arXiv 2312.13299): every attribute channel of the sorted grid is
// blurred with a 2-D Gaussian and the deviation of each value from the blur
// is penalised.  Here the penalty is the squared deviation with per-channel
// weights lam_c:
//     r = x - B x,   L = (1/M) sum lam_c r^2,   dL/dx = (2 g / M) lam_c (r - B r)
// B is separable with zero padding and symmetric taps, so B^T = B.
//
// One kernel evaluates v = u - B u for u = x (forward, and the first backward
// pass) or u = r (second backward pass).
//
// stream_kernel (half-widths h <= 7): a thread owns one channel c of XB = 4
// consecutive cells and walks down a band of rows, loading each row one row
// ahead of its use.  Consecutive threads take
// consecutive channels, so every load of a warp is one contiguous run of the
// channel-last grid.  Each input row's XB + 2h values are loaded once and
// blurred along x in registers into a ring of the last 2h+1 blurred rows; the
// centre row of the ring is then blurred along y.  The row loop is unrolled by
// 2h+1, so every ring slot is a static register.  No shared memory, no
// barriers.
//
// smooth_kernel (larger h): a CTA owns a strip of 32 cells x all C channels,
// blurs each input row along x into a ring of 2h+1 rows in shared memory and
// the centre row along y.
//
// Both use the same FMA chains (ascending taps along x, then along y).  Loss
// partial sums are FP32 over at most (2h+1) x 8 terms, then FP64 per CTA,
// reduced in a fixed order.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/plas.h"
#include "plas_kernels.h"

namespace plas {
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);  // plas_api.cu
}

namespace plas_loss {

constexpr int kTX = 32;       // cells per strip
constexpr int kTYS = 32;      // rows per CTA
constexpr int kMaxH = 15;     // ksize <= 31
constexpr int kThreads = 256;

struct Taps {
    float b[2 * kMaxH + 1];
};

// The penalty of a residual v and the value the backward's first pass
// stores: squared form (hd <= 0): v^2 and v; Huber form (hd = delta > 0):
// v^2 / 2 or delta (|v| - delta / 2), and clamp(v, -delta, delta).
__device__ __forceinline__ float loss_term(float v, float hd) {
    if (hd > 0.0f) {
        const float a = fabsf(v);
        return a <= hd ? __fmul_rn(0.5f, __fmul_rn(v, v)) : __fmul_rn(hd, __fsub_rn(a, 0.5f * hd));
    }
    return __fmul_rn(v, v);
}
__device__ __forceinline__ float resid_out(float v, float hd) {
    return hd > 0.0f ? fminf(fmaxf(v, -hd), hd) : v;
}
// gradient scale: 2 g / M for the squared form, g / M for Huber
__device__ __forceinline__ float grad_coef(const float* gscalar, double inv_m, float hd) {
    return (float)((hd > 0.0f ? 1.0 : 2.0) * (double)(*gscalar) * inv_m);
}


template <bool GRAD>
__global__ void __launch_bounds__(kThreads) smooth_kernel(
    const float* __restrict__ u, int H, int W, int C, int h, Taps tp,
    const float* __restrict__ lam, float* __restrict__ out, const float* __restrict__ gscalar,
    double inv_m, float hd, double* __restrict__ partials) {
    extern __shared__ __align__(16) float sm[];
    const int x0 = blockIdx.x * kTX;
    const int y0 = blockIdx.y * kTYS;
    const int ncell = min(kTX, W - x0);
    const int rowlen = kTX * C;                  // outputs per row
    const int seglen = (kTX + 2 * h) * C;        // input segment with halo
    const int ring_rows = 2 * h + 1;
    float* seg = sm;                             // seglen
    float* ring = sm + seglen;                   // ring_rows x rowlen
    const int tid = threadIdx.x;
    double part = 0.0;
    float coef = 0.0f;
    if (GRAD) coef = grad_coef(gscalar, inv_m, hd);

    const int ylast = min(y0 + kTYS, H) - 1;
    for (int yi = y0 - h; yi <= ylast + h; ++yi) {
        // (1) input row segment [x0 - h, x0 + kTX + h) x C, zero outside
        const bool yok = yi >= 0 && yi < H;
        const long long rowbase = (long long)yi * W * C;
        for (int e = tid; e < seglen; e += kThreads) {
            const int xs = x0 - h + e / C;
            float v = 0.0f;
            if (yok && xs >= 0 && xs < W) v = u[rowbase + (long long)(x0 - h) * C + e];
            seg[e] = v;
        }
        __syncthreads();
        // (2) blur along x into the ring
        float* dst = ring + ((yi - (y0 - h)) % ring_rows) * rowlen;
        for (int e = tid; e < rowlen; e += kThreads) {
            float acc = 0.0f;
#pragma unroll 4
            for (int j = 0; j <= 2 * h; ++j) acc = __fmaf_rn(tp.b[j], seg[e + j * C], acc);
            dst[e] = acc;
        }
        __syncthreads();
        // (3) blur along y at the centre row yc = yi - h
        const int yc = yi - h;
        if (yc >= y0 && yc <= ylast) {
            const long long cbase = ((long long)yc * W + x0) * C;
            for (int e = tid; e < ncell * C; e += kThreads) {
                float acc = 0.0f;
                for (int j = 0; j <= 2 * h; ++j) {
                    const int rr = (yc - h + j - (y0 - h)) % ring_rows;
                    acc = __fmaf_rn(tp.b[j], ring[rr * rowlen + e], acc);
                }
                const int c = e % C;
                const float l = lam ? __ldg(lam + c) : 1.0f;
                const float v = __fsub_rn(__ldg(u + cbase + e), acc);
                if (GRAD) {
                    out[cbase + e] = __fmul_rn(__fmul_rn(coef, l), v);
                } else {
                    if (out) out[cbase + e] = resid_out(v, hd);
                    part += (double)l * (double)loss_term(v, hd);
                }
            }
        }
        // the next iteration's step (1) overwrites seg only after this
        // barrier; the ring slot it writes in (2) is the oldest row
        __syncthreads();
    }
    if (!GRAD) {
        __shared__ double red[kThreads / 32];
        for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
        if ((tid & 31) == 0) red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += red[w];
            partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}

constexpr int kStreamMaxH = 7;  // largest half-width of the staged kernel

// ---------------------------------------------------------------------------
// staged_kernel (h <= 7, C <= 256): each input row of the CTA's span (cells
// [x0 - h, x0 + XC + h) x all C channels, one contiguous run of the
// channel-last grid) is copied into a ring of shared-memory rows by 16-byte
// cp.async, kSgAhead rows ahead of its use.  A thread owns one channel c of 8
// consecutive cells: it reads its 8 + 2h taps of the row from shared memory,
// blurs them along x into a register ring of the last 2h+1 rows and blurs
// the ring's centre row along y.  Cells are processed as pairs (i, i + 4), so
// both passes run as packed FMAs (two IEEE FMAs per instruction: the same
// chains as scalar FMAs).  Cells outside [0, W) and rows outside the grid
// are zero-filled by the copy itself.
// ---------------------------------------------------------------------------
constexpr int kSgThreads = 256;
constexpr int kSgCells = 8;
constexpr int kSgAhead = 3;

__device__ __forceinline__ void cp_async_16z(void* sdst, const void* gsrc, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_4z(void* sdst, const void* gsrc, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ring slots: a slot is rewritten only after the rows read in the previous
// iteration (the blurred row and the centre row h rows above it)
__host__ __device__ constexpr int sg_slots(int h) { return kSgAhead + h + 2; }

template <int HH, bool GRAD, bool HUBER, bool WRITE>
__device__ __forceinline__ void staged_body(const float* __restrict__ u, int H, int W, int C,
                                            int band, int G, int slot_f, const Taps& tp,
                                            const float* __restrict__ lam, float* __restrict__ out,
                                            float coef0, float hd, double* __restrict__ partials,
                                            float* __restrict__ sg) {
    constexpr int R = 2 * HH + 1;
    constexpr int NS = sg_slots(HH);
    constexpr int NP = kSgCells / 2;
    const int XC = kSgCells * G;
    const int x0 = blockIdx.x * XC;
    const int y0 = blockIdx.y * band, y1 = min(y0 + band, H);
    const long long WC = (long long)W * C;
    const int span = (XC + 2 * HH) * C;
    const int n4 = (span + 6) / 4;  // 16-byte chunks incl. the alignment shift
    const int t = threadIdx.x;

    const int g = t / C;
    const int c = t - g * C;
    const int xg = x0 + kSgCells * g;
    const bool ok = g < G && xg < W;
    const int soff = ok ? kSgCells * g * C + c : 0;  // unused threads read in-bounds
    // cells of the pair (i, i + 4) that are inside the grid (branch-free
    // masks; the staged row already holds zeros beyond the grid)
    bool va[NP], vb[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        va[i] = ok && xg + i < W;
        vb[i] = ok && xg + i + NP < W;
    }
    // output pointer of this thread's channel at cell xg of row 0
    float* const obase = (GRAD || WRITE) ? out + (long long)xg * C + c : nullptr;
    const float l = (lam && ok) ? __ldg(lam + c) : 1.0f;
    const float2 coef2 = GRAD ? make_float2(__fmul_rn(coef0, l), __fmul_rn(coef0, l))
                              : make_float2(0.0f, 0.0f);
    float2 b2[R];
#pragma unroll
    for (int j = 0; j < R; ++j) b2[j] = make_float2(tp.b[j], tp.b[j]);

    const int ystart = y0 - HH, yend = y1 + HH;
    const int wc4 = (int)(WC & 3);
    // staging cursor: the next row to copy, its slot and its first flat index
    int st_row = ystart, st_slot = 0;
    long long st_gs = (long long)ystart * WC + (long long)(x0 - HH) * C;
    // Only the row's own cells [row0, row1) are copied; everything else
    // (cells outside [0, W), rows outside the grid) lands as zeros.  A chunk
    // that straddles a row boundary (only when W*C is not a multiple of 4) is
    // copied float by float.
    auto stage = [&]() {
        float* dst = sg + (size_t)st_slot * slot_f;
        const bool yok = st_row >= 0 && st_row < H;
        const long long row0 = yok ? (long long)st_row * WC : 0, row1 = yok ? row0 + WC : 0;
        const long long s0 = st_gs & ~3LL;  // floor to a 16-byte boundary
        for (int q = t; q < n4; q += kSgThreads) {
            const long long p = s0 + 4LL * q;
            if (p >= row0 && p + 4 <= row1) {
                cp_async_16z(dst + 4 * q, u + p, 16);
            } else if (p + 4 <= row0 || p >= row1) {
                cp_async_16z(dst + 4 * q, u, 0);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in = p + e >= row0 && p + e < row1;
                    cp_async_4z(dst + 4 * q + e, in ? (const void*)(u + p + e) : (const void*)u, in ? 4 : 0);
                }
            }
        }
        cp_async_commit();
        ++st_row;
        st_slot = st_slot + 1 == NS ? 0 : st_slot + 1;
        st_gs += WC;
    };
    // read cursors: row yi (x pass) and row yi - HH (centre)
    int x_slot = 0, x_off = (int)(((long long)ystart * WC + (long long)(x0 - HH) * C) & 3);
    int c_slot = NS - HH, c_off = (int)(((long long)(ystart - HH) * WC + (long long)(x0 - HH) * C) & 3);

    // cells are processed as pairs (i, i + 4), i < 4, so both passes run as
    // packed FMAs (two IEEE FMAs per instruction, the same chains as scalar)
    float2 hr[R][NP];  // x-blurred rows; row yi in slot (yi - ystart) mod R
    double part = 0.0;
    float2 band_acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int a = 0; a < kSgAhead; ++a) stage();
    for (int yb = ystart; yb < yend; yb += R) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int yi = yb + q;
            if (yi < yend) {  // uniform over the CTA
                stage();      // row yi + kSgAhead (past the band: copied, never read)
                cp_async_wait<kSgAhead>();
                __syncthreads();
                const float* rx = sg + (size_t)x_slot * slot_f + x_off + soff;
                float2 v2[NP + 2 * HH];  // (tap k, tap k + 4)
#pragma unroll
                for (int k = 0; k < NP + 2 * HH; ++k) v2[k] = make_float2(rx[k * C], rx[(k + NP) * C]);
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int j = 0; j < R; ++j) acc = __ffma2_rn(b2[j], v2[i + j], acc);
                    hr[q][i] = acc;
                }
                const int yc = yi - HH;
                if (yc >= y0) {
                    const float* rc = sg + (size_t)c_slot * slot_f + c_off + soff + HH * C;
                    float2 sq = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int j = 0; j < R; ++j) acc = __ffma2_rn(b2[j], hr[(q + 1 + j) % R][i], acc);
                        // centre - blur, one rounding (FMA with -1)
                        const float2 vv = __ffma2_rn(make_float2(-1.0f, -1.0f), acc,
                                                     make_float2(rc[i * C], rc[(i + NP) * C]));
                        if (GRAD || WRITE) {
                            float* o = obase + (long long)yc * WC + (long long)i * C;
                            float2 w = vv;
                            if (GRAD) w = __fmul2_rn(coef2, vv);
                            else if (HUBER) w = make_float2(resid_out(vv.x, hd), resid_out(vv.y, hd));
                            if (va[i]) o[0] = w.x;
                            if (vb[i]) o[NP * C] = w.y;
                        }
                        if (!GRAD) {
                            const float2 m2 = make_float2(va[i] ? vv.x : 0.0f, vb[i] ? vv.y : 0.0f);
                            if (HUBER)
                                sq = __fadd2_rn(sq, make_float2(loss_term(m2.x, hd), loss_term(m2.y, hd)));
                            else
                                sq = __ffma2_rn(m2, m2, sq);
                        }
                    }
                    if (!GRAD) band_acc = __ffma2_rn(make_float2(l, l), sq, band_acc);
                }
                // advance the read cursors
                x_slot = x_slot + 1 == NS ? 0 : x_slot + 1;
                x_off = (x_off + wc4) & 3;
                c_slot = c_slot + 1 == NS ? 0 : c_slot + 1;
                c_off = (c_off + wc4) & 3;
            }
        }
        if (!GRAD) {  // at most R rows x 4 cells in each FP32 partial
            part += (double)band_acc.x + (double)band_acc.y;
            band_acc = make_float2(0.0f, 0.0f);
        }
    }
    cp_async_wait<0>();
    if (!GRAD) {
        __shared__ double red[kSgThreads / 32];
        for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
        if ((t & 31) == 0) red[t >> 5] = part;
        __syncthreads();
        if (t == 0) {
            double s2 = 0.0;
            for (int w = 0; w < kSgThreads / 32; ++w) s2 += red[w];
            partials[blockIdx.y * gridDim.x + blockIdx.x] = s2;
        }
    }
}

template <int HH, bool GRAD, bool HUBER, bool WRITE>
__global__ void __launch_bounds__(kSgThreads) staged_kernel(
    const float* __restrict__ u, int H, int W, int C, int band, int G, int slot_f, Taps tp,
    const float* __restrict__ lam, float* __restrict__ out, const float* __restrict__ gscalar,
    double inv_m, float hd, double* __restrict__ partials) {
    extern __shared__ __align__(16) float sg[];
    const float coef0 = GRAD ? grad_coef(gscalar, inv_m, hd) : 0.0f;
    staged_body<HH, GRAD, HUBER, WRITE>(u, H, W, C, band, G, slot_f, tp, lam, out, coef0, hd, partials,
                                        sg);
}

// Fixed-order sum of the per-CTA partials (one CTA, fixed tree).
__global__ void finish_loss_kernel(const double* __restrict__ partials, int n, double inv_m,
                                   float* __restrict__ loss) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] * inv_m);
}

static size_t smem_bytes(int C, int h) {
    return sizeof(float) * ((size_t)(kTX + 2 * h) * C + (size_t)(2 * h + 1) * kTX * C);
}

static int check_args(const float* x, int H, int W, int C, float sigma, int ksize) {
    if (!x) { plas::set_last_error("x is NULL"); return PLAS_ERR_INVALID_ARG; }
    if (H < 1 || W < 1 || C < 1) { plas::set_last_error("H, W, C must be >= 1"); return PLAS_ERR_INVALID_ARG; }
    if (ksize < 1 || ksize % 2 == 0 || ksize > 2 * kMaxH + 1) {
        plas::set_last_error("ksize must be odd and <= 31");
        return PLAS_ERR_INVALID_ARG;
    }
    if (!(sigma > 0.0f)) { plas::set_last_error("sigma must be > 0"); return PLAS_ERR_INVALID_ARG; }
    // the shared-memory strip kernel (ksize > 15, or C > 256) holds 32 + 2h
    // cells x C channels
    if ((ksize / 2 > kStreamMaxH || C > kSgThreads) && smem_bytes(C, ksize / 2) > 200 * 1024) {
        plas::set_last_error("too many channels");
        return PLAS_ERR_INVALID_ARG;
    }
    return PLAS_OK;
}

static Taps make_taps(float sigma, int ksize) {
    // taps exp(-j^2 / (2 sigma^2)), normalised to sum 1 over the window (FP64)
    Taps t{};
    const int h = ksize / 2;
    double b[2 * kMaxH + 1], sum = 0.0;
    for (int j = -h; j <= h; ++j) {
        b[j + h] = std::exp(-((double)j * (double)j) / (2.0 * (double)sigma * (double)sigma));
        sum += b[j + h];
    }
    for (int j = 0; j <= 2 * h; ++j) t.b[j] = (float)(b[j] / sum);
    return t;
}

static dim3 grid_of(int H, int W) { return dim3((W + kTX - 1) / kTX, (H + kTYS - 1) / kTYS); }

// Partial sums of either kernel for any ksize (the larger of the two counts).
static size_t partial_bytes(int H, int W, int C) {
    const dim3 g = grid_of(H, W);
    long long n = (long long)g.x * g.y;
    if (C <= kSgThreads) {
        const int G = kSgThreads / C;
        n = std::max<long long>(n, (long long)((W + kSgCells * G - 1) / (kSgCells * G)) * ((H + 31) / 32));
    }
    return ((size_t)n * sizeof(double) + 255) / 256 * 256;
}

static size_t ws_bytes_for(int H, int W, int C) {
    return partial_bytes(H, W, C) + (size_t)H * W * C * sizeof(float);
}

// Dynamic shared memory above 48 KB needs an opt-in; request exactly what the
// launch uses (the kernel also has a little static shared memory).
template <bool GRAD>
static bool set_smem_attr(size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(smooth_kernel<GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes) == cudaSuccess;
}

// Launch plan of one pass: the staged kernel for h <= 7, C <= 256 and a
// 16-byte aligned input (row bands chosen so that the grid has at most
// max_partials CTAs), else the shared-memory strip kernel.
struct Plan {
    bool ok = true;  // false: the grid needs more than 65535 CTA rows
    bool staged = false;
    dim3 grid;
    int band = 0;
    int G = 0, slot_f = 0;
    size_t smem = 0;
    long long partials = 0;
};

constexpr size_t kSgMaxSmem = 160 * 1024;
constexpr long long kMaxGridY = 65535;  // CUDA's limit on gridDim.y

static Plan plan_for(const float* u, int H, int W, int C, int h, long long max_partials) {
    Plan p;
    if (h <= kStreamMaxH && C <= kSgThreads && (reinterpret_cast<uintptr_t>(u) % 16) == 0) {
        const int G = kSgThreads / C;
        const int span = (kSgCells * G + 2 * h) * C;
        const int slot_f = ((span + 6) / 4) * 4;
        const size_t smem = (size_t)sg_slots(h) * slot_f * sizeof(float);
        const long long gx = (W + kSgCells * G - 1) / (kSgCells * G);
        // row bands of 32 rows, taller where the CTA count (one partial each)
        // would exceed max_partials or the grid's y extent CUDA's 65535
        int band = 32;
        auto rows = [&](int b) { return (long long)((H + (long long)b - 1) / b); };
        while ((gx * rows(band) > max_partials || rows(band) > kMaxGridY) && band < H) band *= 2;
        if (smem <= kSgMaxSmem && gx * rows(band) <= max_partials && rows(band) <= kMaxGridY) {
            p.staged = true;
            p.G = G;
            p.slot_f = slot_f;
            p.smem = smem;
            p.band = band;
            p.grid = dim3((unsigned)gx, (unsigned)((H + band - 1) / band));
            p.partials = gx * ((H + band - 1) / band);
            return p;
        }
    }
    p.grid = grid_of(H, W);
    p.ok = (H + kTYS - 1) / kTYS <= kMaxGridY;
    p.smem = smem_bytes(C, h);
    p.partials = (long long)p.grid.x * p.grid.y;
    return p;
}

static int plan_error() {
    plas::set_last_error("grid too tall: the strip kernel needs ceil(H/32) <= 65535");
    return PLAS_ERR_INVALID_ARG;
}

template <int HH, bool GRAD, bool HUBER, bool WRITE>
static int launch_staged_t(const Plan& p, const float* u, int H, int W, int C, const Taps& tp,
                           const float* lam, float* out, const float* g, double inv_m, float hd,
                           double* partials, cudaStream_t st) {
    if (p.smem > 48 * 1024 &&
        cudaFuncSetAttribute(staged_kernel<HH, GRAD, HUBER, WRITE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess)
        return PLAS_ERR_INVALID_ARG;
    staged_kernel<HH, GRAD, HUBER, WRITE><<<p.grid, kSgThreads, p.smem, st>>>(
        u, H, W, C, p.band, p.G, p.slot_f, tp, lam, out, g, inv_m, hd, partials);
    return PLAS_OK;
}

// The gradient pass has no penalty-specific work (its scale is read from hd),
// so it needs no Huber variant.
template <int HH>
static int launch_staged(bool grad, const Plan& p, const float* u, int H, int W, int C,
                         const Taps& tp, const float* lam, float* out, const float* g,
                         double inv_m, float hd, double* partials, cudaStream_t st) {
    if (grad)
        return launch_staged_t<HH, true, false, true>(p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
    if (hd > 0.0f) {
        if (out)
            return launch_staged_t<HH, false, true, true>(p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
        return launch_staged_t<HH, false, true, false>(p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
    }
    if (out)
        return launch_staged_t<HH, false, false, true>(p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
    return launch_staged_t<HH, false, false, false>(p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
}

// v = u - B u over the grid (GRAD: out = coef lam v, coef = 2 g / M or g / M
// for Huber; else out = v (clamped for Huber) if given, and the per-CTA
// weighted sums of the penalty of v into partials).
static int run_pass(bool grad, const Plan& p, const float* u, int H, int W, int C, int h,
                    const Taps& tp, const float* lam, float* out, const float* g, double inv_m,
                    float hd, double* partials, cudaStream_t st) {
    if (p.staged) {
        switch (h) {
            case 0: return launch_staged<0>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 1: return launch_staged<1>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 2: return launch_staged<2>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 3: return launch_staged<3>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 4: return launch_staged<4>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 5: return launch_staged<5>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            case 6: return launch_staged<6>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
            default: return launch_staged<7>(grad, p, u, H, W, C, tp, lam, out, g, inv_m, hd, partials, st);
        }
    }
    if (grad) {
        if (!set_smem_attr<true>(p.smem)) return PLAS_ERR_INVALID_ARG;
        smooth_kernel<true><<<p.grid, kThreads, p.smem, st>>>(u, H, W, C, h, tp, lam, out, g, inv_m,
                                                              hd, partials);
    } else {
        if (!set_smem_attr<false>(p.smem)) return PLAS_ERR_INVALID_ARG;
        smooth_kernel<false><<<p.grid, kThreads, p.smem, st>>>(u, H, W, C, h, tp, lam, out, g,
                                                               inv_m, hd, partials);
    }
    return PLAS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free forward: the per-CTA partial sums live in this file-scope
// device array instead of caller or stream-ordered memory.  Every GPU that
// loads the library holds it (512 KB) until the process exits.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPartials = 65536;  // (ceil(W/32) * ceil(H/32)) limit
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

// Device address of g_noalloc_partials for the current device.  In host code
// the symbol is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The
// cache is atomic: threads that race on a device's first call each look the
// address up and store the same value.  A cudaDeviceReset of a device makes
// its cached address stale; the allocation-free entry point is not meant to
// be used across one.
static double* noalloc_partials(int* err) {
    static std::atomic<double*> addr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = PLAS_ERR_CUDA;
        return nullptr;
    }
    double* a = addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) {
            cudaGetLastError();
            *err = PLAS_ERR_CUDA;
            return nullptr;
        }
        a = (double*)p;
        addr[dev].store(a, std::memory_order_release);
    }
    *err = PLAS_OK;
    return a;
}

}  // namespace plas_loss

using namespace plas_loss;

extern "C" {

size_t plas_smooth_loss_workspace_bytes(int H, int W, int C) {
    if (H < 1 || W < 1 || C < 1) return 0;
    return ws_bytes_for(H, W, C);
}

int plas_smooth_loss_fwd_ex(const float* x, int H, int W, int C, float sigma, int ksize,
                            const float* ch_weights, float huber_delta, float* loss,
                            void* workspace, size_t ws_bytes, void* stream) {
    if (int e = check_args(x, H, W, C, sigma, ksize)) return e;
    if (!(huber_delta >= 0.0f) || huber_delta > 3.0e38f) {
        plas::set_last_error("huber_delta must be finite and >= 0");
        return PLAS_ERR_INVALID_ARG;
    }
    if (!loss) { plas::set_last_error("loss is NULL"); return PLAS_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int h = ksize / 2;
    const Plan p = plan_for(x, H, W, C, h, 1LL << 40);
    if (!p.ok) return plan_error();
    const size_t need = (size_t)p.partials * sizeof(double);
    void* mem = workspace;
    if (mem) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(mem) % 256)) {
            plas::set_last_error("workspace too small or misaligned");
            return PLAS_ERR_INVALID_ARG;
        }
    } else if (plas::dev_alloc(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        plas::set_last_error("allocation failed");
        return PLAS_ERR_OOM;
    }
    const double inv_m = 1.0 / ((double)H * W * C);
    int rc = run_pass(false, p, x, H, W, C, h, make_taps(sigma, ksize), ch_weights, nullptr, nullptr,
                      inv_m, huber_delta, (double*)mem, st);
    if (rc == PLAS_OK)
        finish_loss_kernel<<<1, 1024, 0, st>>>((const double*)mem, (int)p.partials, inv_m, loss);
    cudaError_t e = cudaGetLastError();
    if (!workspace) cudaFreeAsync(mem, st);
    if (rc != PLAS_OK) {
        plas::set_last_error("too many channels for the shared-memory tile");
        return rc;
    }
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
}

int plas_smooth_loss_bwd_ex(const float* x, int H, int W, int C, float sigma, int ksize,
                            const float* ch_weights, float huber_delta, const float* grad_loss,
                            float* grad_x, void* workspace, size_t ws_bytes, void* stream) {
    if (int e = check_args(x, H, W, C, sigma, ksize)) return e;
    if (!(huber_delta >= 0.0f) || huber_delta > 3.0e38f) {
        plas::set_last_error("huber_delta must be finite and >= 0");
        return PLAS_ERR_INVALID_ARG;
    }
    if (!grad_loss || !grad_x) { plas::set_last_error("grad_loss / grad_x is NULL"); return PLAS_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int h = ksize / 2;
    const Plan p = plan_for(x, H, W, C, h, 1LL << 40);
    if (!p.ok) return plan_error();
    const size_t need = ws_bytes_for(H, W, C);
    void* mem = workspace;
    if (mem) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(mem) % 256)) {
            plas::set_last_error("workspace too small or misaligned");
            return PLAS_ERR_INVALID_ARG;
        }
    } else if (plas::dev_alloc(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        plas::set_last_error("allocation failed");
        return PLAS_ERR_OOM;
    }
    float* r = (float*)((char*)mem + partial_bytes(H, W, C));
    const double inv_m = 1.0 / ((double)H * W * C);
    const Taps tp = make_taps(sigma, ksize);
    // pass 1: r = x - B x (clamped to [-delta, delta] for Huber); the
    // weighted penalty sums are a by-product
    int rc = run_pass(false, p, x, H, W, C, h, tp, ch_weights, r, nullptr, inv_m, huber_delta,
                      (double*)mem, st);
    // pass 2: grad = coef lam (r - B r), coef = 2 g / M (squared) or g / M (Huber)
    if (rc == PLAS_OK)
        rc = run_pass(true, p, r, H, W, C, h, tp, ch_weights, grad_x, grad_loss, inv_m, huber_delta,
                      nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (!workspace) cudaFreeAsync(mem, st);
    if (rc != PLAS_OK) {
        plas::set_last_error("too many channels for the shared-memory tile");
        return rc;
    }
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
}

int plas_smooth_loss_fwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, float* loss, void* workspace, size_t ws_bytes,
                         void* stream) {
    return plas_smooth_loss_fwd_ex(x, H, W, C, sigma, ksize, ch_weights, 0.0f, loss, workspace,
                                   ws_bytes, stream);
}

int plas_smooth_loss_bwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, const float* grad_loss, float* grad_x,
                         void* workspace, size_t ws_bytes, void* stream) {
    return plas_smooth_loss_bwd_ex(x, H, W, C, sigma, ksize, ch_weights, 0.0f, grad_loss, grad_x,
                                   workspace, ws_bytes, stream);
}

// Same result as plas_smooth_loss_fwd; allocates nothing (see plas.h).
int plas_smooth_loss_fwd_noalloc(const float* x, int H, int W, int C, float sigma, int ksize,
                                 const float* ch_weights, float* loss, void* stream) {
    if (int e = check_args(x, H, W, C, sigma, ksize)) return e;
    if (!loss) { plas::set_last_error("loss is NULL"); return PLAS_ERR_INVALID_ARG; }
    const dim3 g = grid_of(H, W);
    if ((long long)g.x * g.y > kNoAllocMaxPartials) {
        plas::set_last_error("grid too large for the allocation-free loss: "
                             "ceil(W/32)*ceil(H/32) must be <= 65536");
        return PLAS_ERR_INVALID_ARG;
    }
    int err = PLAS_OK;
    double* partials = noalloc_partials(&err);
    if (!partials) {
        plas::set_last_error("cudaGetSymbolAddress failed for the loss scratch array");
        return err;
    }
    const int h = ksize / 2;
    // taller row bands keep the CTA count (one partial each) within the array
    const Plan p = plan_for(x, H, W, C, h, kNoAllocMaxPartials);
    if (!p.ok) return plan_error();
    cudaStream_t st = (cudaStream_t)stream;
    const double inv_m = 1.0 / ((double)H * W * C);
    // every CTA writes its own partial, so the array needs no clearing
    int rc = run_pass(false, p, x, H, W, C, h, make_taps(sigma, ksize), ch_weights, nullptr, nullptr,
                      inv_m, 0.0f, partials, st);
    if (rc != PLAS_OK) {
        cudaGetLastError();
        plas::set_last_error("too many channels for the shared-memory tile");
        return rc;
    }
    finish_loss_kernel<<<1, 1024, 0, st>>>(partials, (int)p.partials, inv_m, loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
}

}  // extern "C"
