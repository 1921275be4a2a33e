// loss_kernels.cu -- the grid smoothness loss of Sec. 3.2 (Morgenstern et
// al., arXiv 2312.13299): every attribute channel of the sorted grid is
// blurred with a 2-D Gaussian and the deviation of each value from the blur
// is penalised.  Here the penalty is the squared deviation with per-channel
// weights lam_c:
//     r = x - B x,   L = (1/M) sum lam_c r^2,   dL/dx = (2 g / M) lam_c (r - B r)
// B is separable with zero padding and symmetric taps, so B^T = B.
//
// One streaming kernel evaluates v = u - B u for u = x (forward, and the first
// backward pass) or u = r (second backward pass).  A CTA owns a strip of 32
// cells x all C channels and walks down TYS rows: each input row segment
// (with a halo of h cells) is loaded once, blurred along x into a ring of
// 2h+1 rows in shared memory, and the centre row of the ring is blurred along
// y.  Partial sums are FP64 per CTA and reduced in a fixed order.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/plas.h"
#include "plas_kernels.h"

namespace plas_loss {

constexpr int kTX = 32;       // cells per strip
constexpr int kTYS = 32;      // rows per CTA
constexpr int kMaxH = 15;     // ksize <= 31
constexpr int kThreads = 256;

struct Taps {
    float b[2 * kMaxH + 1];
};


template <bool GRAD>
__global__ void __launch_bounds__(kThreads) smooth_kernel(
    const float* __restrict__ u, int H, int W, int C, int h, Taps tp,
    const float* __restrict__ lam, float* __restrict__ out, const float* __restrict__ gscalar,
    double inv_m, double* __restrict__ partials) {
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
    if (GRAD) coef = (float)(2.0 * (double)(*gscalar) * inv_m);

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
                    if (out) out[cbase + e] = v;
                    part += (double)l * (double)v * (double)v;
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
    if (smem_bytes(C, ksize / 2) > 200 * 1024) { plas::set_last_error("too many channels"); return PLAS_ERR_INVALID_ARG; }
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

static size_t ws_bytes_for(int H, int W, int C) {
    const dim3 g = grid_of(H, W);
    const size_t part = ((size_t)g.x * g.y * sizeof(double) + 255) / 256 * 256;
    return part + (size_t)H * W * C * sizeof(float);
}

// Dynamic shared memory above 48 KB needs an opt-in; request exactly what the
// launch uses (the kernel also has a little static shared memory).
template <bool GRAD>
static bool set_smem_attr(size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(smooth_kernel<GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes) == cudaSuccess;
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
// cudaGetSymbolAddress, once per device, with that device current.
static double* noalloc_partials(int* err) {
    static double* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = PLAS_ERR_CUDA;
        return nullptr;
    }
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) {
            cudaGetLastError();
            *err = PLAS_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = (double*)p;
    }
    *err = PLAS_OK;
    return addr[dev];
}

}  // namespace plas_loss

using namespace plas_loss;

extern "C" {

size_t plas_smooth_loss_workspace_bytes(int H, int W, int C) {
    if (H < 1 || W < 1 || C < 1) return 0;
    return ws_bytes_for(H, W, C);
}

int plas_smooth_loss_fwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, float* loss, void* workspace, size_t ws_bytes,
                         void* stream) {
    if (int e = check_args(x, H, W, C, sigma, ksize)) return e;
    if (!loss) { plas::set_last_error("loss is NULL"); return PLAS_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g = grid_of(H, W);
    const size_t need = (size_t)g.x * g.y * sizeof(double);
    void* mem = workspace;
    if (mem) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(mem) % 256)) {
            plas::set_last_error("workspace too small or misaligned");
            return PLAS_ERR_INVALID_ARG;
        }
    } else if (cudaMallocAsync(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        plas::set_last_error("allocation failed");
        return PLAS_ERR_OOM;
    }
    const int h = ksize / 2;
    const size_t sm = smem_bytes(C, h);
    if (!set_smem_attr<false>(sm)) {
        cudaGetLastError();
        if (!workspace) cudaFreeAsync(mem, st);
        plas::set_last_error("too many channels for the shared-memory tile");
        return PLAS_ERR_INVALID_ARG;
    }
    const double inv_m = 1.0 / ((double)H * W * C);
    smooth_kernel<false><<<g, kThreads, sm, st>>>(x, H, W, C, h, make_taps(sigma, ksize), ch_weights,
                                                  nullptr, nullptr, inv_m, (double*)mem);
    finish_loss_kernel<<<1, 1024, 0, st>>>((const double*)mem, (int)(g.x * g.y), inv_m, loss);
    cudaError_t e = cudaGetLastError();
    if (!workspace) cudaFreeAsync(mem, st);
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
}

int plas_smooth_loss_bwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, const float* grad_loss, float* grad_x,
                         void* workspace, size_t ws_bytes, void* stream) {
    if (int e = check_args(x, H, W, C, sigma, ksize)) return e;
    if (!grad_loss || !grad_x) { plas::set_last_error("grad_loss / grad_x is NULL"); return PLAS_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g = grid_of(H, W);
    const size_t need = ws_bytes_for(H, W, C);
    void* mem = workspace;
    if (mem) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(mem) % 256)) {
            plas::set_last_error("workspace too small or misaligned");
            return PLAS_ERR_INVALID_ARG;
        }
    } else if (cudaMallocAsync(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        plas::set_last_error("allocation failed");
        return PLAS_ERR_OOM;
    }
    const size_t part = ((size_t)g.x * g.y * sizeof(double) + 255) / 256 * 256;
    float* r = (float*)((char*)mem + part);
    const int h = ksize / 2;
    const size_t sm = smem_bytes(C, h);
    if (!set_smem_attr<false>(sm) || !set_smem_attr<true>(sm)) {
        cudaGetLastError();
        if (!workspace) cudaFreeAsync(mem, st);
        plas::set_last_error("too many channels for the shared-memory tile");
        return PLAS_ERR_INVALID_ARG;
    }
    const double inv_m = 1.0 / ((double)H * W * C);
    const Taps tp = make_taps(sigma, ksize);
    // pass 1: r = x - B x (the weighted residual sum is produced as a by-product)
    smooth_kernel<false><<<g, kThreads, sm, st>>>(x, H, W, C, h, tp, ch_weights, r, nullptr, inv_m,
                                                  (double*)mem);
    // pass 2: grad = (2 g / M) lam (r - B r)
    smooth_kernel<true><<<g, kThreads, sm, st>>>(r, H, W, C, h, tp, ch_weights, grad_x, grad_loss,
                                                 inv_m, nullptr);
    cudaError_t e = cudaGetLastError();
    if (!workspace) cudaFreeAsync(mem, st);
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
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
    const size_t sm = smem_bytes(C, h);
    if (!set_smem_attr<false>(sm)) {
        cudaGetLastError();
        plas::set_last_error("too many channels for the shared-memory tile");
        return PLAS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double inv_m = 1.0 / ((double)H * W * C);
    // every CTA writes its own partial, so the array needs no clearing
    smooth_kernel<false><<<g, kThreads, sm, st>>>(x, H, W, C, h, make_taps(sigma, ksize), ch_weights,
                                                  nullptr, nullptr, inv_m, partials);
    finish_loss_kernel<<<1, 1024, 0, st>>>(partials, (int)(g.x * g.y), inv_m, loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        plas::set_last_error(cudaGetErrorString(e));
        return PLAS_ERR_CUDA;
    }
    return PLAS_OK;
}

}  // extern "C"
