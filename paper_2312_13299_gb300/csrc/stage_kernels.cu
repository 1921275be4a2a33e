// stage_kernels.cu -- preparation of 3DGS attributes before the sort (Sec.
// 3.1 "Organizing Gaussians into a 2D Grid" and Sec. 3.3 "Coordinate space
// contraction" of Morgenstern et al., arXiv 2312.13299):
//
// * activation: the sort runs on the values the renderer sees -- coordinates
//   through the contraction's activation sign(v) (exp(|v|) - 1), exp scale,
//   unit quaternion, sigmoid opacity, DC colour as stored;
// * grid sizing: the largest square grid the Gaussians fill completely,
//   keeping the ones with the highest opacity (the others are pruned).
//   The kept set is exact: the side^2 largest opacity logits, ties to the
//   lower index, listed in ascending index order.  It is found by a radix
//   select of the threshold key (4 passes of 8 bits) and a stream
//   compaction with per-block counts and a single-block offset scan.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "plas_host.h"

namespace plas {

namespace {

constexpr int kSelThreads = 256;
constexpr int kSelPerThread = 4;
constexpr int kSelBlock = kSelThreads * kSelPerThread;  // elements per compaction block

// Order-preserving key of an opacity logit: larger logit -> larger key; -0
// reads as +0; NaN gets the smallest key (pruned first).
__device__ __forceinline__ uint32_t opacity_key(float v) {
    if (v != v) return 0u;
    const uint32_t b = __float_as_uint(__fadd_rn(v, 0.0f));
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// A CTA activates blocks of kActRows rows.  The 14 leading floats of each
// raw row are read as contiguous 56-byte runs (consecutive threads take
// consecutive floats of a row, then of the next row), one thread per row
// activates them in shared memory, and the block's output, kActRows x 14
// contiguous floats, is written back with consecutive threads on consecutive
// floats.  The tile pads rows to 15 floats, so the per-row accesses of the
// middle step fall in distinct banks.
constexpr int kActRows = 256, kActPad = 15;

__device__ __forceinline__ void activate_row(const float* r, float* o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // coordinates: sign(v) (exp(|v|) - 1), via expm1
        const float v = r[k];
        const float m = expm1f(fabsf(v));
        o[k] = v < 0.0f ? -m : m;
    }
#pragma unroll
    for (int k = 3; k < 6; ++k) o[k] = expf(r[k]);  // scale
    const float q0 = r[6], q1 = r[7], q2 = r[8], q3 = r[9];
    const float nn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)),
                                                    __fmul_rn(q2, q2)),
                                          __fmul_rn(q3, q3)));
    const float qs[4] = {q0, q1, q2, q3};
#pragma unroll
    for (int k = 0; k < 4; ++k) o[6 + k] = nn > 0.0f ? __fdiv_rn(qs[k], nn) : 0.0f;
    o[10] = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-r[10])));  // opacity
#pragma unroll
    for (int k = 11; k < 14; ++k) o[k] = r[k];  // DC colour
}

__global__ void __launch_bounds__(kActRows) activate_kernel(const float* __restrict__ raw, long long n,
                                                            int stride, float* __restrict__ out) {
    __shared__ float tile[kActRows * kActPad];
    for (long long base = (long long)blockIdx.x * kActRows; base < n;
         base += (long long)gridDim.x * kActRows) {
        const int rows = (int)min((long long)kActRows, n - base);
        for (int e = threadIdx.x; e < rows * 14; e += kActRows) {
            const int r = e / 14, k = e - r * 14;
            tile[r * kActPad + k] = __ldg(raw + (base + r) * stride + k);
        }
        __syncthreads();
        if ((int)threadIdx.x < rows) {
            float v[14];
            float* t = tile + threadIdx.x * kActPad;
#pragma unroll
            for (int k = 0; k < 14; ++k) v[k] = t[k];
            activate_row(v, t);
        }
        __syncthreads();
        float* o = out + base * 14;
        for (int e = threadIdx.x; e < rows * 14; e += kActRows) {
            const int r = e / 14, k = e - r * 14;
            o[e] = tile[r * kActPad + k];
        }
        __syncthreads();
    }
}

// Selection state in device memory.
struct SelState {
    uint32_t prefix;    // high digits of the threshold key found so far
    uint32_t mask;      // the digits fixed in prefix
    uint32_t remain;    // keys still to take among those matching prefix
    uint32_t pad_;
    uint32_t hist[256];
};

__global__ void select_init_kernel(SelState* s, uint32_t k) {
    const int t = threadIdx.x;
    if (t == 0) {
        s->prefix = 0u;
        s->mask = 0u;
        s->remain = k;
    }
    s->hist[t] = 0u;
}

// histogram of digit 'shift' among keys matching the prefix
__global__ void select_hist_kernel(const float* __restrict__ op, long long n, int stride,
                                   SelState* s, int shift) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t prefix = s->prefix, mask = s->mask;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t key = opacity_key(op[i * stride]);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&s->hist[threadIdx.x], h[threadIdx.x]);
}

// pick the digit holding the remain-th largest key; clear the histogram
__global__ void select_pick_kernel(SelState* s, int shift) {
    if (threadIdx.x == 0) {
        uint32_t above = 0u, d = 0u;
        for (int b = 255; b >= 0; --b) {
            const uint32_t c = s->hist[b];
            if (above + c >= s->remain) {
                d = (uint32_t)b;
                break;
            }
            above += c;
        }
        s->remain -= above;
        s->prefix |= d << shift;
        s->mask |= 0xFFu << shift;
    }
    __syncthreads();
    s->hist[threadIdx.x] = 0u;
}

// per block: keys above the threshold and keys equal to it
__global__ void select_count_kernel(const float* __restrict__ op, long long n, int stride,
                                    const SelState* __restrict__ s, uint32_t* __restrict__ cnt) {
    const uint32_t thr = s->prefix;
    uint32_t gt = 0u, eq = 0u;
    const long long base = (long long)blockIdx.x * kSelBlock;
    for (int e = threadIdx.x; e < kSelBlock; e += kSelThreads) {
        const long long i = base + e;
        if (i < n) {
            const uint32_t key = opacity_key(op[i * stride]);
            gt += key > thr;
            eq += key == thr;
        }
    }
    __shared__ uint32_t sg[kSelThreads], se[kSelThreads];
    sg[threadIdx.x] = gt;
    se[threadIdx.x] = eq;
    __syncthreads();
    for (int w = kSelThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sg[threadIdx.x] += sg[threadIdx.x + w];
            se[threadIdx.x] += se[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cnt[2 * blockIdx.x] = sg[0];
        cnt[2 * blockIdx.x + 1] = se[0];
    }
}

// one block: per compaction block, the rank of its first equal key and its
// output offset (exclusive scans, in block order)
__global__ void select_offsets_kernel(const uint32_t* __restrict__ cnt, int nblocks,
                                      const SelState* __restrict__ s, uint32_t* __restrict__ eq_off,
                                      uint32_t* __restrict__ out_off) {
    __shared__ uint32_t part_eq[1024], part_out[1024];
    const int t = threadIdx.x;
    const int per = (nblocks + 1023) / 1024;
    const int b0 = t * per, b1 = min(b0 + per, nblocks);
    const uint32_t need = s->remain;
    // first sweep: this thread's equal count
    uint32_t e = 0u;
    for (int b = b0; b < b1; ++b) e += cnt[2 * b + 1];
    part_eq[t] = e;
    __syncthreads();
    if (t == 0) {  // exclusive scan over the 1024 thread partials (fixed order)
        uint32_t run = 0u;
        for (int i = 0; i < 1024; ++i) {
            const uint32_t v = part_eq[i];
            part_eq[i] = run;
            run += v;
        }
    }
    __syncthreads();
    // second sweep: equal offsets and kept counts per block
    uint32_t er = part_eq[t], kept = 0u;
    for (int b = b0; b < b1; ++b) {
        eq_off[b] = er;
        const uint32_t ce = cnt[2 * b + 1];
        const uint32_t take = er >= need ? 0u : min(ce, need - er);
        kept += cnt[2 * b] + take;
        er += ce;
    }
    part_out[t] = kept;
    __syncthreads();
    if (t == 0) {
        uint32_t run = 0u;
        for (int i = 0; i < 1024; ++i) {
            const uint32_t v = part_out[i];
            part_out[i] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t oo = part_out[t];
    er = part_eq[t];
    for (int b = b0; b < b1; ++b) {
        out_off[b] = oo;
        const uint32_t ce = cnt[2 * b + 1];
        const uint32_t take = er >= need ? 0u : min(ce, need - er);
        oo += cnt[2 * b] + take;
        er += ce;
    }
}

// per block: keep = key > thr, or key == thr among the first 'need' equal keys
// in index order; kept indices written in index order
__global__ void select_write_kernel(const float* __restrict__ op, long long n, int stride,
                                    const SelState* __restrict__ s,
                                    const uint32_t* __restrict__ eq_off,
                                    const uint32_t* __restrict__ out_off, int32_t* __restrict__ keep) {
    const uint32_t thr = s->prefix, need = s->remain;
    const long long base = (long long)blockIdx.x * kSelBlock;
    const int t = threadIdx.x;
    // thread t handles elements base + t*P .. base + t*P + P - 1 (contiguous)
    uint32_t key[kSelPerThread];
    uint32_t neq = 0u;
#pragma unroll
    for (int e = 0; e < kSelPerThread; ++e) {
        const long long i = base + (long long)t * kSelPerThread + e;
        key[e] = i < n ? opacity_key(op[i * stride]) : 0u;
        neq += (i < n && key[e] == thr);
    }
    __shared__ uint32_t scan_eq[kSelThreads], scan_k[kSelThreads];
    scan_eq[t] = neq;
    __syncthreads();
    // inclusive Hillis-Steele scan (exact integers)
    for (int w = 1; w < kSelThreads; w <<= 1) {
        const uint32_t v = t >= w ? scan_eq[t - w] : 0u;
        __syncthreads();
        scan_eq[t] += v;
        __syncthreads();
    }
    uint32_t er = eq_off[blockIdx.x] + scan_eq[t] - neq;  // equal keys before this thread
    bool kf[kSelPerThread];
    uint32_t nk = 0u;
#pragma unroll
    for (int e = 0; e < kSelPerThread; ++e) {
        const long long i = base + (long long)t * kSelPerThread + e;
        bool k = false;
        if (i < n) {
            if (key[e] > thr) k = true;
            else if (key[e] == thr) {
                k = er < need;
                ++er;
            }
        }
        kf[e] = k;
        nk += k;
    }
    scan_k[t] = nk;
    __syncthreads();
    for (int w = 1; w < kSelThreads; w <<= 1) {
        const uint32_t v = t >= w ? scan_k[t - w] : 0u;
        __syncthreads();
        scan_k[t] += v;
        __syncthreads();
    }
    uint32_t pos = out_off[blockIdx.x] + scan_k[t] - nk;
#pragma unroll
    for (int e = 0; e < kSelPerThread; ++e)
        if (kf[e]) keep[pos++] = (int32_t)(base + (long long)t * kSelPerThread + e);
}

size_t select_ws_bytes(long long n) {
    const long long nb = (n + kSelBlock - 1) / kSelBlock;
    return align_up(sizeof(SelState), 256) + align_up((size_t)nb * 2 * sizeof(uint32_t), 256) +
           2 * align_up((size_t)nb * sizeof(uint32_t), 256);
}

}  // namespace

}  // namespace plas

using namespace plas;

extern "C" int plas_activate_3dgs(const float* raw, long long N, int stride, float* out,
                                  void* stream) {
    set_last_error("");
    if (N < 0 || stride < 14) return fail(PLAS_ERR_INVALID_ARG, "N >= 0 and stride >= 14 required");
    if (N == 0) return PLAS_OK;
    if (!raw || !out) return fail(PLAS_ERR_INVALID_ARG, "raw and out are required");
    const unsigned blocks = (unsigned)std::min<long long>((N + kActRows - 1) / kActRows, (long long)num_sms() * 8);
    activate_kernel<<<blocks, kActRows, 0, (cudaStream_t)stream>>>(raw, N, stride, out);
    return check_launch("activate");
}

extern "C" size_t plas_grid_select_workspace_bytes(long long N) {
    if (N < 1 || N > (1LL << 31) - 1) return 0;
    return select_ws_bytes(N);
}

extern "C" int plas_grid_select(const float* opacity, long long N, int stride, int32_t* keep,
                                int* side_out, void* workspace, size_t ws_bytes, void* stream) {
    set_last_error("");
    if (!side_out) return fail(PLAS_ERR_INVALID_ARG, "side_out is NULL");
    *side_out = 0;
    if (N < 0 || N > (1LL << 31) - 1 || stride < 1)
        return fail(PLAS_ERR_INVALID_ARG, "0 <= N < 2^31 and stride >= 1 required");
    long long side = (long long)std::floor(std::sqrt((double)N));
    while (side * side > N) --side;
    while ((side + 1) * (side + 1) <= N) ++side;
    *side_out = (int)side;
    if (side == 0) return PLAS_OK;
    if (!opacity || !keep) return fail(PLAS_ERR_INVALID_ARG, "opacity and keep are required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t need = select_ws_bytes(N);
    void* mem = workspace;
    if (mem) {
        if (ws_bytes < need || !aligned(mem, 256)) return fail(PLAS_ERR_INVALID_ARG, "workspace too small or misaligned");
    } else if (plas::dev_alloc(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "grid-select workspace");
    }
    char* p = (char*)mem;
    SelState* s = (SelState*)p;
    p += align_up(sizeof(SelState), 256);
    const long long nb = (N + kSelBlock - 1) / kSelBlock;
    uint32_t* cnt = (uint32_t*)p;
    p += align_up((size_t)nb * 2 * sizeof(uint32_t), 256);
    uint32_t* eq_off = (uint32_t*)p;
    p += align_up((size_t)nb * sizeof(uint32_t), 256);
    uint32_t* out_off = (uint32_t*)p;
    const unsigned hb = (unsigned)std::min<long long>((N + 255) / 256, (long long)num_sms() * 8);
    select_init_kernel<<<1, 256, 0, st>>>(s, (uint32_t)(side * side));
    for (int shift = 24; shift >= 0; shift -= 8) {
        select_hist_kernel<<<hb, 256, 0, st>>>(opacity, N, stride, s, shift);
        select_pick_kernel<<<1, 256, 0, st>>>(s, shift);
    }
    select_count_kernel<<<(unsigned)nb, kSelThreads, 0, st>>>(opacity, N, stride, s, cnt);
    select_offsets_kernel<<<1, 1024, 0, st>>>(cnt, (int)nb, s, eq_off, out_off);
    select_write_kernel<<<(unsigned)nb, kSelThreads, 0, st>>>(opacity, N, stride, s, eq_off, out_off, keep);
    const int rc = check_launch("grid select");
    if (!workspace) cudaFreeAsync(mem, st);
    return rc;
}
