// plas_device.cuh -- device-side building blocks of the PLAS sort (sm_103a).
//
// Random sources (Sec. 3.1: random initial placement, random block shift,
// random grouping permutation).  Every random decision is a pure function of
// (seed, stream tag, counter):
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
//     32x32->64 multiplies by 0xD2511F53 / 0xCD9E8D57, crossing the high halves
//     with words 1 and 3 and the round key; the key advances by the Weyl
//     increments 0x9E3779B9 / 0xBB67AE85 between rounds.
//   * a keyed permutation of [0, n): balanced six-round Feistel network on 2h
//     bits (2^(2h) >= n); round function = first Philox word of counter
//     (R, tag<<8 | round, counter_lo, counter_hi), masked to h bits; cycle
//     walking keeps the result inside [0, n).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace plas {

constexpr uint32_t kTagInit = 1u;   // initial random placement
constexpr uint32_t kTagShift = 2u;  // block shift per shift epoch
constexpr uint32_t kTagGroup = 3u;  // grouping permutation per iteration

__host__ __device__ inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Half width (bits) of the Feistel network for a domain of n elements.
__host__ __device__ inline uint32_t feistel_half_bits(uint32_t n) {
    uint32_t m = 0;
    while (m < 32 && ((uint64_t)1 << m) < (uint64_t)n) ++m;
    const uint32_t h = (m + 1) >> 1;
    return h == 0 ? 1u : h;
}

__device__ __forceinline__ uint32_t feistel_encrypt(uint32_t v, uint32_t h, uint32_t k0,
                                                    uint32_t k1, uint32_t tag,
                                                    uint64_t counter) {
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = v >> h, R = v & mask;
#pragma unroll
    for (uint32_t round = 0; round < 6; ++round) {
        const uint4 o = philox4x32_10(
            make_uint4(R, (tag << 8) | round, (uint32_t)counter, (uint32_t)(counter >> 32)), k0,
            k1);
        const uint32_t nl = R;
        R = L ^ (o.x & mask);
        L = nl;
    }
    return (L << h) | R;
}

// Keyed bijection of [0, n).  Terminates: v lies on a cycle of the Feistel
// permutation of [0, 2^(2h)), and that cycle returns to v < n.
__device__ __forceinline__ uint32_t keyed_permute(uint32_t v, uint32_t n, uint32_t h,
                                                  uint64_t seed, uint32_t tag,
                                                  uint64_t counter) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t y = feistel_encrypt(v, h, k0, k1, tag, counter);
    while (y >= n) y = feistel_encrypt(y, h, k0, k1, tag, counter);
    return y;
}

// Block shift of a shift epoch (Sec. 3.1): dy in [0, min(beta, H-beta+1)),
// dx likewise, so at least one full block always fits.
__device__ __forceinline__ void block_shift(uint64_t seed, long long epoch, int beta, int H,
                                            int W, int* dy, int* dx) {
    const uint4 o = philox4x32_10(
        make_uint4((uint32_t)(uint64_t)epoch, (uint32_t)((uint64_t)epoch >> 32), kTagShift, 0u),
        (uint32_t)seed, (uint32_t)(seed >> 32));
    const int my = beta < H - beta + 1 ? beta : H - beta + 1;
    const int mx = beta < W - beta + 1 ? beta : W - beta + 1;
    *dy = (int)(((uint64_t)o.x * (uint64_t)my) >> 32);
    *dx = (int)(((uint64_t)o.y * (uint64_t)mx) >> 32);
}

// Device-resident schedule state.  The first 64 bytes mirror plas_state.
struct DevState {
    long long it;
    long long epoch;
    long long redraws;
    int level;
    int stall;
    int has_prev;
    int done;
    double d_prev;
    double d_last;
    int scale_exp;
    int status;
    // ---- private part ----
    unsigned long long S;     // fixed-point residual sum of the running iteration
    unsigned int arrivals;    // CTAs of the running assignment launch that finished
    int nonfinite;            // input held NaN / Inf
    int bad_index;            // a caller-supplied permutation entry was out of range
    int box_exp;              // box target: fixed-point exponent s of the features
    long long grouped;        // cells that took part in a group, summed
    long long max_iters;      // 0 = none
    // work of the iterations run (for the algorithmic roofline counts)
    double fmas_y;            // in-range tap FMAs of the passes along y
    double fmas_x;            // in-range tap FMAs of the passes along x
    double beta2_sum;         // grouping-table entries generated
    int fused_pending;        // the running iteration's target ran both passes in one launch
    long long fused_its;      // iterations whose target ran in one launch
    double fmas_xf;           // the pass-along-x FMAs of those iterations (not in fmas_x)
    unsigned int lo_bits[64]; // per-channel minimum, order-preserving encoding
    unsigned int hi_bits[64]; // per-channel maximum, order-preserving encoding
};

// Bytes of the state the host reads back when it polls (everything before
// the min/max encodings).
constexpr size_t kStateHeaderBytes = offsetof(DevState, lo_bits);

// In-range taps summed over every position of a pass of length len with
// half-width r <= len - 1: sum_p (min(r, p) + min(r, len-1-p) + 1).
__host__ __device__ inline double pass_taps(long long len, long long r) {
    return (double)(len * (2 * r + 1) - r * (r + 1));
}

// A grid takes no further iteration once its schedule is done or its
// iteration cap is reached.
__device__ __forceinline__ bool sweep_idle(const DevState* st) {
    return st->done || (st->max_iters > 0 && st->it >= st->max_iters);
}

// Order-preserving float <-> uint32 map (for exact atomic min / max).
__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

}  // namespace plas
