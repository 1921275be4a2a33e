// plas_kernels.h -- launch wrappers of the sort kernels (internal to the
// CUDA library; the C ABI in plas_api.cu calls these).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "plas_device.cuh"

namespace plas {

constexpr int kMaxD = 64;
constexpr int kFirX = 8;  // outputs per thread of the FIR passes (register window)

struct Weights {
    float w[kMaxD];
};

// Per-level blur geometry.  Row pass: taps padded on the left to a multiple of
// kFirX ('rp' zeros before tap -r) and on the right to 'ntp' entries.
struct LevelDesc {
    double phi;
    int r;      // floor(phi): blur half-width
    int beta;   // block side
    int rx, rpx, ntpx;  // row pass: radius capped at W-1, left pad, padded taps
    int ry, rpy, ntpy;  // column pass
    long long off_tx, off_ty, off_nx, off_ny;  // offsets into the float table
};

// Cell strides of the working grid G (features + index, padded to float4) and
// of the target T (features, padded to float4).
inline int grid_stride(int D) { return (D + 1 + 3) & ~3; }
inline int target_stride(int D) { return (D + 3) & ~3; }

// ---- preparation -----------------------------------------------------------
void launch_state_reset(DevState* st, cudaStream_t s);
void launch_minmax(const float* x, long long N, int D, DevState* st, int num_sms,
                   cudaStream_t s);
void launch_finalize_prep(DevState* st, long long N, int D, const Weights& w, int normalize,
                          cudaStream_t s);
// mode 0: identity placement, 1: keyed random placement, 2: perm_init
void launch_pack(const float* x, int N, int D, const Weights& w, int normalize,
                 DevState* st, int mode, const int32_t* perm_init, uint64_t seed,
                 float* G, cudaStream_t s);
void launch_norms(const LevelDesc* lv_dev, int nlev, int H, int W, float* table,
                  cudaStream_t s);

// ---- one iteration -----------------------------------------------------------
struct RowPlan {
    int dc;       // channels per CTA
    int threads;  // 32 * dc
    size_t smem;  // dynamic shared memory bytes
};
RowPlan plan_rows(int W, int D, int ntpx);
void launch_blur_rows(const float* G, int gs, int H, int W, int D, float* H1,
                      const DevState* st, int level, const LevelDesc& lv, const float* table,
                      const RowPlan& plan, cudaStream_t s);

struct ColPlan {
    int ty;       // output rows per CTA
    int threads;  // 32 * ty / kFirX
    size_t smem;
};
ColPlan plan_cols(int H);
void launch_blur_cols(const float* H1, int H, int W, int D, int ts, float* T,
                      const DevState* st, int level, const LevelDesc& lv, const float* table,
                      const ColPlan& plan, cudaStream_t s);

void launch_group_table(uint64_t seed, const DevState* st, int level, int beta, uint32_t* pi,
                        int num_sms, cudaStream_t s);

struct AssignArgs {
    float* G;
    const float* T;
    const uint32_t* pi;
    DevState* st;
    int H, W, D;
    int level, beta, ngroups, nlevels;
    uint64_t seed;
    double tol;
    long long* trace_S;   // optional per-iteration residual sums
    int* trace_level;     // optional per-iteration level
    long long trace_cap;
};
int assign_grid_size(int H, int W, int beta, int num_sms);
void launch_assign(const AssignArgs& a, int grid, cudaStream_t s);

// ---- outputs -----------------------------------------------------------------
void launch_extract_perm(const float* G, int N, int D, int32_t* perm, cudaStream_t s);
// Entries of perm outside [0, N) are not read; their rows are written as zeros.
void launch_gather_rows(const float* src, long long N, int C, const int32_t* perm, float* dst,
                        cudaStream_t s);
void launch_copy_features(const float* T, int N, int D, int ts, float* out, cudaStream_t s);
// acc[0] sum of neighbour L2, acc[1] sum |diff|*scale, acc[2] sum (|diff|*scale)^2
void launch_neighbour_metrics(const float* g, int stride, int H, int W, int D, double scale,
                              double* acc, int num_sms, cudaStream_t s);

// ---- errors (thread-local message behind plas_last_error) ---------------------
void set_last_error(const char* msg);

// ---- debug / standalone --------------------------------------------------------
void launch_keyed_permutation(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n,
                              uint32_t* out, int num_sms, cudaStream_t s);
void launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out,
                   cudaStream_t s);

}  // namespace plas
