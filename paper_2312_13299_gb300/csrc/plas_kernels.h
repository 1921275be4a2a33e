// plas_kernels.h -- kernels and launch wrappers of the PLAS sort (internal to
// the CUDA library; the C ABI in plas_api.cu / engine.cu calls these).
//
// Every per-iteration kernel works on a list of grids (GridRef) and reads each
// grid's current radius level from that grid's device state, so one launch
// per kernel class advances every active grid by one iteration (a "sweep").
// A CTA finds its grid through a per-launch map {grid, local CTA, CTAs of that
// grid}; a single sort is the one-grid case with no map.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "plas_device.cuh"

namespace plas {

constexpr int kMaxD = 64;
constexpr int kFirX = 8;       // outputs per lane and column of the FIR passes
constexpr int kFirCols = 128;  // columns per FIR CTA (four per lane)
// FIR tilings (identical results); which one a radius uses is a tuning choice
// Both passes in one launch (fused_kernels.cu) for radii up to kFusedMaxR and
// up to 16 channels, one kernel per radius group (variants kFirFused + g for
// radii up to kFusedGroupMaxR[g]).
constexpr int kFusedGroups = 3;
constexpr int kFusedGroupMaxR[kFusedGroups] = {3, 7, 11};
constexpr int kFusedMaxR = 11, kFusedMaxD = 16;
constexpr int kFirLargeRadius = 0, kFirSmallRadius = 1, kFirMediumRadius = 2, kFirFused = 3,
              kFirTilings = kFirFused + kFusedGroups;
inline int fused_variant(int r) {
    return kFirFused + (r <= kFusedGroupMaxR[0] ? 0 : r <= kFusedGroupMaxR[1] ? 1 : 2);
}

// Row stride (floats) of the first-pass output H1 ([x][y][d], W rows of H*D
// values): padded to 16 bytes so that tensor copies can stream its rows.
__host__ __device__ inline int h1_stride(int H, int D) { return (H * D + 3) & ~3; }

// The large tiling's persistent tensor-copy kernel (single grids, even D):
// per grid, a tensor map of G (pass 0, [H][W][gs] floats) and of H1 (pass 1,
// [W][h1_stride] floats), the shared-memory row size of each pass and the
// tap steps kept resident.  ok = false: the chunked ring kernel runs instead.
struct FirTma {
    alignas(64) unsigned char map[2][128];  // CUtensorMap per pass
    int rowf[2];    // floats per ring row (pass 0: ncell * gs, pass 1: 128)
    int ncell;      // cells per pass-0 row box
    int steps;      // tap steps kept in shared memory (>= every level's)
    bool ok = false;
};
// Builds *t for a grid whose G and H1 live at the given addresses; max_steps
// = the largest padded tap-step count of any level.  false: not eligible.
bool make_fir_tma(const float* G, const float* H1, int H, int W, int D, int max_steps, FirTma* t);
constexpr int kAssignThreads = 256;

struct Weights {
    float w[kMaxD];
};

// Per-level blur geometry.  Taps are stored as duplicated pairs (k, k): tap j
// (-r <= j <= r) at pair index rp + j (rp = r, so tap -r is step 0), then
// zero pairs up to 'ntp' entries, a multiple of kFirX.  The border norms of an axis of length len follow,
// then (at offset round_up(len, 4)) their reciprocals RN(1/n).
struct LevelDesc {
    double phi;
    int r;      // floor(phi): blur half-width
    int beta;   // block side
    int rx, rpx, ntpx;  // pass along x: radius capped at W-1, left pad, padded taps
    int ry, rpy, ntpy;  // pass along y
    long long off_tx, off_ty, off_nx, off_ny;  // float offsets into the level table
};

// One grid of a sweep.
struct GridRef {
    float* G;             // N x GS working grid (features, index, pad)
    float* T;             // N x TS target
    float* H1;            // N x D first-pass output, [x][y][d]
    uint32_t* pi;         // grouping table (>= max beta^2 entries)
    DevState* st;
    const LevelDesc* lv;  // nlev entries
    const float* table;   // level table (taps, norms)
    int H, W;
    int nlev;
    int target_mode;      // 0 Gaussian target, 1 box target
    uint64_t seed;
    long long* trace_S;   // optional per-iteration residual sums
    int* trace_level;     // optional per-iteration level
    long long trace_cap;
    long long* sat;       // box target: N x round_up(D, 2) int64 summed-area table
    int checked;          // checked run: device bounds checks into the status word
    int edge_blocks;      // 1: the blocks cut by the grid border take part (default)
};

// CTA -> grid map entry of a batched launch.
struct CtaMap {
    int grid;   // index into the GridRef array
    int local;  // CTA index within that grid
    int count;  // CTAs of that grid in this launch
    int pad_;
};

struct CtaRef {
    int g, local, count;
};

// The grid, CTA index within the grid and the grid's CTA count of this CTA
// (no map: one grid, the whole launch).
__device__ __forceinline__ CtaRef resolve_cta(const CtaMap* __restrict__ map) {
    if (map == nullptr) return CtaRef{0, (int)blockIdx.x, (int)gridDim.x};
    const CtaMap m = map[blockIdx.x];
    return CtaRef{m.grid, m.local, m.count};
}

// The grouping permutation of the current iteration (Sec. 3.1: one random
// permutation of the beta^2 block cells, shared by all blocks), pi[m] for
// m < beta^2, spread over 'count' CTAs of 'threads' threads (this CTA is
// number 'local').  The assignment launch that follows reads it.  Entry m
// holds the block cell l = pi(m) already split into its row and column,
// (l / beta) << 16 | (l % beta) (beta <= 8192), so the assignment divides
// nothing.
__device__ __forceinline__ void write_group_table(const GridRef& gr, const LevelDesc& lv,
                                                  const DevState* st, int local, int count,
                                                  int threads) {
    const uint32_t beta = (uint32_t)lv.beta;
    const uint32_t n = beta * beta;
    const uint32_t h = feistel_half_bits(n);
    const uint64_t it = (uint64_t)st->it;
    const uint32_t stride = (uint32_t)count * (uint32_t)threads;
    for (uint32_t m = (uint32_t)local * (uint32_t)threads + threadIdx.x; m < n; m += stride) {
        const uint32_t l = keyed_permute(m, n, h, gr.seed, kTagGroup, it);
        const uint32_t ly = l / beta;
        gr.pi[m] = (ly << 16) | (l - ly * beta);
    }
}

// Cell strides of the working grid G (features + index, padded to float4) and
// of the target T (features, padded to float4).
inline int grid_stride(int D) { return (D + 1 + 3) & ~3; }
inline int target_stride(int D) { return (D + 3) & ~3; }

// ---- CTA counts per grid ------------------------------------------------------
int fir_ctas(int rows, int cols, int variant);  // rows = blur axis length, cols = cells * D
int fused_ctas(int H, int W);
// CTAs of pass 'pass' (0: along y, 1: along x) of an H x W x D grid in FIR
// variant 'var' (the fused variant runs everything in its pass-0 launch)
inline int fir_pass_ctas(int pass, int H, int W, int D, int var) {
    if (var >= kFirFused) return pass == 0 ? fused_ctas(H, W) : 0;
    return pass == 0 ? fir_ctas(H, W * D, var) : fir_ctas(W, H * D, var);
}
constexpr int kAssignMaxPerSm = 16;
int assign_ctas(int H, int W, int num_sms, int per_sm);

// ---- preparation (per grid) ----------------------------------------------------
void launch_state_reset(DevState* st, cudaStream_t s);
void launch_minmax(const float* x, long long N, int D, DevState* st, int num_sms,
                   cudaStream_t s);
void launch_finalize_prep(DevState* st, long long N, int D, const Weights& w, int normalize,
                          cudaStream_t s);
// mode 0: identity placement, 1: keyed random placement, 2: perm_init
void launch_pack(const float* x, int N, int D, const Weights& w, int normalize, DevState* st,
                 int mode, const int32_t* perm_init, uint64_t seed, float* G, cudaStream_t s);
void launch_norms(const LevelDesc* lv_dev, int nlev, int H, int W, float* table,
                  cudaStream_t s);

// ---- one sweep (every grid in 'grids' advances by one iteration) --------------
// map == nullptr: one grid (grids[0]), CTA index = blockIdx.x.
// pass 0: along y (G -> H1), also writes the iteration's grouping table;
// pass 1: along x (H1 -> T).  Variants kFirFused + g: pass 0 runs both
// passes (G -> T) and the grouping table, pass 1 launches nothing.
// (prepare_fir_launches sets the FIR kernels' shared-memory opt-in once per
// device; launch_fir calls it too, but a stream capture calls it first)
void prepare_fir_launches();
void prepare_fused_launches();
void launch_fir_fused(const GridRef* grids, const CtaMap* map, int ctas, int D, int group,
                      cudaStream_t s);
void launch_fir(int pass, const GridRef* grids, const CtaMap* map, int ctas, int D, int variant,
                cudaStream_t s, const FirTma* tma = nullptr);
void launch_assign(const GridRef* grids, const CtaMap* map, int ctas, int D, double tol,
                   cudaStream_t s, bool checked = false);

// ---- persistent sweep: k iterations of every grid in one cooperative launch ----
// Work items per phase as the per-class launches would run them (the medium
// FIR tiling; map == nullptr: one grid, items 0..n-1).  ctl: device control
// block (reset by the launch).  Waits at the grid barriers give up after
// limit_ns (PLAS_ERR_TIMEOUT in ctl->status and in every grid's status word).
// Returns 0, -1 (unsupported D) or -3 (a CUDA call failed).
struct PersistCtl {
    unsigned int arrive;  // CTAs arrived at the current barrier
    unsigned int gen;     // barrier generation
    int status;           // 0, or PLAS_ERR_TIMEOUT after a wait gave up
    int pad_;
};
int launch_persist(const GridRef* grids, int ngrids, const CtaMap* map_y, int n_y,
                   const CtaMap* map_x, int n_x, const CtaMap* map_a, int n_a, int D, int k,
                   double tol, PersistCtl* ctl, unsigned long long limit_ns, cudaStream_t s);

// ---- box target (target_mode 1): one grid -------------------------------------
// (prepare_box_launches: the shared-memory opt-in, once per device, before a
// stream capture; launch_box_target calls it too)
void prepare_box_launches();
void launch_box_target(const GridRef* grid, int H, int W, int D, int num_sms, cudaStream_t s);

// ---- outputs -----------------------------------------------------------------
void launch_extract_perm(const float* G, int N, int D, int32_t* perm, cudaStream_t s);
// bijection check of perm over [0, N): res[0] (preset to INT_MAX) receives the
// smallest position holding an out-of-range or repeated value; seen and dup
// are zeroed bitmaps of ceil(N/32) words
void launch_check_permutation(const int32_t* perm, int N, uint32_t* seen, uint32_t* dup, int* res,
                              int num_sms, cudaStream_t s);
// dst[p] = src[perm[p]] for p < N; src has Nsrc rows (< 0: N).  Entries of
// perm outside [0, Nsrc) are not read; their rows are written as zeros.
void launch_gather_rows(const float* src, long long N, int C, const int32_t* perm, float* dst,
                        cudaStream_t s, long long Nsrc = -1);
void launch_copy_features(const float* T, int N, int D, int ts, float* out, cudaStream_t s);
// acc[0] sum of neighbour L2, acc[1] sum |diff|*scale, acc[2] sum (|diff|*scale)^2
void launch_neighbour_metrics(const float* g, int stride, int H, int W, int D, double scale,
                              double* acc, int num_sms, cudaStream_t s);

// ---- checked runs ---------------------------------------------------------------
constexpr int kGuardBytes = 256;          // guard band after every workspace region
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kMaxGuards = 16;
struct Guards {
    unsigned char* at[kMaxGuards];
    int n;
};
// bad[0] = number of guard bytes that differ from kGuardByte
void launch_fill_guards(const Guards& g, cudaStream_t s);
void launch_check_guards(const Guards& g, unsigned int* bad, cudaStream_t s);

// ---- errors (thread-local message behind plas_last_error) ---------------------
void set_last_error(const char* msg);

// seeded uniform [0, 1) values (Philox, tag 4), for synthetic tuning inputs
void launch_fill_uniform(float* out, long long n, uint64_t seed, cudaStream_t s);

// ---- debug / standalone --------------------------------------------------------
void launch_keyed_permutation(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n,
                              uint32_t* out, int num_sms, cudaStream_t s);
void launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out,
                   cudaStream_t s);

}  // namespace plas
