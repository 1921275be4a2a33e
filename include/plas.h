/*
 * plas.h -- C ABI of the GB300 (sm_103a) implementation of Parallel Linear
 * Assignment Sorting (PLAS) and of the grid smoothness loss from
 * Morgenstern et al., "Compact 3D Scene Representation via Self-Organizing
 * Gaussian Grids" (arXiv 2312.13299).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers marked "device" are CUDA device (or managed) pointers; "host"
 *    pointers are ordinary CPU memory.  The caller owns every buffer passed
 *    in; the library never frees or retains caller memory after a call.
 *  - Grids are row-major: cell (y, x) of an H x W grid is row y*W + x of an
 *    N x K matrix (N = H*W, K values per cell, contiguous).  All floating
 *    point data is IEEE float32.
 *  - 'stream' is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work is enqueued on it, in order.
 *  - Every function returns PLAS_OK (0) or a negative PLAS_ERR_* code; no
 *    C++ exception crosses this boundary.  plas_last_error() gives a
 *    human-readable message for the most recent failure on the calling
 *    thread.  Invalid arguments are rejected before any work is enqueued.
 *  - Results are a pure function of the inputs, the seed and the schedule:
 *    no floating-point reduction whose order depends on scheduling feeds a
 *    decision of the sort.
 */
#ifndef PLAS_H_
#define PLAS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------- */
/* status codes                                                           */
/* ---------------------------------------------------------------------- */
#define PLAS_OK 0
#define PLAS_ERR_INVALID_ARG (-1) /* bad size, NULL pointer, misalignment   */
#define PLAS_ERR_OOM (-2)         /* device allocation failed               */
#define PLAS_ERR_CUDA (-3)        /* a CUDA runtime call failed             */
#define PLAS_ERR_TIMEOUT (-4)     /* a bounded device wait gave up (the     */
                                  /* target kernel's pipeline waits, ~2 s)  */
#define PLAS_ERR_NONFINITE (-5)   /* input holds NaN or +-Inf               */
#define PLAS_ERR_BUDGET (-6)      /* batch does not fit its memory budget   */
#define PLAS_ERR_INTERNAL (-7)    /* an internal consistency check failed   */
#define PLAS_ERR_NOT_PERMUTATION (-8) /* plas_check_permutation: not a        */
                                      /* bijection of [0, N)                  */

/* ---------------------------------------------------------------------- */
/* schedule of the sort (Sec. 3.1, "Sorting High Dimensional Gaussians")  */
/* ---------------------------------------------------------------------- */
typedef struct plas_schedule {
    double phi0;        /* start radius; <= 0 selects min(H,W)/2 - 1, the    */
                        /* paper's w/2 - 1 (Sec. 3.1)                        */
    double shrink;      /* radius factor per level, 0.95 (Sec. 3.1)          */
    double phi_min;     /* the sort ends when phi falls below this, 1.0      */
    double tol;         /* relative improvement below which an assignment    */
                        /* counts as a stall, 1e-4 (supplementary)           */
    double sigma_ratio; /* Gaussian sigma = sigma_ratio * phi, default 2.0;  */
                        /* the blur half-width is floor(phi) (the paper      */
                        /* fixes neither)                                    */
    int min_block;      /* smallest block side beta, 16 (Sec. 3.1)           */
    int shuffle_init;   /* 1: random initial placement (Sec. 3.1); 0: start  */
                        /* from the identity (or from perm_init)             */
    int normalize;      /* 1: per-channel [0,1] normalisation before the     */
                        /* weights (Sec. 3.1); 0: weights only               */
    int iters_per_poll; /* iterations enqueued between two host reads of the */
                        /* 128-byte device state header; <= 0 selects 8      */
    long long max_iters;/* stop once the iteration counter reaches this;     */
                        /* 0 = run the full schedule                         */
    int profile;        /* 1: time every kernel class with CUDA events and   */
                        /* report it in plas_stats (adds event records;      */
                        /* implies direct launches)                          */
    int graphs;         /* 1: each batch of iters_per_poll iterations is     */
                        /* captured once as a CUDA graph and replayed (the   */
                        /* kernels read the level from device state, so one  */
                        /* graph serves every level); 0: direct launches.    */
                        /* Identical results either way.                     */
    int target_mode;    /* 0: Gaussian target (Sec. 3.1, the default).       */
                        /* 1: box target, a fast low-pass variant: the mean  */
                        /* of the in-range cells of the (2r+1)^2 window on   */
                        /* fixed-point features q = rint(F 2^s), s the       */
                        /* largest <= 40 with max|F| bound * 2^s <= 2^31;    */
                        /* T = ((float)S / (float)n) * 2^-s.  Its cost does  */
                        /* not grow with r (summed-area tables).  Single     */
                        /* sorts only (plas_sort, plas_target_box).          */
    int persistent;     /* 1: one cooperative launch per batch of           */
                        /* iters_per_poll iterations of every grid of a      */
                        /* sweep (grid-wide barriers between the phases,     */
                        /* bounded waits); 0 (default) or -1: separate       */
                        /* launches per kernel class, graph-replayed (faster */
                        /* in every configuration measured).  Gaussian       */
                        /* target only.  Identical results either way.  A    */
                        /* persistent launch holds up to every SM; sorts on  */
                        /* other streams at the same time may delay it, and  */
                        /* a barrier that waits 2 s gives up with            */
                        /* PLAS_ERR_TIMEOUT (the GPU stays usable).  The     */
                        /* concurrent server policy never uses it.           */
    int whole_blocks;   /* 0 (default): every block that meets the grid is  */
                        /* re-assigned, the blocks cut by the grid border    */
                        /* included (their groups of four cells inside the   */
                        /* grid; Sec. 3.1, the shifted blocks cover the      */
                        /* whole grid).  1: whole blocks from the shift on   */
                        /* only (the alternative reading)                    */
    int checked;        /* 1: checked run (plas_sort): 256-byte guard bands   */
                        /* between the workspace regions are filled with a   */
                        /* pattern and verified after the sort, and the      */
                        /* assignment checks every grouping-table entry and  */
                        /* cell position against the grid; a violation      */
                        /* returns PLAS_ERR_INTERNAL.  0 (default): off      */
    long long* trace_S; /* device or NULL: trace_S[it] = fixed-point residual */
                        /* sum of iteration it (mean L2 distance * N * 2^k)  */
    int* trace_level;   /* device or NULL: level of iteration it             */
    long long trace_cap;/* entries of the trace arrays                       */
} plas_schedule;

/* Resumable schedule state: together with the permutation it is a complete
 * snapshot of a sort in progress (the random streams are counter-based). */
typedef struct plas_state {
    long long it;       /* iterations done                                   */
    long long epoch;    /* block-shift epoch (a new random shift per epoch)  */
    long long redraws;  /* shift redraws caused by a stall                   */
    int level;          /* index of the current radius in the phi sequence   */
    int stall;          /* 1 after one non-improving assignment              */
    int has_prev;       /* d_prev valid (0 right after a level change)       */
    int done;           /* 1 once the radius fell below phi_min              */
    double d_prev;      /* mean L2 distance to the target, previous iteration */
    double d_last;      /* mean L2 distance to the target, last iteration    */
    int scale_exp;      /* exponent k of the fixed-point residual sum        */
    int status;         /* device-side status word (PLAS_OK or an error)     */
} plas_state;

/* kernel classes reported by plas_stats.kernel[] */
#define PLAS_K_PREP 0     /* min/max, normalise, initial placement           */
#define PLAS_K_BLUR_ROWS 1/* target, pass along x                            */
#define PLAS_K_BLUR_COLS 2/* target, pass along y (its launches also write    */
                          /* the iteration's grouping permutation)           */
#define PLAS_K_GROUPS 3   /* grouping permutation of the block cells: no     */
                          /* launches of its own (part of BLUR_COLS)         */
#define PLAS_K_ASSIGN 4   /* 24-permutation scoring, swap, residual, schedule */
#define PLAS_K_GATHER 5   /* permutation + carried-attribute gather          */
#define PLAS_K_COUNT 6

typedef struct plas_kernel_stat {
    long long launches; /* launches of this class (including no-op ones)     */
    double ms;          /* summed CUDA-event time                            */
    double bytes;       /* algorithmic bytes moved (see the design notes)    */
    double flops;       /* algorithmic floating-point operations             */
} plas_kernel_stat;

typedef struct plas_stats {
    long long iterations;   /* assignments performed                          */
    long long redraws;      /* shift redraws                                  */
    long long grouped_cells;/* cells that took part in a group, summed        */
    int levels;             /* radius levels in the schedule                  */
    int status;             /* PLAS_OK or the device status word              */
    double final_l2_to_target; /* mean L2 grid-to-target distance, last iter  */
    double neighbour_l2;    /* mean L2 distance of 4-neighbours, final grid   */
    double ms_total;        /* wall time of the call (host clock)             */
    long long launches;     /* kernel launches made by the call (idle ones    */
                            /* after a level change included)                 */
    plas_kernel_stat kernel[PLAS_K_COUNT]; /* filled when schedule.profile=1  */
    long long graph_launches; /* CUDA graph replays (batches of sweeps)       */
    long long graph_captures; /* graphs captured (0 with direct launches)     */
} plas_stats;

/* Fill *out with the defaults above.  Returns PLAS_OK, or
 * PLAS_ERR_INVALID_ARG if out is NULL. */
int plas_default_schedule(plas_schedule* out);

/* Number of radius levels the schedule runs for an H x W grid
 * (phi_L = phi0 * shrink^L while phi_L >= phi_min).  Returns the count
 * (>= 1) or a negative error code for invalid arguments. */
int plas_num_levels(int H, int W, const plas_schedule* sched /* host or NULL */);

/* Device workspace plas_sort needs for an H x W grid of D sort channels
 * (C carried channels do not need workspace).  0 on invalid sizes. */
size_t plas_sort_workspace_bytes(int H, int W, int D);
/* The same for a given schedule (the box target needs an extra N x D int64
 * table).  sched: host or NULL (defaults). */
size_t plas_sort_workspace_bytes_ex(int H, int W, int D, const plas_schedule* sched);

/*
 * plas_sort -- the PLAS grid sort (Sec. 3.1 and its "Blockwise Linear
 * Assignment" and "Organizing Gaussians into a 2D Grid" paragraphs).
 *
 * Finds one permutation that places the N = H*W rows of x on an H x W grid
 * so that grid neighbours are close in the weighted, normalised feature
 * space; all attribute planes then follow that one permutation (Sec. 3,
 * Fig. "grid2splat").
 *
 *   x            device, N x D float32: the sort features of each Gaussian
 *                (activated values, Sec. 3.1).  1 <= D <= 64.
 *   H, W         grid sides, H*W = N, 0 <= N <= 2^26 and max(H, W) * D <=
 *                2^26 (the target passes index columns in 32 bits).  N == 0
 *                is a no-op.
 *   weights      host, D floats (NULL = all ones): per-channel factors
 *                applied after normalisation (Sec. 3.1, Tab. "params").
 *   carried      device, N x C float32 or NULL: attributes that follow the
 *                permutation (e.g. the 45 SH-rest coefficients).
 *   C            carried channels (0 if carried is NULL).
 *   seed         key of every random decision (initial placement, block
 *                shifts, groupings); Philox4x32-10 counters, so results do
 *                not depend on launch shapes or batch composition.
 *   sched        host or NULL (defaults).
 *   perm_init    device, N int32 or NULL: start arrangement (position p
 *                holds Gaussian perm_init[p]).  Required when resuming.
 *   state_io     host or NULL.  If non-NULL and state_io->it > 0 or
 *                state_io->level > 0, the sort resumes from that state and
 *                perm_init (a snapshot); on return it holds the final state.
 *   perm_out     device, N int32: Gaussian index at each grid position
 *                (gather form: sorted = x[perm_out]).
 *   carried_out  device, N x C or NULL: carried[perm_out].
 *   sorted_out   device, N x D or NULL: x[perm_out] (un-normalised).
 *   workspace    device or NULL.  If non-NULL it must hold
 *                plas_sort_workspace_bytes(H, W, D) bytes, 256-byte
 *                aligned, and the call allocates nothing; if NULL the call
 *                allocates and frees stream-ordered memory itself.
 *   ws_bytes     size of workspace.
 *   stats        host or NULL: filled after the sort (the call then waits
 *                for the stream).
 *   stream       cudaStream_t.
 *
 * The call reads a 64-byte state block back to the host every
 * sched->iters_per_poll iterations, so it returns once the whole sort has
 * run on the device.  Errors: PLAS_ERR_INVALID_ARG (sizes, NULL, D range,
 * misaligned pointers), PLAS_ERR_NONFINITE (x holds NaN/Inf; nothing is
 * written to the outputs), PLAS_ERR_OOM, PLAS_ERR_CUDA, PLAS_ERR_TIMEOUT (a
 * wait inside the large-radius target kernel saw no progress for about two
 * seconds; the kernel gave up and left the GPU usable), PLAS_ERR_INTERNAL
 * (the host saw a grid make no progress over five state read-backs).
 */
int plas_sort(const float* x, int H, int W, int D, const float* weights,
              const float* carried, int C, uint64_t seed, const plas_schedule* sched,
              const int32_t* perm_init, plas_state* state_io, int32_t* perm_out,
              float* carried_out, float* sorted_out, void* workspace, size_t ws_bytes,
              plas_stats* stats, void* stream);

/*
 * plas_gather_rows -- dst[p, :] = src[perm[p], :] for p < N (Sec. 3: every
 * attribute plane follows the one permutation).  src, dst: device N x C
 * float32 (must not overlap); perm: device N int32 with values in [0, N)
 * (not checked).  C >= 1.
 */
/*
 * plas_select_rows -- dst[p, :] = src[idx[p], :] for p < n_out, from a
 * source of n_src rows (the kept Gaussians of plas_grid_select, or any
 * subset).  Entries of idx outside [0, n_src) give zero rows.  src: device
 * n_src x C float32, dst: device n_out x C float32 (no overlap), idx: device
 * n_out int32.  C >= 1.
 */
int plas_select_rows(const float* src, long long n_src, int C, const int32_t* idx,
                     long long n_out, float* dst, void* stream);
/*
 * plas_check_permutation -- checks that perm (device, N int32) is a
 * permutation of [0, N), the one-to-one placement of Gaussians on grid cells
 * that the sort produces (Sec. 3.1: every Gaussian lands on exactly one
 * cell).  Returns PLAS_OK, or PLAS_ERR_NOT_PERMUTATION with *first_bad (host
 * int, or NULL) = the smallest position whose value lies outside [0, N) or
 * occurs more than once (a missing value implies such a position).
 * *first_bad is -1 otherwise.  N = 0 is a valid, empty permutation.  Device
 * work: two passes over perm with two bitmaps of ceil(N/32) words, allocated
 * and freed on 'stream'; the call synchronises the stream.  Errors:
 * PLAS_ERR_INVALID_ARG (N < 0 or N > 2^30, or perm NULL with N > 0), PLAS_ERR_OOM,
 * PLAS_ERR_CUDA.
 */
int plas_check_permutation(const int32_t* perm, int N, int* first_bad, void* stream);
int plas_gather_rows(const float* src, int N, int C, const int32_t* perm, float* dst,
                     void* stream);

/*
 * plas_target -- the low-pass target of Sec. 3.1 for one arrangement: the
 * separable Gaussian blur of the weighted, normalised features of x[perm]
 * at radius phi (half-width floor(phi), sigma = sigma_ratio*phi, taps
 * truncated at the border and renormalised by the in-range tap mass).
 * x: device N x D; perm: device N int32; T: device N x D output.
 * weights: host D floats or NULL.  The same kernels as plas_sort's loop.
 */
int plas_target(const float* x, int H, int W, int D, const float* weights, int normalize,
                const int32_t* perm, double phi, double sigma_ratio, float* T, void* stream);
/* plas_target_box -- the box target of schedule.target_mode = 1 for one
 * arrangement (the mean of the in-range cells of the (2r+1)^2 window,
 * r = floor(phi), on fixed-point features; see plas_schedule).  Arguments as
 * plas_target. */
int plas_target_box(const float* x, int H, int W, int D, const float* weights, int normalize,
                    const int32_t* perm, double phi, float* T, void* stream);

/*
 * plas_group_permutation -- the grouping permutation of Sec. 3.1 (one random
 * ordering of the cells of a block, the same for every block): out[m]
 * for m < n, a keyed bijection of [0, n) (six-round Feistel network driven
 * by Philox4x32-10, cycle walking).  tag/counter select the stream (3 and
 * the iteration for groupings, 1 and 0 for the initial placement).
 * out: device n uint32.  1 <= n <= 2^26.
 */
int plas_group_permutation(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n,
                           uint32_t* out, void* stream);

/*
 * plas_philox -- Philox4x32-10 (Salmon et al., SC'11) on the device:
 * out[4i..4i+3] = philox(ctr[4i..4i+3], key).  ctr, out: device 4n uint32.
 */
int plas_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n, uint32_t* out,
                void* stream);

/*
 * plas_grid_metrics -- quality of an H x W x D grid (device, float32):
 *   out[0] mean L2 distance over all horizontal and vertical neighbour pairs;
 *   out[1] VAD: population variance of |a - b| over all neighbour pairs and
 *          all channels, on values multiplied by 'scale' (supplementary,
 *          "Sorting performance"; scale 255 for [0,1] colours);
 *   out[2] mean |a - b| (same pairs, scaled).
 * out: host, 3 doubles.  Waits for the stream.  FP64 accumulation.
 */
int plas_grid_metrics(const float* grid, int H, int W, int D, double scale, double* out,
                      void* stream);

/* ---------------------------------------------------------------------- */
/* smoothness loss (Sec. 3.2)                                             */
/* ---------------------------------------------------------------------- */
/*
 * x: device H x W x C float32, channel-last.  B is the separable Gaussian
 * of 'ksize' taps (odd, 1..31) with the given sigma, normalised to sum 1
 * over the full window, with zero padding.  r = x - Bx.
 *   loss = (1/M) * sum_{y,x,c} lam_c * r^2,   M = H*W*C
 *   dloss/dx = (2 g / M) * lam_c * (r - B r)     (B^T = B: symmetric taps,
 *                                                 zero padding)
 * ch_weights: device C floats or NULL (all ones).
 * plas_smooth_loss_fwd writes loss (device, 1 float).  It accumulates in
 * FP64 with a fixed reduction order, so the value does not depend on
 * scheduling.  plas_smooth_loss_bwd reads grad_loss (device scalar g) and
 * writes grad_x (device H x W x C, must not overlap x); it recomputes r from
 * x.  workspace: device or NULL (then allocated stream-ordered per call),
 * at least plas_smooth_loss_workspace_bytes(H, W, C) bytes, 256-byte
 * aligned.  Errors: PLAS_ERR_INVALID_ARG (sizes, even or too large ksize,
 * sigma <= 0, NULL), PLAS_ERR_OOM, PLAS_ERR_CUDA.
 */
size_t plas_smooth_loss_workspace_bytes(int H, int W, int C);
int plas_smooth_loss_fwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, float* loss, void* workspace,
                         size_t ws_bytes, void* stream);
int plas_smooth_loss_bwd(const float* x, int H, int W, int C, float sigma, int ksize,
                         const float* ch_weights, const float* grad_loss, float* grad_x,
                         void* workspace, size_t ws_bytes, void* stream);

/*
 * The same pair with the penalty chosen by huber_delta (host float, finite,
 * >= 0).  0: the squared form above.  delta > 0: the Huber form that Sec.
 * 3.2 names for the deviation from the blurred grid (delta is not stated in
 * the paper; PyTorch's default is 1.0):
 *   h(r) = r^2 / 2 for |r| <= delta, delta * (|r| - delta / 2) otherwise,
 *   loss = (1/M) * sum lam_c * h(r),
 *   dloss/dx = (g / M) * (psi - B psi),  psi = lam_c * clamp(r, -delta, delta).
 * The paper's configuration (supplementary, Tab. "params") is ksize 5,
 * sigma 3, weights 0.09 on opacity and 0.91 on the rotation channels.
 * Arguments, layout, workspace and errors as above.
 */
int plas_smooth_loss_fwd_ex(const float* x, int H, int W, int C, float sigma, int ksize,
                            const float* ch_weights, float huber_delta, float* loss,
                            void* workspace, size_t ws_bytes, void* stream);
int plas_smooth_loss_bwd_ex(const float* x, int H, int W, int C, float sigma, int ksize,
                            const float* ch_weights, float huber_delta, const float* grad_loss,
                            float* grad_x, void* workspace, size_t ws_bytes, void* stream);

/*
 * plas_smooth_loss_fwd_noalloc -- the same loss as plas_smooth_loss_fwd, for
 * callers that cannot allocate device memory during the call: a host loop
 * whose memory is owned by another allocator with a fixed budget, or a
 * latency-critical loop where cudaMalloc (which may synchronise the device)
 * is not allowed.  The paper has no counterpart; it is a deployment variant.
 *
 * The per-CTA partial sums use a 512 KB array of static device memory inside
 * the library (held on every GPU that loads the library until the process
 * exits).  Limit: ceil(W/32) * ceil(H/32) <= 65536 (e.g. grids up to
 * 8192 x 8192); larger grids return PLAS_ERR_INVALID_ARG.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it (threads
 * that race on that first call store the same address); make that first
 * call before any stream capture.  A cudaDeviceReset invalidates the cached
 * address: do not use this entry point on a device after resetting it.
 * All calls share the one array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 *
 * Result: bit-identical to plas_smooth_loss_fwd whenever the regular call's
 * row bands of 32 rows fit the array, i.e. ceil(W / (8 G)) * ceil(H / 32) <=
 * 65536 with G = floor(256 / C) (channel-last tiles of the ksize <= 15,
 * C <= 256, 16-byte-aligned path), and always on the strip path (ksize > 15,
 * C > 256 or a misaligned x).  Otherwise the bands are taller, the FP64
 * partial sums are added in another grouping, and the value agrees within
 * rounding (relative 1e-12 in practice; the tests allow 1e-5).  Arguments,
 * layout and errors as for plas_smooth_loss_fwd; grids whose strip-path
 * launch would need more than 65535 CTA rows (H > 2,097,120 with ksize > 15,
 * C > 256 or a misaligned x) return PLAS_ERR_INVALID_ARG on every loss entry
 * point.
 */
int plas_smooth_loss_fwd_noalloc(const float* x, int H, int W, int C, float sigma, int ksize,
                                 const float* ch_weights, float* loss, void* stream);

/* ---------------------------------------------------------------------- */
/* preparation of 3DGS attributes before the sort (Sec. 3.1, Sec. 3.3)     */
/* ---------------------------------------------------------------------- */
/*
 * plas_activate_3dgs -- the sort runs on activated values (Sec. 3.1).  Row
 * i of raw (stride floats apart, stride >= 14) holds the trained parameters
 * xyz 0-2 (contracted, Sec. 3.3 "Coordinate space contraction"), log-scale
 * 3-5, quaternion 6-9, opacity logit 10, DC colour 11-13.  out (device,
 * N x 14) receives
 *   xyz = sign(v) * (exp(|v|) - 1), scale = exp(v), quaternion / |q| (a zero
 *   quaternion stays zero), opacity = 1 / (1 + exp(-v)), DC as stored,
 * in FP32 with the CUDA math library (within a few ulp of the FP64 values).
 *
 * plas_grid_select -- the largest square grid the Gaussians fill (Sec.
 * 3.1): side = floor(sqrt(N)), written to *side_out (host).  keep (device,
 * side^2 int32) receives the indices of the side^2 Gaussians with the
 * highest opacity logit, in ascending index order.  Ties go to the lower
 * index, -0 reads as +0, and NaN ranks lowest.  The rest are pruned.
 * 'opacity' points at the first logit, 'stride' floats apart (14 for the raw
 * layout above, from raw + 10).  workspace: device or NULL,
 * plas_grid_select_workspace_bytes(N) bytes, 256-byte aligned.  N < 2^31.
 * Errors: PLAS_ERR_INVALID_ARG, PLAS_ERR_OOM, PLAS_ERR_CUDA.
 */
int plas_activate_3dgs(const float* raw, long long N, int stride, float* out, void* stream);
size_t plas_grid_select_workspace_bytes(long long N);
int plas_grid_select(const float* opacity, long long N, int stride, int32_t* keep, int* side_out,
                     void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* quantisation of the sorted attribute grids (Sec. 3.4)                   */
/* ---------------------------------------------------------------------- */
/*
 * After training, each attribute channel of the sorted grid is clipped to a
 * range and rounded to the nearest of q equally spaced values (Sec. 3.4,
 * "Quantization & Compression"; the paper's q: 2^14 for coordinates, 2^6
 * for scale, opacity and rotation, 2^5 for the SH rest; its clip ranges:
 * DC colour [-2, 4], opacity [-6, 12], SH rest [-1, 1], rotation [-1, 2]).
 *   code = rint(t * (q - 1)),  t = (min(max(x, lo), hi) - lo) / (hi - lo)
 * in FP32 with IEEE division and round-half-to-even (hi == lo gives 0; NaN
 * gives 0).  plas_dequantize maps codes back:
 *   x' = lo + code * ((hi - lo) / (q - 1)).
 * x / out: device N x C float32 (row-major, channel fastest); codes: device
 * N x C uint16; lo, hi: host C floats (finite, lo <= hi); q: host C ints in
 * [2, 65536]; 1 <= C <= 256.  Enqueued on 'stream'.  Errors:
 * PLAS_ERR_INVALID_ARG, PLAS_ERR_CUDA.  The paper has no kernel for this
 * step; the codec that stores the planes (JPEG XL) is not part of this
 * library.
 */
int plas_quantize(const float* x, long long N, int C, const float* lo, const float* hi,
                  const int* q, uint16_t* codes, void* stream);
int plas_dequantize(const uint16_t* codes, long long N, int C, const float* lo,
                    const float* hi, const int* q, float* out, void* stream);

/* ---------------------------------------------------------------------- */
/* batched sort: many independent grids advanced together                 */
/* ---------------------------------------------------------------------- */
typedef struct plas_job {
    const float* x;        /* device, N x D                                  */
    int H, W;              /* grid sides                                     */
    const float* carried;  /* device, N x C or NULL                          */
    int C;
    uint64_t seed;
    int32_t* perm_out;     /* device, N                                      */
    float* carried_out;    /* device, N x C or NULL                          */
    plas_state* state_out; /* host or NULL: final state of this grid         */
} plas_job;

/* Device bytes plas_batch_sort needs for these jobs (all of one D). */
size_t plas_batch_workspace_bytes(int n, const plas_job* jobs, int D);

/*
 * plas_batch_sort -- sorts n independent grids of D channels with one
 * schedule, advancing every unfinished grid by one iteration per sweep:
 * each sweep is one launch per kernel class over all grids, so small grids
 * share the GPU instead of running one after another.  Every grid keeps its
 * own counters and random streams, so each result is bit-identical to
 * plas_sort on that grid alone with the same seed and schedule.
 * jobs: host array of n descriptors; weights: host D floats or NULL.
 * workspace: device, plas_batch_workspace_bytes(...) bytes, or NULL
 * (allocated internally).  Returns PLAS_ERR_INVALID_ARG for a bad job.
 */
int plas_batch_sort(int n, const plas_job* jobs, int D, const float* weights,
                    const plas_schedule* sched, void* workspace, size_t ws_bytes,
                    void* stream);

/* ---------------------------------------------------------------------- */
/* launch-shape autotuning                                                 */
/* ---------------------------------------------------------------------- */
/*
 * Launch shapes the sort can choose without changing any result: the FIR
 * tiling of the target passes (128 rows per CTA with 16 warps, 64 rows with
 * 2 CTAs per SM, or 32 rows per CTA loaded straight into registers without
 * shared memory; the same FMA chains in every case) and the
 * number of assignment CTAs (the residual sum is exact and order-free).  The
 * paper has no counterpart; it is GPU plumbing.
 *
 * plas_autotune: times the candidates on a synthetic H x W x D grid (seeded
 *   uniform values made on the device): the three FIR tilings at radii from 1 up
 *   to the grid's start radius, and the assignment at 2, 4, 8 and 16 CTAs
 *   per SM at the start radius and at radius 8.  It installs the fastest
 *   choice for sorts on this device with D channels and the nearest cell
 *   count, and returns it with the measurements in *out.  Allocates and
 *   frees its own device buffers on 'stream' and synchronises it.
 *   PLAS_ERR_INVALID_ARG for unsupported sizes.
 * plas_set_tuning: installs *t for (H, W, D) on the current device
 *   (t == NULL removes the entry); plas_get_tuning: what a sort of this
 *   shape on the current device would use (the defaults 12, 96 and 4 when
 *   nothing is installed).  A radius r takes the small-radius path when
 *   r < fir_small_below (both passes in one launch when small_fused is 1,
 *   r <= 11 and D <= 16; otherwise the direct kernel), else the 64-row one
 *   when r < fir_medium_below, else the 128-row one, which streams with
 *   tensor copies when large_tma is 1 and the grid allows it.  plas_autotune
 *   times the one-launch kernel for the small path where it applies.
 *   Thread-safe.
 */
#define PLAS_TUNE_MAX_RADII 16
#define PLAS_TUNE_ASSIGN_CANDIDATES 4
typedef struct plas_tuning {
    int fir_small_below;    /* the direct FIR kernel for radii below this      */
    int fir_medium_below;   /* else the 64-row tiling for radii below this     */
    int assign_ctas_per_sm; /* cap on assignment CTAs per SM, 1..16           */
    int n_radii;            /* radii measured by plas_autotune                */
    int radius[PLAS_TUNE_MAX_RADII];
    float fir_small_us[PLAS_TUNE_MAX_RADII];  /* both passes, direct kernel;
                                                 -1: not timed (r > 32)       */
    float fir_medium_us[PLAS_TUNE_MAX_RADII]; /* both passes, 64-row tiling   */
    float fir_large_us[PLAS_TUNE_MAX_RADII];  /* both passes, 128-row tiling  */
    int assign_per_sm[PLAS_TUNE_ASSIGN_CANDIDATES];
    float assign_us[PLAS_TUNE_ASSIGN_CANDIDATES]; /* sum over the two radii   */
    int large_tma;          /* 1: the large tiling streams its input rows with */
                            /* tensor copies (persistent CTAs, single grids of */
                            /* an even D with an instantiated row box); 0: the */
                            /* chunked ring.  Default 0 (the chunked ring was  */
                            /* faster on every grid measured)                  */
    float fir_large_ring_us[PLAS_TUNE_MAX_RADII]; /* both passes, chunked    */
    float fir_large_tma_us[PLAS_TUNE_MAX_RADII];  /* both passes, tensor      */
                                                  /* copies; -1: not eligible */
    int small_fused;        /* 1: radii of the small path up to 11, with at    */
                            /* most 16 channels, run both passes in one launch */
                            /* (the pass along y into shared memory, then the  */
                            /* pass along x); 0: the direct kernel, two        */
                            /* launches.  Same bits.  Default 1                */
} plas_tuning;
int plas_autotune(int H, int W, int D, void* stream, plas_tuning* out);
int plas_set_tuning(int H, int W, int D, const plas_tuning* t /* host or NULL */);
int plas_get_tuning(int H, int W, int D, plas_tuning* out);

/* ---------------------------------------------------------------------- */
/* served sorts: continuous batching under a device-memory budget          */
/* ---------------------------------------------------------------------- */
/*
 * A server owns a FIFO of submitted sort requests and a set of admitted
 * grids that advance together, one iteration per sweep (the kernels of
 * plas_batch_sort).  A request is admitted as soon as its workspace
 * (plas_sort_workspace_bytes) fits into 'mem_budget' next to the admitted
 * ones; requests that arrive while others run join the next sweep.  Results
 * equal plas_sort of the same request alone (per-grid counters and random
 * streams).  A server and its calls belong to one host thread.
 *
 * plas_server_create: D sort channels for every request; weights: host D
 *   floats or NULL; sched: host or NULL; mem_budget in bytes (0 = no
 *   limit); stream: cudaStream_t for all of the server's work.
 * plas_server_submit: queues *job (copied; the device buffers it names must
 *   stay valid until the request completes) and returns its ticket (0, 1,
 *   ...).  PLAS_ERR_BUDGET if the request alone exceeds mem_budget,
 *   PLAS_ERR_INVALID_ARG for a bad descriptor.
 * plas_server_step: admits queued requests that fit, enqueues 'sweeps'
 *   sweeps over the grids the policy chooses, and reports in
 *   done[0..*n_done) (at most 'cap') the tickets whose outputs are complete
 *   on return.  The call does not wait for the sweeps it enqueues: it reads
 *   the grids' state one step behind, so a request is reported a step or two
 *   after its last iteration, and the GPU stays busy while the host runs.
 *   It waits for the stream only when no grid is left to sweep.  A finished
 *   request's workspace is released (stream-ordered) before the next
 *   admission.  job->state_out, if given, is filled on completion.
 * plas_server_set_policy: which admitted grids each step's sweeps advance
 *   (results are the same under every policy; only the timing differs):
 *   PLAS_SERVE_FIFO_FILL (default): in admission order until the estimated
 *     time of one sweep over the chosen grids reaches 0.6 ms (one grid at a
 *     large radius fills a sweep; grids at small radii share one);
 *   PLAS_SERVE_SHORTEST_FIRST: least estimated work left first, same fill;
 *   PLAS_SERVE_ALL: every admitted grid in every sweep.
 *   PLAS_SERVE_CONCURRENT: up to 16 admitted requests each advance on a
 *     stream of their own, in graph-replayed batches of 'sweeps' iterations
 *     with two batches in flight, so every request moves at its own pace.
 *     The oldest admitted request's stream has the highest priority and the
 *     others the lowest: its CTAs get the SMs first, as on the plain path,
 *     and younger requests fill the SMs it leaves idle.  When it finishes,
 *     the next oldest is moved to a high-priority stream.  A step feeds
 *     every lane and waits only when no lane can move.  Switching to or from
 *     this policy needs a server with nothing admitted.
 *   PLAS_SERVE_ADAPTIVE: FIFO_FILL while fewer than eight requests are
 *     admitted, ALL under a larger backlog.
 *   PLAS_ERR_INVALID_ARG for an unknown policy.
 * plas_server_cancel: withdraws a request that is queued or running.  A
 *   queued request is removed at once; a running one leaves the sweeps at
 *   the next plas_server_step, which releases its workspace (stream-ordered,
 *   after the sweeps already enqueued on it).  A cancelled request is never
 *   reported in done[]; its outputs and state_out are left as they are.  No
 *   work enqueued after that step touches its buffers, but work enqueued
 *   before it may still read x on the server's stream: release them
 *   stream-ordered on that stream, or after synchronising it.
 *   The other requests' results do not change.  PLAS_ERR_INVALID_ARG for a
 *   ticket that is unknown, already finished (its outputs are enqueued or
 *   reported) or already cancelled.  The paper has no counterpart; it is a
 *   serving control.
 * plas_server_status: queued and admitted requests, device bytes in use.
 * plas_server_destroy: waits for the stream and frees everything; requests
 *   still queued or running are abandoned (their outputs are undefined).
 */
typedef struct plas_server plas_server;
enum { PLAS_SERVE_FIFO_FILL = 0, PLAS_SERVE_SHORTEST_FIRST = 1, PLAS_SERVE_ALL = 2,
       PLAS_SERVE_CONCURRENT = 3, PLAS_SERVE_ADAPTIVE = 4 };
int plas_server_create(int D, const float* weights, const plas_schedule* sched,
                       size_t mem_budget, void* stream, plas_server** out);
int plas_server_set_policy(plas_server* srv, int policy);
int plas_server_submit(plas_server* srv, const plas_job* job, long long* ticket);
int plas_server_step(plas_server* srv, int sweeps, long long* done, int cap, int* n_done);
int plas_server_cancel(plas_server* srv, long long ticket);
int plas_server_status(plas_server* srv, int* queued, int* active, size_t* mem_in_use);
int plas_server_destroy(plas_server* srv);

/* ---------------------------------------------------------------------- */
/* diagnostics                                                            */
/* ---------------------------------------------------------------------- */
const char* plas_status_string(int status);
const char* plas_last_error(void);  /* thread-local; "" if none */
/*
 * plas_debug_inject -- host-side fault injection for tests of the error
 * paths; it never faults or stalls the GPU.  The paper has no counterpart.
 *   kind 0: clear every injection (count ignored);
 *   kind 1: the count-th device allocation made by the library from now on
 *           (workspaces, descriptor arrays, scratch) fails as if the device
 *           were out of memory: the call returns PLAS_ERR_OOM after freeing
 *           what it had allocated;
 *   kind 2: the sweep engine's next count state read-backs are frozen (the
 *           host keeps its previous copy), so its progress check sees grids
 *           that do not advance and the call returns PLAS_ERR_INTERNAL;
 *   kind 3: the next count persistent sweep launches (plas_schedule.
 *           persistent) get a zero wait limit at their grid-wide barriers:
 *           the first wait gives up at once, the launch ends early and the
 *           call returns PLAS_ERR_TIMEOUT (the GPU stays usable);
 *   kind 4: the next count checked sorts (plas_schedule.checked) get one
 *           byte of their first guard band overwritten by the host after
 *           the bands are filled: the sort returns PLAS_ERR_INTERNAL.
 * Process-wide (all threads).  Returns PLAS_OK or PLAS_ERR_INVALID_ARG
 * (unknown kind, count < 1).
 */
int plas_debug_inject(int kind, long long count);
int plas_version(void);              /* major*10000 + minor*100 + patch */

#ifdef __cplusplus
}
#endif
#endif /* PLAS_H_ */
