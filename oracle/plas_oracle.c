/*
 * PLAS oracle -- a plain, slow, obviously correct CPU implementation of the
 * Parallel Linear Assignment Sort of Morgenstern et al., "Compact 3D Scene
 * Representation via Self-Organizing Gaussian Grids" (arXiv 2312.13299),
 * and of the grid smoothness loss built next to it.
 *
 * THIS FILE IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline / reference leg may load it.  The product (the
 * CUDA library and its Python binding) never includes, links or calls it, and
 * it shares no code, header or table with the product.
 *
 * Paper passages followed (Sec. 3.1 "Sorting High Dimensional Gaussians into
 * 2D Grids" and its "Blockwise Linear Assignment" and "Organizing Gaussians
 * into a 2D Grid" paragraphs; Sec. 3.2; the supplementary "Sorting
 * performance" section):
 *   - random initial placement, then repeated low-pass target + re-assignment
 *     with a shrinking filter (Sec. 3.1, Fig. "blockwise_assignment");
 *   - blocks of side beta = phi + 1, never below 16, all shifted by a random
 *     (dy, dx) (Sec. 3.1);
 *   - one random permutation of a block's cells, cut into disjoint groups of
 *     four, shared by all blocks; each group takes the best of its 24
 *     permutations by total distance to the target (Sec. 3.1, "Blockwise
 *     Linear Assignment", Fig. "swapping_pixels");
 *   - mean L2 distance to the target after each assignment; < 0.01 %
 *     improvement -> new block shift; no further improvement -> phi *= 0.95;
 *     phi starts at w/2 - 1 and the sort stops when phi falls below 1
 *     (Sec. 3.1; threshold 1e-4 in the supplementary);
 *   - attributes normalised per channel to [0,1] and scaled by weights
 *     (Sec. 3.1 "Organizing Gaussians");
 *   - VAD = variance of the absolute differences of all neighbouring values
 *     over all channels (supplementary, "Sorting performance");
 *   - smoothness loss: deviation of each grid value from a Gaussian blur of
 *     the grid (Sec. 3.2).
 *
 * Where the paper is silent the oracle takes these readings (each also
 * listed with its reason in the design notes):
 *   - cost of a candidate assignment = sum of SQUARED L2 distances; the
 *     schedule uses the (non-squared) mean L2 distance;
 *   - blur: half-width r = floor(phi), sigma = sigma_ratio * phi, taps
 *     truncated at the grid border and renormalised by the in-range tap mass;
 *   - every block that meets the grid is re-assigned, the blocks cut by the
 *     grid border included (their groups whose four cells lie in the grid;
 *     schedule.edge_blocks = 0 keeps whole blocks only); the shift is drawn
 *     from [0, min(beta, side - beta + 1)) per axis, which is [0, beta)
 *     whenever phi0 = min(H, W)/2 - 1;
 *   - the random sources are Philox4x32-10 (Salmon et al., SC'11) driving a
 *     six-round Feistel permutation with cycle walking;
 *   - ties between permutations: the first in lexicographic order wins;
 *   - the mean L2 distance is accumulated as an integer fixed-point sum so
 *     that the schedule decision is independent of summation order.
 *
 * Floating point: compiled with -ffp-contract=off; every fused multiply-add
 * is an explicit fmaf(), every sum runs in the order written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel Random        */
/* Numbers: As Easy as 1, 2, 3").  Ten rounds; each round multiplies words 0 */
/* and 2 by the two Philox constants, crosses the high halves with words 1   */
/* and 3 and the round key; the key is bumped by the Weyl constants between  */
/* rounds.                                                                    */
/* ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream tags: which random decision a Philox counter belongs to. */
#define ORC_TAG_INIT 1u   /* initial random placement (Sec. 3.1)            */
#define ORC_TAG_SHIFT 2u  /* block shift (dy, dx) per shift epoch (Sec. 3.1) */
#define ORC_TAG_GROUP 3u  /* grouping permutation per iteration (Sec. 3.1)  */

/* ------------------------------------------------------------------------- */
/* Keyed pseudo-random permutation of [0, n): a balanced six-round Feistel    */
/* network on 2h bits (2^(2h) >= n) whose round function is the first Philox */
/* output word for counter (R, tag<<8 | round, counter_lo, counter_hi), with  */
/* cycle walking to stay inside [0, n).                                       */
/* ------------------------------------------------------------------------- */
static uint32_t orc_half_bits(uint32_t n)
{
    uint32_t m = 0;
    while (m < 32 && ((uint64_t)1 << m) < (uint64_t)n) ++m;   /* m = ceil(log2 n) */
    uint32_t h = (m + 1) / 2;
    return h == 0 ? 1 : h;
}

static uint32_t orc_feistel(uint32_t x, uint32_t h, uint64_t seed, uint32_t tag, uint64_t counter)
{
    const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t L = x >> h, R = x & mask;
    for (uint32_t round = 0; round < 6; ++round) {
        uint32_t ctr[4] = {R, (tag << 8) | round, (uint32_t)counter, (uint32_t)(counter >> 32)};
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        uint32_t F = o[0] & mask;
        uint32_t newL = R;
        uint32_t newR = L ^ F;
        L = newL;
        R = newR;
    }
    return (L << h) | R;
}

uint32_t orc_prp(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n, uint32_t x)
{
    uint32_t h = orc_half_bits(n);
    uint32_t y = orc_feistel(x, h, seed, tag, counter);
    while (y >= n) y = orc_feistel(y, h, seed, tag, counter);
    return y;
}

void orc_prp_table(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n, uint32_t* out)
{
    for (uint32_t m = 0; m < n; ++m) out[m] = orc_prp(seed, tag, counter, n, m);
}

/* ------------------------------------------------------------------------- */
/* Schedule constants (Sec. 3.1).                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
    double phi0;        /* <= 0: min(H,W)/2 - 1  (Sec. 3.1)                    */
    double shrink;      /* 0.95                  (Sec. 3.1)                    */
    double phi_min;     /* 1.0: stop when phi would fall below it (Sec. 3.1)  */
    double tol;         /* 1e-4 relative improvement (supplementary)          */
    double sigma_ratio; /* sigma = sigma_ratio * phi (paper silent)           */
    int min_block;      /* 16 (Sec. 3.1)                                      */
    int shuffle_init;   /* 1: random initial placement (Sec. 3.1)             */
    int normalize;      /* 1: per-channel [0,1] normalisation (Sec. 3.1)      */
    int target_mode;    /* 0: Gaussian target (Sec. 3.1); 1: box target      */
    long long max_iters;/* stop after this many iterations in total; 0 = none */
    int edge_blocks;    /* reading of the borders after the shift (Sec. 3.1): */
                        /* 1 (the default reading) every block that meets    */
                        /* the grid is re-assigned, those cut by the grid    */
                        /* border included: each of their groups of four     */
                        /* whose cells all lie inside the grid (the others   */
                        /* stay put); 0 only whole blocks                    */
    int pad_;
} orc_schedule;

typedef struct {
    long long it;       /* iterations done                                    */
    long long epoch;    /* block-shift epoch                                  */
    long long redraws;  /* shift redraws caused by a stall                    */
    int level;          /* index into the phi sequence                        */
    int stall;          /* 1 after one non-improving assignment               */
    int has_prev;       /* d_prev valid (0 right after a level change)        */
    int done;           /* phi fell below phi_min                             */
    double d_prev;      /* previous mean L2 distance to the target            */
    double d_last;      /* mean L2 distance of the last iteration             */
    int scale_exp;      /* fixed-point exponent k of the residual sum         */
    int pad_;
} orc_state;

static double orc_phi0(const orc_schedule* s, int H, int W)
{
    double p = s->phi0 > 0.0 ? s->phi0 : (double)(H < W ? H : W) / 2.0 - 1.0;
    if (p < s->phi_min) p = s->phi_min;   /* tiny grids: one level at phi_min */
    return p;
}

/* phi_L = phi0 * shrink^L by repeated multiplication, while phi >= phi_min. */
int orc_levels(const orc_schedule* s, int H, int W, double* phis, int cap)
{
    double p = orc_phi0(s, H, W);
    int n = 0;
    while (p >= s->phi_min) {
        if (phis && n < cap) phis[n] = p;
        ++n;
        p = s->shrink * p;
    }
    return n;
}

static int orc_block_side(int r, int min_block, int H, int W)
{
    int b = r + 1;                       /* beta = phi + 1 (Sec. 3.1) */
    if (b < min_block) b = min_block;    /* never below 16            */
    if (b > H) b = H;
    if (b > W) b = W;
    return b;
}

void orc_shift(uint64_t seed, uint64_t epoch, int beta, int H, int W, int* dy, int* dx)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)epoch, (uint32_t)(epoch >> 32), ORC_TAG_SHIFT, 0u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    int my = beta < H - beta + 1 ? beta : H - beta + 1;
    int mx = beta < W - beta + 1 ? beta : W - beta + 1;
    *dy = (int)(((uint64_t)o[0] * (uint64_t)my) >> 32);
    *dx = (int)(((uint64_t)o[1] * (uint64_t)mx) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Low-pass target (Sec. 3.1): separable Gaussian, taps k_j for j=-r..r,      */
/* truncated at the border and renormalised by the in-range tap mass.         */
/* ------------------------------------------------------------------------- */
void orc_taps(int r, double sigma, float* taps /* 2r+1 */)
{
    for (int j = -r; j <= r; ++j) {
        double q = (double)j * (double)j;
        double den = 2.0 * sigma * sigma;
        taps[j + r] = (float)exp(-q / den);
    }
}

/* One 1-D pass over 'len' samples at stride 'step' (in floats). */
static float orc_fir_at(const float* src, long step, int len, int pos, int r, const float* taps)
{
    int jlo = -r, jhi = r;
    if (pos + jlo < 0) jlo = -pos;
    if (pos + jhi > len - 1) jhi = len - 1 - pos;
    float acc = 0.0f, nrm = 0.0f;
    for (int j = jlo; j <= jhi; ++j) acc = fmaf(taps[j + r], src[(long)(pos + j) * step], acc);
    for (int j = jlo; j <= jhi; ++j) nrm = nrm + taps[j + r];
    return acc / nrm;
}

/* G: H x W cells, cell stride gs floats, features at [0, D).  T: H x W x D.
 * The first pass runs along y (columns), the second along x (rows); each
 * divides by its own in-range tap mass. */
void orc_blur(const float* G, int gs, int H, int W, int D, int r, double sigma, float* T)
{
    float* taps = (float*)malloc(sizeof(float) * (size_t)(2 * r + 1));
    float* H1 = (float*)malloc(sizeof(float) * (size_t)H * W * D);
    orc_taps(r, sigma, taps);
    /* pass 1: along y */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d)
                H1[((long)y * W + x) * D + d] =
                    orc_fir_at(G + (long)x * gs + d, (long)W * gs, H, y, r, taps);
    /* pass 2: along x */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d)
                T[((long)y * W + x) * D + d] =
                    orc_fir_at(H1 + (long)y * W * D + d, D, W, x, r, taps);
    free(H1);
    free(taps);
}

/* ------------------------------------------------------------------------- */
/* The 24 permutations of 4 positions in lexicographic order (Fig.            */
/* "swapping_pixels": brute force over all 24).  Built by counting, not by a  */
/* stored table.                                                              */
/* ------------------------------------------------------------------------- */
static int orc_perm24[24][4];
static int orc_perm24_ready = 0;

static void orc_build_perm24(void)
{
    if (orc_perm24_ready) return;
    int n = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d)
                    if (a != b && a != c && a != d && b != c && b != d && c != d) {
                        orc_perm24[n][0] = a; orc_perm24[n][1] = b;
                        orc_perm24[n][2] = c; orc_perm24[n][3] = d;
                        ++n;
                    }
    orc_perm24_ready = 1;
}

void orc_perm24_table(int* out /* 96 */)
{
    orc_build_perm24();
    memcpy(out, orc_perm24, sizeof(orc_perm24));
}

/* C[i*4+j] = cost of putting element i at position j.  Returns the
 * lexicographic index of the first permutation of minimum total cost. */
int orc_best_perm(const float* C)
{
    orc_build_perm24();
    int best = 0;
    float best_cost = 0.0f;
    for (int s = 0; s < 24; ++s) {
        const int* p = orc_perm24[s];
        float cost = ((C[0 * 4 + p[0]] + C[1 * 4 + p[1]]) + C[2 * 4 + p[2]]) + C[3 * 4 + p[3]];
        if (s == 0 || cost < best_cost) {
            best = s;
            best_cost = cost;
        }
    }
    return best;
}

/* Squared L2 distance between a grid cell and a target cell, d ascending. */
static float orc_sqdist(const float* g, const float* t, int D)
{
    float acc = 0.0f;
    for (int d = 0; d < D; ++d) {
        float delta = g[d] - t[d];
        acc = fmaf(delta, delta, acc);
    }
    return acc;
}

/* ------------------------------------------------------------------------- */
/* Feature preparation (Sec. 3.1 "Organizing Gaussians into a 2D Grid").      */
/* ------------------------------------------------------------------------- */
/* Exact per-channel min / max.  -0 is read as +0 (v + 0.0f) so the result
 * does not depend on which of two equal zeros comes first. */
void orc_minmax(const float* x, long N, int D, float* lo, float* hi)
{
    for (int d = 0; d < D; ++d) {
        float a = x[d] + 0.0f, b = x[d] + 0.0f;
        for (long i = 1; i < N; ++i) {
            float v = x[i * D + d] + 0.0f;
            if (v < a) a = v;
            if (v > b) b = v;
        }
        lo[d] = a;
        hi[d] = b;
    }
}

void orc_normalize(const float* x, long N, int D, const float* w, int normalize, float* F)
{
    float* lo = (float*)malloc(sizeof(float) * (size_t)D);
    float* hi = (float*)malloc(sizeof(float) * (size_t)D);
    orc_minmax(x, N, D, lo, hi);
    for (long i = 0; i < N; ++i)
        for (int d = 0; d < D; ++d) {
            float wd = w ? w[d] : 1.0f;
            float v = x[i * D + d];
            if (normalize) {
                if (hi[d] == lo[d]) {
                    F[i * D + d] = 0.0f;
                } else {
                    float u = (v - lo[d]) / (hi[d] - lo[d]);
                    F[i * D + d] = wd * u;
                }
            } else {
                F[i * D + d] = wd * v;
            }
        }
    free(lo);
    free(hi);
}

/* Fixed-point exponent k of the residual sum S = sum_p rint(e_p * 2^k):
 * the largest k <= 32 with N * E * 2^k < 2^62, where E bounds every e_p. */
int orc_scale_exp(const float* x, long N, int D, const float* w, int normalize)
{
    float* lo = (float*)malloc(sizeof(float) * (size_t)(D > 0 ? D : 1));
    float* hi = (float*)malloc(sizeof(float) * (size_t)(D > 0 ? D : 1));
    if (N > 0) orc_minmax(x, N, D, lo, hi);
    double e2 = 0.0;
    for (int d = 0; d < D; ++d) {
        double span = normalize ? 1.0 : ((N > 0) ? (double)hi[d] - (double)lo[d] : 0.0);
        double s = (double)(w ? w[d] : 1.0f) * span;
        e2 = e2 + s * s;
    }
    free(lo);
    free(hi);
    double m = (double)N * sqrt(e2);
    int k = 32;
    while (k > 0 && ldexp(m, k) >= 0x1p62) --k;
    return k;
}

/* ------------------------------------------------------------------------- */
/* The sort (Sec. 3.1).                                                       */
/*   x        N x D input attributes (N = H*W), row i = Gaussian i           */
/*   perm_in  optional N start permutation (position p holds Gaussian        */
/*            perm_in[p]); required when resuming                            */
/*   st       in: start state when resume != 0; out: final state             */
/*   perm_out N: Gaussian index at each grid position                        */
/*   trace_S / trace_level: per-iteration residual sum and level (optional) */
/*   T_out    optional H x W x D: the target of the last iteration           */
/* Returns the number of iterations run in this call, or -1 on bad input.    */
/* ------------------------------------------------------------------------- */
void orc_box_target(const float* G, int gs, int H, int W, int D, int r, int s_exp, float* T);
int orc_box_exp(const float* x, long N, int D, const float* w, int normalize);

long long orc_sort(const float* x, int H, int W, int D, const float* w, uint64_t seed,
                   const orc_schedule* sch, const int32_t* perm_in, int resume, orc_state* st,
                   int32_t* perm_out, long long* trace_S, int* trace_level, long long trace_cap,
                   float* T_out)
{
    if (H < 0 || W < 0 || D < 1) return -1;
    const long N = (long)H * W;
    if (resume && !perm_in) return -1;
    if (N == 0) {
        memset(st, 0, sizeof(*st));
        st->done = 1;
        return 0;
    }
    orc_build_perm24();

    /* per-channel normalisation and weights (Sec. 3.1) */
    float* F = (float*)malloc(sizeof(float) * (size_t)N * D);
    orc_normalize(x, N, D, w, sch->normalize, F);

    /* working grid: features + the Gaussian index */
    const int gs = D + 1;
    float* G = (float*)malloc(sizeof(float) * (size_t)N * gs);
    int32_t* gid = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (perm_in) {
        for (long p = 0; p < N; ++p) gid[p] = perm_in[p];
    } else if (sch->shuffle_init) {
        /* random initial placement: Gaussian i goes to position pi0(i) */
        for (long i = 0; i < N; ++i)
            gid[orc_prp(seed, ORC_TAG_INIT, 0, (uint32_t)N, (uint32_t)i)] = (int32_t)i;
    } else {
        for (long p = 0; p < N; ++p) gid[p] = (int32_t)p;
    }
    for (long p = 0; p < N; ++p) {
        for (int d = 0; d < D; ++d) G[p * gs + d] = F[(long)gid[p] * D + d];
    }

    /* schedule */
    int nlev = orc_levels(sch, H, W, NULL, 0);
    double* phis = (double*)malloc(sizeof(double) * (size_t)nlev);
    orc_levels(sch, H, W, phis, nlev);
    orc_state s;
    if (resume) {
        s = *st;
    } else {
        memset(&s, 0, sizeof(s));
    }
    s.scale_exp = orc_scale_exp(x, N, D, w, sch->normalize);
    const int box_exp = sch->target_mode == 1 ? orc_box_exp(x, N, D, w, sch->normalize) : 0;
    const double denom = ldexp((double)N, s.scale_exp);
    if (s.level >= nlev) s.done = 1;

    float* T = (float*)malloc(sizeof(float) * (size_t)N * D);
    float* Gn = (float*)malloc(sizeof(float) * (size_t)N * gs);
    int32_t* gidn = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    uint32_t* pi = NULL;
    long long ran = 0;

    while (!s.done && !(sch->max_iters > 0 && s.it >= sch->max_iters)) {
        const double phi = phis[s.level];
        const int r = (int)floor(phi);
        const double sigma = sch->sigma_ratio * phi;
        const int beta = orc_block_side(r, sch->min_block, H, W);

        /* (1) idealised target: low-pass filter of the current grid */
        if (sch->target_mode == 1)
            orc_box_target(G, gs, H, W, D, r, box_exp, T);
        else
            orc_blur(G, gs, H, W, D, r, sigma, T);

        /* (2) blocks shifted by a random (dy, dx): the whole blocks from
         *     (dy, dx) on, or (edge_blocks) every block that meets the grid */
        int dy, dx;
        orc_shift(seed, (uint64_t)s.epoch, beta, H, W, &dy, &dx);
        int nby = (H - dy) / beta, nbx = (W - dx) / beta;
        if (sch->edge_blocks) {
            if (dy > 0) dy -= beta;
            if (dx > 0) dx -= beta;
            nby = (H - dy + beta - 1) / beta;
            nbx = (W - dx + beta - 1) / beta;
        }

        /* (3) one random permutation of a block's cells, shared by all blocks */
        const uint32_t nb2 = (uint32_t)beta * (uint32_t)beta;
        pi = (uint32_t*)realloc(pi, sizeof(uint32_t) * nb2);
        orc_prp_table(seed, ORC_TAG_GROUP, (uint64_t)s.it, nb2, pi);
        const long ngroups = (long)(nb2 / 4);

        /* (4) every group of four takes its best permutation (brute force) */
        memcpy(Gn, G, sizeof(float) * (size_t)N * gs);
        memcpy(gidn, gid, sizeof(int32_t) * (size_t)N);
#pragma omp parallel for schedule(static)
        for (long bg = 0; bg < (long)nby * nbx * ngroups; ++bg) {
            const long blk = bg / ngroups, g = bg % ngroups;
            const int oy = dy + (int)(blk / nbx) * beta, ox = dx + (int)(blk % nbx) * beta;
            long pos[4];
            int inside = 1;
            for (int k = 0; k < 4; ++k) {
                uint32_t l = pi[4 * g + k];
                const int y = oy + (int)(l / (uint32_t)beta), x = ox + (int)(l % (uint32_t)beta);
                inside = inside && y >= 0 && y < H && x >= 0 && x < W;
                pos[k] = (long)y * W + x;
            }
            if (!inside) continue; /* only with edge_blocks: a cell beyond the border */
            float C[16];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    C[i * 4 + j] = orc_sqdist(G + pos[i] * gs, T + pos[j] * D, D);
            const int* best = orc_perm24[orc_best_perm(C)];
            for (int i = 0; i < 4; ++i) {
                long dst = pos[best[i]];
                memcpy(Gn + dst * gs, G + pos[i] * gs, sizeof(float) * (size_t)gs);
                gidn[dst] = gid[pos[i]];
            }
        }
        { float* t = G; G = Gn; Gn = t; }
        { int32_t* t = gid; gid = gidn; gidn = t; }

        /* (5) mean L2 distance between the grid and the target, as an
         *     integer fixed-point sum */
        long long S = 0;
#pragma omp parallel for schedule(static) reduction(+ : S)
        for (long p = 0; p < N; ++p) {
            float e = sqrtf(orc_sqdist(G + p * gs, T + p * D, D));
            S += llrint((double)e * ldexp(1.0, s.scale_exp));
        }
        const double d = (double)S / denom;
        if (trace_S && s.it < trace_cap) trace_S[s.it] = S;
        if (trace_level && s.it < trace_cap) trace_level[s.it] = s.level;

        /* (6) schedule: improvement below tol -> new shift; again -> shrink */
        int improved = !s.has_prev || (d < s.d_prev && (s.d_prev - d) >= sch->tol * s.d_prev);
        if (improved) {
            s.stall = 0;
            s.d_prev = d;
            s.has_prev = 1;
        } else if (s.stall == 0) {
            s.stall = 1;
            s.epoch += 1;
            s.redraws += 1;
            s.d_prev = d;
            s.has_prev = 1;
        } else {
            s.level += 1;
            s.stall = 0;
            s.epoch += 1;
            s.has_prev = 0;
            s.d_prev = 0.0;
        }
        s.d_last = d;
        s.it += 1;
        ++ran;
        if (s.level >= nlev) s.done = 1;
    }

    if (T_out) memcpy(T_out, T, sizeof(float) * (size_t)N * D);
    for (long p = 0; p < N; ++p) perm_out[p] = gid[p];
    *st = s;
    free(pi);
    free(gidn);
    free(Gn);
    free(T);
    free(phis);
    free(gid);
    free(G);
    free(F);
    return ran;
}

/* ------------------------------------------------------------------------- */
/* Box target (a fast low-pass variant of the target, Sec. 3.1 asks only for */
/* a low-pass filter whose radius shrinks): the mean of the in-range cells   */
/* of the (2r+1) x (2r+1) window, on features in fixed point.                */
/*   q = rint(F * 2^s) (int64), S = sum of q over the in-range window,       */
/*   n = in-range cells, T = ((float)S / (float)n) * 2^-s   (FP32)           */
/* s = the largest value <= 40 with B * 2^s <= 2^31, B = max_d |w_d| (times  */
/* max(|lo_d|, |hi_d|) without normalisation) bounding every |F|.  The sums  */
/* are exact integers, so the order of summation is free; here they are      */
/* sliding window sums along y, then along x.                                */
/* ------------------------------------------------------------------------- */
int orc_box_exp(const float* x, long N, int D, const float* w, int normalize)
{
    double B = 0.0;
    float* lo = (float*)malloc(sizeof(float) * (size_t)(D > 0 ? D : 1));
    float* hi = (float*)malloc(sizeof(float) * (size_t)(D > 0 ? D : 1));
    if (N > 0) orc_minmax(x, N, D, lo, hi);
    for (int d = 0; d < D; ++d) {
        double m = fabs((double)(w ? w[d] : 1.0f));
        if (!normalize) m *= fmax(fabs((double)lo[d]), fabs((double)hi[d]));
        if (m > B) B = m;
    }
    free(lo);
    free(hi);
    int s = 40;
    while (s > -60 && ldexp(B, s) > 0x1p31) --s;
    return s;
}

void orc_box_target(const float* G, int gs, int H, int W, int D, int r, int s_exp, float* T)
{
    const long N = (long)H * W;
    long long* q = (long long*)malloc(sizeof(long long) * (size_t)N * D);
    long long* sy = (long long*)malloc(sizeof(long long) * (size_t)N * D);
    for (long p = 0; p < N; ++p)
        for (int d = 0; d < D; ++d) q[p * D + d] = llrint(ldexp((double)G[p * gs + d], s_exp));
    /* window sums along y: rows [y - r, y + r] within the grid */
#pragma omp parallel for schedule(static)
    for (long xd = 0; xd < (long)W * D; ++xd) {
        const int x = (int)(xd / D), d = (int)(xd % D);
        long long run = 0;
        for (int y = 0; y <= r && y < H; ++y) run += q[((long)y * W + x) * D + d];
        for (int y = 0; y < H; ++y) {
            sy[((long)y * W + x) * D + d] = run;
            if (y + r + 1 < H) run += q[((long)(y + r + 1) * W + x) * D + d];
            if (y - r >= 0) run -= q[((long)(y - r) * W + x) * D + d];
        }
    }
    /* window sums of those along x, then the mean over the in-range cells */
#pragma omp parallel for schedule(static)
    for (long yd = 0; yd < (long)H * D; ++yd) {
        const int y = (int)(yd / D), d = (int)(yd % D);
        const int ny = (y + r < H - 1 ? y + r : H - 1) - (y - r > 0 ? y - r : 0) + 1;
        long long run = 0;
        for (int x = 0; x <= r && x < W; ++x) run += sy[((long)y * W + x) * D + d];
        for (int x = 0; x < W; ++x) {
            const int nx = (x + r < W - 1 ? x + r : W - 1) - (x - r > 0 ? x - r : 0) + 1;
            const float mean = (float)run / (float)(ny * nx);
            T[((long)y * W + x) * D + d] = ldexpf(mean, -s_exp);
            if (x + r + 1 < W) run += sy[((long)y * W + x + r + 1) * D + d];
            if (x - r >= 0) run -= sy[((long)y * W + x - r) * D + d];
        }
    }
    free(sy);
    free(q);
}

/* Box target of a given arrangement at a given radius (per-step checks). */
void orc_target_box(const float* x, int H, int W, int D, const float* w, int normalize,
                    const int32_t* perm, double phi, float* T)
{
    const long N = (long)H * W;
    float* F = (float*)malloc(sizeof(float) * (size_t)N * D);
    float* G = (float*)malloc(sizeof(float) * (size_t)N * D);
    orc_normalize(x, N, D, w, normalize, F);
    for (long p = 0; p < N; ++p)
        for (int d = 0; d < D; ++d) G[p * D + d] = F[(long)perm[p] * D + d];
    orc_box_target(G, D, H, W, D, (int)floor(phi), orc_box_exp(x, N, D, w, normalize), T);
    free(G);
    free(F);
}

/* Target of a given arrangement at a given level (for per-step checks). */
void orc_target(const float* x, int H, int W, int D, const float* w, int normalize,
                const int32_t* perm, double phi, double sigma_ratio, float* T)
{
    const long N = (long)H * W;
    float* F = (float*)malloc(sizeof(float) * (size_t)N * D);
    float* G = (float*)malloc(sizeof(float) * (size_t)N * D);
    orc_normalize(x, N, D, w, normalize, F);
    for (long p = 0; p < N; ++p)
        for (int d = 0; d < D; ++d) G[p * D + d] = F[(long)perm[p] * D + d];
    orc_blur(G, D, H, W, D, (int)floor(phi), sigma_ratio * phi, T);
    free(G);
    free(F);
}

/* Carried attributes follow the permutation (Sec. 3, Fig. "grid2splat"). */
void orc_gather(const float* src, long N, int C, const int32_t* perm, float* dst)
{
    for (long p = 0; p < N; ++p)
        for (int c = 0; c < C; ++c) dst[p * C + c] = src[(long)perm[p] * C + c];
}

/* ------------------------------------------------------------------------- */
/* Grid quality metrics.  Mean neighbour L2 over all horizontal and vertical  */
/* pairs; VAD (supplementary): population variance of |a - b| over all       */
/* neighbouring pairs and all channels, on values multiplied by 'scale'.     */
/* ------------------------------------------------------------------------- */
void orc_metrics(const float* g, int H, int W, int D, double scale, double* mean_nl2, double* vad)
{
    double sum_l2 = 0.0, s1 = 0.0, s2 = 0.0;
    long npairs = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int dir = 0; dir < 2; ++dir) {
                int y2 = y + (dir == 1), x2 = x + (dir == 0);
                if (y2 >= H || x2 >= W) continue;
                const float* a = g + ((long)y * W + x) * D;
                const float* b = g + ((long)y2 * W + x2) * D;
                double q = 0.0;
                for (int d = 0; d < D; ++d) {
                    double diff = (double)a[d] - (double)b[d];
                    q += diff * diff;
                    double ad = fabs(diff * scale);
                    s1 += ad;
                    s2 += ad * ad;
                }
                sum_l2 += sqrt(q);
                ++npairs;
            }
    *mean_nl2 = npairs ? sum_l2 / (double)npairs : 0.0;
    double nv = (double)npairs * (double)D;
    *vad = npairs ? (s2 / nv - (s1 / nv) * (s1 / nv)) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Smoothness loss (Sec. 3.2) in FP64.  x: H x W x C channel-last.  B is a    */
/* separable Gaussian of 'ksize' taps (sigma), normalised to sum 1 over the   */
/* full window, zero padding.  r = x - Bx;  L = (1/M) sum_c lam_c sum r^2;    */
/* dL/dx = (2 g / M) lam_c (r - B^T r), and B^T = B for symmetric taps with   */
/* zero padding.                                                              */
/* ------------------------------------------------------------------------- */
static void orc_blur64(const double* in, int H, int W, int C, const double* b, int h, double* out)
{
    double* tmp = (double*)malloc(sizeof(double) * (size_t)H * W * C);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int j = -h; j <= h; ++j) {
                    int xx = x + j;
                    if (xx < 0 || xx >= W) continue;
                    acc += b[j + h] * in[((long)y * W + xx) * C + c];
                }
                tmp[((long)y * W + x) * C + c] = acc;
            }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int j = -h; j <= h; ++j) {
                    int yy = y + j;
                    if (yy < 0 || yy >= H) continue;
                    acc += b[j + h] * tmp[((long)yy * W + x) * C + c];
                }
                out[((long)y * W + x) * C + c] = acc;
            }
    free(tmp);
}

void orc_smooth_taps64(double sigma, int ksize, double* b)
{
    int h = ksize / 2;
    double sum = 0.0;
    for (int j = -h; j <= h; ++j) {
        b[j + h] = exp(-((double)j * (double)j) / (2.0 * sigma * sigma));
        sum += b[j + h];
    }
    for (int j = 0; j < 2 * h + 1; ++j) b[j] /= sum;
}

/* x given in FP64 so finite-difference checks can perturb it exactly. */
double orc_smooth_loss64(const double* x, int H, int W, int C, double sigma, int ksize,
                         const double* lam, double grad_loss, double* grad /* or NULL */)
{
    const long M = (long)H * W * C;
    const int h = ksize / 2;
    double* b = (double*)malloc(sizeof(double) * (size_t)(2 * h + 1));
    double* bx = (double*)malloc(sizeof(double) * (size_t)M);
    double* rr = (double*)malloc(sizeof(double) * (size_t)M);
    orc_smooth_taps64(sigma, ksize, b);
    orc_blur64(x, H, W, C, b, h, bx);
    double L = 0.0;
    for (long i = 0; i < M; ++i) {
        int c = (int)(i % C);
        double l = lam ? lam[c] : 1.0;
        rr[i] = x[i] - bx[i];
        L += l * rr[i] * rr[i];
    }
    L /= (double)M;
    if (grad) {
        double* wr = (double*)malloc(sizeof(double) * (size_t)M);
        double* bwr = (double*)malloc(sizeof(double) * (size_t)M);
        for (long i = 0; i < M; ++i) wr[i] = (lam ? lam[i % C] : 1.0) * rr[i];
        orc_blur64(wr, H, W, C, b, h, bwr);
        for (long i = 0; i < M; ++i) grad[i] = 2.0 * grad_loss / (double)M * (wr[i] - bwr[i]);
        free(bwr);
        free(wr);
    }
    free(rr);
    free(bx);
    free(b);
    return L;
}

/* Huber form of the smoothness loss (Sec. 3.2: the deviation of each cell
 * from the blurred grid is penalised with a Huber loss, less sensitive to
 * outliers than the squared error):
 *   h(r) = r^2 / 2 for |r| <= delta, delta * (|r| - delta / 2) otherwise,
 *   L = (1/M) sum lam_c h(x - Bx),
 *   dL/dx = (g/M) (psi - B psi),  psi = lam_c * clamp(x - Bx, -delta, delta)
 * (B symmetric with zero padding, so B^T = B).  delta > 0. */
double orc_smooth_loss64_huber(const double* x, int H, int W, int C, double sigma, int ksize,
                               const double* lam, double delta, double grad_loss,
                               double* grad /* or NULL */)
{
    const long M = (long)H * W * C;
    const int h = ksize / 2;
    double* b = (double*)malloc(sizeof(double) * (size_t)(2 * h + 1));
    double* bx = (double*)malloc(sizeof(double) * (size_t)M);
    double* psi = (double*)malloc(sizeof(double) * (size_t)M);
    orc_smooth_taps64(sigma, ksize, b);
    orc_blur64(x, H, W, C, b, h, bx);
    double L = 0.0;
    for (long i = 0; i < M; ++i) {
        const double l = lam ? lam[i % C] : 1.0;
        const double r = x[i] - bx[i];
        const double a = fabs(r);
        L += l * (a <= delta ? 0.5 * r * r : delta * (a - 0.5 * delta));
        psi[i] = l * (r < -delta ? -delta : (r > delta ? delta : r));
    }
    L /= (double)M;
    if (grad) {
        double* bpsi = (double*)malloc(sizeof(double) * (size_t)M);
        orc_blur64(psi, H, W, C, b, h, bpsi);
        for (long i = 0; i < M; ++i) grad[i] = grad_loss / (double)M * (psi[i] - bpsi[i]);
        free(bpsi);
    }
    free(psi);
    free(bx);
    free(b);
    return L;
}

/* Quantisation of Sec. 3.4: clip channel c to [lo_c, hi_c], map linearly to
 * [0, 1] and round to the nearest of q_c equally spaced values (FP32, the
 * integer decided by rounding half to even; hi == lo gives 0).  Written
 * out as the definition; fmaxf/fminf send NaN to the bound. */
void orc_quantize(const float* x, long n, int C, const float* lo, const float* hi, const int* q,
                  unsigned short* codes)
{
    for (long i = 0; i < n * C; ++i) {
        const int c = (int)(i % C);
        int k = 0;
        if (hi[c] > lo[c]) {
            const float v = fminf(fmaxf(x[i], lo[c]), hi[c]);
            const float t = (v - lo[c]) / (hi[c] - lo[c]);
            k = (int)rintf(t * (float)(q[c] - 1));
        }
        codes[i] = (unsigned short)k;
    }
}

/* The value a code stands for (the inverse step of Sec. 3.4): level k of
 * channel c is lo_c + k * ((hi_c - lo_c) / (q_c - 1)) in FP32 (lo_c when the
 * range is degenerate). */
void orc_dequantize(const unsigned short* codes, long n, int C, const float* lo, const float* hi,
                    const int* q, float* out)
{
    for (long i = 0; i < n * C; ++i) {
        const int c = (int)(i % C);
        const float step = hi[c] > lo[c] ? (hi[c] - lo[c]) / (float)(q[c] - 1) : 0.0f;
        out[i] = lo[c] + (float)codes[i] * step;
    }
}

/* Activation of raw 3DGS parameters into the sort features (Sec. 3.1: the
 * sort uses the values the renderer sees; Sec. 3.3: coordinates go through
 * x = sign(v) (exp(|v|) - 1)).  Row layout of raw (stride floats apart):
 * xyz 0-2, log-scale 3-5, quaternion 6-9, opacity logit 10, DC 11-13.
 * Evaluated in FP64 and rounded once to FP32. */
void orc_activate_3dgs(const float* raw, long n, int stride, float* out)
{
    for (long i = 0; i < n; ++i) {
        const float* r = raw + i * stride;
        float* o = out + i * 14;
        for (int k = 0; k < 3; ++k) {
            const double v = r[k];
            const double m = exp(fabs(v)) - 1.0;
            o[k] = (float)(v < 0 ? -m : m);
        }
        for (int k = 3; k < 6; ++k) o[k] = (float)exp((double)r[k]);
        double nn = 0.0;
        for (int k = 6; k < 10; ++k) nn += (double)r[k] * (double)r[k];
        nn = sqrt(nn);
        for (int k = 6; k < 10; ++k) o[k] = nn > 0 ? (float)((double)r[k] / nn) : 0.0f;
        o[10] = (float)(1.0 / (1.0 + exp(-(double)r[10])));
        for (int k = 11; k < 14; ++k) o[k] = r[k];
    }
}

/* Largest square grid that the Gaussians fill (Sec. 3.1: the ones with the
 * lowest opacity that do not fit are pruned): side = floor(sqrt(n)); keep
 * receives the side^2 indices with the largest opacity logits (ties to the
 * lower index; -0 equals +0; NaN ranks lowest), in ascending index order.
 * Written as a plain sort.  Returns side. */
static const float* g_sel_op;
static long g_sel_stride;
static int sel_cmp(const void* a, const void* b)
{
    const long i = *(const long*)a, j = *(const long*)b;
    const float x = g_sel_op[i * g_sel_stride], y = g_sel_op[j * g_sel_stride];
    const int xn = x != x, yn = y != y;
    if (xn != yn) return xn ? 1 : -1;         /* NaN last */
    if (!xn && x != y) return x > y ? -1 : 1; /* larger logit first (-0 == +0) */
    return i < j ? -1 : (i > j ? 1 : 0);      /* then the lower index */
}
static int idx_cmp(const void* a, const void* b)
{
    const long i = *(const long*)a, j = *(const long*)b;
    return i < j ? -1 : (i > j ? 1 : 0);
}
int orc_grid_select(const float* opacity, long n, int stride, int* keep)
{
    long side = (long)floor(sqrt((double)n));
    while (side * side > n) --side;
    while ((side + 1) * (side + 1) <= n) ++side;
    long* idx = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) idx[i] = i;
    g_sel_op = opacity;
    g_sel_stride = stride;
    qsort(idx, (size_t)n, sizeof(long), sel_cmp);
    qsort(idx, (size_t)(side * side), sizeof(long), idx_cmp);
    for (long i = 0; i < side * side; ++i) keep[i] = (int)idx[i];
    free(idx);
    return (int)side;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the parallel loops use from now on (test and timing plumbing: the
 * results do not depend on it, every parallel loop writes independent
 * outputs or sums integers). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
