// plas_api.cu -- host side of the C ABI declared in include/plas.h: argument
// checks, workspace layout, the per-level blur tables, and the iteration
// loop of the PLAS sort (Sec. 3.1 of Morgenstern et al., arXiv 2312.13299).
//
// The loop is device-driven: the schedule (stall test, block-shift redraw,
// radius shrink, termination) runs on the device at the end of every
// assignment launch, and kernels of a finished level return immediately.  The
// host only enqueues batches of iterations for the level it last saw and
// reads the 64-byte state back once per batch (one batch of look-ahead), so
// the GPU never waits for a host decision inside a level.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/plas.h"
#include "plas_kernels.h"

namespace plas {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define PLAS_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(PLAS_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

static int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PLAS_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return PLAS_OK;
}

static int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 152;
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static bool channels_supported(int D) {
    return (D >= 1 && D <= 16) || D == 20 || D == 24 || D == 32 || D == 48 || D == 64;
}

// ---------------------------------------------------------------------------
// schedule geometry (Sec. 3.1): phi_L = phi0 * shrink^L while >= phi_min;
// r = floor(phi); beta = min(max(r + 1, min_block), H, W); sigma =
// sigma_ratio * phi; taps k_j = (float) exp(-j^2 / (2 sigma^2)).
// ---------------------------------------------------------------------------
struct Geometry {
    std::vector<LevelDesc> lv;
    std::vector<float> table;  // padded taps per level (norms filled on device)
    size_t table_floats = 0;
};

static double start_radius(const plas_schedule& s, int H, int W) {
    double p = s.phi0 > 0.0 ? s.phi0 : (double)std::min(H, W) / 2.0 - 1.0;
    if (p < s.phi_min) p = s.phi_min;
    return p;
}

static int count_levels(const plas_schedule& s, int H, int W) {
    double p = start_radius(s, H, W);
    int n = 0;
    while (p >= s.phi_min && n < 100000) {
        ++n;
        p = s.shrink * p;
    }
    return n;
}

static void padded_taps(int r, int rcap, double sigma, int* rp, int* ntp, std::vector<float>& out) {
    const int X = kFirX;
    const int rr = std::min(r, rcap);
    *rp = (rr + X - 1) / X * X;
    *ntp = (*rp + rr + 1 + X - 1) / X * X;
    out.assign((size_t)*ntp, 0.0f);
    for (int j = -rr; j <= rr; ++j) {
        double q = (double)j * (double)j;
        double den = 2.0 * sigma * sigma;
        out[(size_t)(*rp + j)] = (float)std::exp(-q / den);
    }
}

static Geometry build_geometry(const plas_schedule& s, int H, int W) {
    Geometry g;
    const int nlev = count_levels(s, H, W);
    double phi = start_radius(s, H, W);
    size_t off = 0;
    std::vector<float> tx, ty;
    for (int L = 0; L < nlev; ++L) {
        LevelDesc d{};
        d.phi = phi;
        d.r = (int)std::floor(phi);
        int b = std::max(d.r + 1, s.min_block);
        b = std::min(b, H);
        b = std::min(b, W);
        d.beta = b;
        const double sigma = s.sigma_ratio * phi;
        padded_taps(d.r, W - 1, sigma, &d.rpx, &d.ntpx, tx);
        d.rx = std::min(d.r, W - 1);
        padded_taps(d.r, H - 1, sigma, &d.rpy, &d.ntpy, ty);
        d.ry = std::min(d.r, H - 1);
        d.off_tx = (long long)off; off += align_up((size_t)d.ntpx, 4);
        d.off_ty = (long long)off; off += align_up((size_t)d.ntpy, 4);
        d.off_nx = (long long)off; off += align_up((size_t)W, 4);
        d.off_ny = (long long)off; off += align_up((size_t)H, 4);
        g.table.resize(off, 0.0f);
        std::copy(tx.begin(), tx.end(), g.table.begin() + d.off_tx);
        std::copy(ty.begin(), ty.end(), g.table.begin() + d.off_ty);
        g.lv.push_back(d);
        phi = s.shrink * phi;
    }
    g.table_floats = off;
    return g;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Workspace {
    DevState* st;
    float* G;
    float* T;
    float* H1;
    uint32_t* pi;
    LevelDesc* lv;
    float* table;
    double* macc;
};

static size_t workspace_layout(int H, int W, int D, int nlev, size_t table_floats,
                               Workspace* ws, char* base) {
    const long long N = (long long)H * W;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return base ? (void*)(base + o) : nullptr;
    };
    Workspace w{};
    w.st = (DevState*)take(sizeof(DevState));
    w.G = (float*)take(sizeof(float) * (size_t)N * grid_stride(D));
    w.T = (float*)take(sizeof(float) * (size_t)N * target_stride(D));
    w.H1 = (float*)take(sizeof(float) * (size_t)N * D);
    w.pi = (uint32_t*)take(sizeof(uint32_t) * (size_t)std::max<long long>(N, 4));
    w.lv = (LevelDesc*)take(sizeof(LevelDesc) * (size_t)nlev);
    w.table = (float*)take(sizeof(float) * table_floats);
    w.macc = (double*)take(sizeof(double) * 4);
    if (ws) *ws = w;
    return off;
}

static size_t sort_workspace_bytes(int H, int W, int D, const plas_schedule& s) {
    Geometry g = build_geometry(s, H, W);
    return workspace_layout(H, W, D, (int)g.lv.size(), g.table_floats, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// pinned staging for the state poll (one per host thread)
// ---------------------------------------------------------------------------
struct PollBuf {
    DevState* h = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int device = -1;
    ~PollBuf() {
        // process teardown: the CUDA context may already be gone; leak quietly
    }
};
static thread_local PollBuf g_poll;

static int poll_buffers(DevState** h, cudaEvent_t* ev) {
    int dev = 0;
    PLAS_CUDA(cudaGetDevice(&dev));
    if (g_poll.h == nullptr || g_poll.device != dev) {
        void* p = nullptr;
        PLAS_CUDA(cudaMallocHost(&p, 2 * sizeof(DevState)));
        g_poll.h = (DevState*)p;
        PLAS_CUDA(cudaEventCreateWithFlags(&g_poll.ev[0], cudaEventDisableTiming));
        PLAS_CUDA(cudaEventCreateWithFlags(&g_poll.ev[1], cudaEventDisableTiming));
        g_poll.device = dev;
    }
    *h = g_poll.h;
    ev[0] = g_poll.ev[0];
    ev[1] = g_poll.ev[1];
    return PLAS_OK;
}

// ---------------------------------------------------------------------------
// profiling: CUDA events at kernel boundaries of one batch
// ---------------------------------------------------------------------------
struct Profiler {
    bool on = false;
    struct Mark {
        cudaEvent_t a, b;
        int cls;
        double bytes, flops;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    plas_kernel_stat k[PLAS_K_COUNT] = {};

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(cudaStream_t s, cudaEvent_t* a) {
        if (!on) return;
        *a = get();
        cudaEventRecord(*a, s);
    }
    void end(cudaStream_t s, cudaEvent_t a, int cls, double bytes, double flops) {
        if (!on) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, s);
        marks.push_back({a, b, cls, bytes, flops});
    }
    // harvest every mark (the caller has synchronised the stream)
    void harvest() {
        for (auto& m : marks) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, m.a, m.b);
            k[m.cls].launches += 1;
            k[m.cls].ms += ms;
            k[m.cls].bytes += m.bytes;
            k[m.cls].flops += m.flops;
            pool.push_back(m.a);
            pool.push_back(m.b);
        }
        marks.clear();
    }
    ~Profiler() {
        for (auto& m : marks) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Algorithmic FMA count of one blur pass of one level: in-range taps of every
// output position, times the other side and the channels.
static double pass_fmas(int len, int r, long long other, int D) {
    double t = 0.0;
    for (int p = 0; p < len; ++p) {
        const int lo = std::max(-r, -p), hi = std::min(r, len - 1 - p);
        t += (double)(hi - lo + 1);
    }
    return t * (double)other * D;
}

// ---------------------------------------------------------------------------
// the sort
// ---------------------------------------------------------------------------
struct SortArgs {
    const float* x;
    int H, W, D;
    Weights w;
    const float* carried;
    int C;
    uint64_t seed;
    plas_schedule s;
    const int32_t* perm_init;
    plas_state* state_io;
    int32_t* perm_out;
    float* carried_out;
    float* sorted_out;
    plas_stats* stats;
    cudaStream_t stream;
};

static int run_sort(const SortArgs& a, char* wsbase) {
    const auto t0 = std::chrono::steady_clock::now();
    const int H = a.H, W = a.W, D = a.D;
    const long long N = (long long)H * W;
    const plas_schedule& s = a.s;
    cudaStream_t st = a.stream;
    const int nsm = num_sms();

    Geometry g = build_geometry(s, H, W);
    const int nlev = (int)g.lv.size();
    Workspace ws{};
    workspace_layout(H, W, D, nlev, g.table_floats, &ws, wsbase);

    // ---- device state ----
    DevState init{};
    const bool resume = a.state_io && (a.state_io->it > 0 || a.state_io->level > 0);
    if (resume) {
        init.it = a.state_io->it;
        init.epoch = a.state_io->epoch;
        init.redraws = a.state_io->redraws;
        init.level = a.state_io->level;
        init.stall = a.state_io->stall;
        init.has_prev = a.state_io->has_prev;
        init.done = a.state_io->done;
        init.d_prev = a.state_io->d_prev;
        init.d_last = a.state_io->d_last;
    }
    init.max_iters = s.max_iters;
    if (init.level >= nlev) init.done = 1;
    PLAS_CUDA(cudaMemcpyAsync(ws.st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st));
    PLAS_CUDA(cudaMemcpyAsync(ws.lv, g.lv.data(), sizeof(LevelDesc) * nlev, cudaMemcpyHostToDevice, st));
    PLAS_CUDA(cudaMemcpyAsync(ws.table, g.table.data(), sizeof(float) * g.table_floats,
                              cudaMemcpyHostToDevice, st));

    Profiler prof;
    prof.on = s.profile != 0;
    cudaEvent_t ea = nullptr;
    long long launches = 0;

    // ---- preparation: min/max, scale exponent, normalise + place ----
    prof.begin(st, &ea);
    launch_state_reset(ws.st, st);
    launch_minmax(a.x, N, D, ws.st, nsm, st);
    launch_finalize_prep(ws.st, N, D, a.w, s.normalize, st);
    const int mode = a.perm_init ? 2 : (s.shuffle_init ? 1 : 0);
    launch_pack(a.x, (int)N, D, a.w, s.normalize, ws.st, mode, a.perm_init, a.seed, ws.G, st);
    launch_norms(ws.lv, nlev, H, W, ws.table, st);
    launches += 5;
    prof.end(st, ea, PLAS_K_PREP, (double)N * D * 4 * 2 + (double)N * grid_stride(D) * 4, 0.0);
    if (int e = check_launch("preparation")) return e;

    // ---- per-level launch plans ----
    const int gs = grid_stride(D), ts = target_stride(D);
    const ColPlan cplan = plan_cols(H);
    std::vector<RowPlan> rplans(nlev);
    std::vector<double> row_flops(nlev), col_flops(nlev);
    for (int L = 0; L < nlev; ++L) {
        rplans[L] = plan_rows(W, D, g.lv[L].ntpx);
        if (prof.on) {
            row_flops[L] = 2.0 * pass_fmas(W, g.lv[L].rx, H, D);
            col_flops[L] = 2.0 * pass_fmas(H, g.lv[L].ry, W, D);
        }
    }
    const double blur_bytes = 8.0 * (double)N * D;

    auto enqueue_iteration = [&](int L) -> int {
        const LevelDesc& lv = g.lv[L];
        cudaEvent_t e0 = nullptr;
        prof.begin(st, &e0);
        launch_group_table(a.seed, ws.st, L, lv.beta, ws.pi, nsm, st);
        prof.end(st, e0, PLAS_K_GROUPS, 4.0 * lv.beta * lv.beta, 0.0);
        prof.begin(st, &e0);
        launch_blur_rows(ws.G, gs, H, W, D, ws.H1, ws.st, L, lv, ws.table, rplans[L], st);
        prof.end(st, e0, PLAS_K_BLUR_ROWS, blur_bytes, row_flops[L]);
        prof.begin(st, &e0);
        launch_blur_cols(ws.H1, H, W, D, ts, ws.T, ws.st, L, lv, ws.table, cplan, st);
        prof.end(st, e0, PLAS_K_BLUR_COLS, blur_bytes, col_flops[L]);
        AssignArgs aa{};
        aa.G = ws.G; aa.T = ws.T; aa.pi = ws.pi; aa.st = ws.st;
        aa.H = H; aa.W = W; aa.D = D; aa.level = L; aa.beta = lv.beta;
        aa.ngroups = (lv.beta * lv.beta) / 4; aa.nlevels = nlev; aa.seed = a.seed; aa.tol = s.tol;
        aa.trace_S = s.trace_S; aa.trace_level = s.trace_level; aa.trace_cap = s.trace_cap;
        prof.begin(st, &e0);
        launch_assign(aa, assign_grid_size(H, W, lv.beta, nsm), st);
        prof.end(st, e0, PLAS_K_ASSIGN, 0.0, 0.0);  // bytes from the grouped-cell count
        launches += 4;
        return check_launch("iteration");
    };

    // ---- iteration loop: batches of k iterations, one batch of look-ahead ----
    DevState* hb = nullptr;
    cudaEvent_t pev[2];
    if (int e = poll_buffers(&hb, pev)) return e;
    const int k = s.iters_per_poll > 0 ? s.iters_per_poll : 8;
    int level = init.level;
    bool finished = init.done || (s.max_iters > 0 && init.it >= s.max_iters);
    int slot = 0;
    bool pending = false;
    long long last_it = init.it;
    int stuck = 0;
    while (!finished) {
        for (int i = 0; i < k; ++i)
            if (int e = enqueue_iteration(level)) return e;
        PLAS_CUDA(cudaMemcpyAsync(hb + slot, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        PLAS_CUDA(cudaEventRecord(pev[slot], st));
        if (pending) {
            PLAS_CUDA(cudaEventSynchronize(pev[slot ^ 1]));
            const DevState& h = hb[slot ^ 1];
            if (h.done || (s.max_iters > 0 && h.it >= s.max_iters)) {
                finished = true;
            } else {
                level = h.level;
                stuck = (h.it == last_it) ? stuck + 1 : 0;
                last_it = h.it;
                if (stuck > 4)
                    return fail(PLAS_ERR_INTERNAL, "sort made no progress at iteration %lld", h.it);
            }
        }
        pending = true;
        slot ^= 1;
    }
    // drain the look-ahead batch (its kernels see a finished state and return)
    PLAS_CUDA(cudaEventSynchronize(pev[slot ^ 1]));
    {
        DevState chk{};
        PLAS_CUDA(cudaMemcpyAsync(&chk, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        PLAS_CUDA(cudaStreamSynchronize(st));
        if (chk.status != 0) {
            prof.harvest();
            if (chk.nonfinite) return fail(PLAS_ERR_NONFINITE, "sort input holds NaN or Inf");
            if (chk.bad_index) return fail(PLAS_ERR_INVALID_ARG, "perm_init holds an index outside [0, N)");
            return fail(PLAS_ERR_INTERNAL, "device status %d", chk.status);
        }
    }

    // ---- outputs ----
    prof.begin(st, &ea);
    launch_extract_perm(ws.G, (int)N, D, a.perm_out, st);
    launches += 1;
    if (a.carried && a.carried_out && a.C > 0) {
        launch_gather_rows(a.carried, N, a.C, a.perm_out, a.carried_out, st);
        launches += 1;
    }
    if (a.sorted_out) {
        launch_gather_rows(a.x, N, D, a.perm_out, a.sorted_out, st);
        launches += 1;
    }
    prof.end(st, ea, PLAS_K_GATHER,
             (double)N * 4 * 2 + (a.carried_out ? (double)N * a.C * 8 : 0.0) +
                 (a.sorted_out ? (double)N * D * 8 : 0.0),
             0.0);
    if (int e = check_launch("output gather")) return e;

    DevState fin{};
    if (a.stats) {
        PLAS_CUDA(cudaMemsetAsync(ws.macc, 0, sizeof(double) * 4, st));
        launch_neighbour_metrics(ws.G, gs, H, W, D, 1.0, ws.macc, nsm, st);
        launches += 1;
        double macc[4] = {0, 0, 0, 0};
        PLAS_CUDA(cudaMemcpyAsync(macc, ws.macc, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
        PLAS_CUDA(cudaMemcpyAsync(&fin, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        PLAS_CUDA(cudaStreamSynchronize(st));
        prof.harvest();
        const long long npairs = (long long)H * (W - 1) + (long long)(H - 1) * W;
        plas_stats& o = *a.stats;
        memset(&o, 0, sizeof(o));
        o.iterations = fin.it;
        o.redraws = fin.redraws;
        o.grouped_cells = fin.grouped;
        o.levels = nlev;
        o.status = fin.status;
        o.final_l2_to_target = fin.d_last;
        o.neighbour_l2 = npairs > 0 ? macc[0] / (double)npairs : 0.0;
        for (int c = 0; c < PLAS_K_COUNT; ++c) o.kernel[c] = prof.k[c];
        const long long its = fin.it - init.it;
        o.kernel[PLAS_K_ASSIGN].bytes =
            (double)fin.grouped * (12.0 * D + 8.0) + ((double)its * N - (double)fin.grouped) * 8.0 * D;
        o.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        o.launches = launches;
    } else {
        PLAS_CUDA(cudaMemcpyAsync(&fin, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
        PLAS_CUDA(cudaStreamSynchronize(st));
        prof.harvest();
    }
    if (a.state_io) {
        a.state_io->it = fin.it;
        a.state_io->epoch = fin.epoch;
        a.state_io->redraws = fin.redraws;
        a.state_io->level = fin.level;
        a.state_io->stall = fin.stall;
        a.state_io->has_prev = fin.has_prev;
        a.state_io->done = fin.done;
        a.state_io->d_prev = fin.d_prev;
        a.state_io->d_last = fin.d_last;
        a.state_io->scale_exp = fin.scale_exp;
        a.state_io->status = fin.status;
    }
    return PLAS_OK;
}

static int validate_schedule(const plas_schedule& s) {
    if (!(s.shrink > 0.0 && s.shrink < 1.0)) return fail(PLAS_ERR_INVALID_ARG, "shrink must be in (0,1)");
    if (!(s.phi_min > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "phi_min must be > 0");
    if (!(s.tol >= 0.0)) return fail(PLAS_ERR_INVALID_ARG, "tol must be >= 0");
    if (!(s.sigma_ratio > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "sigma_ratio must be > 0");
    if (s.min_block < 2) return fail(PLAS_ERR_INVALID_ARG, "min_block must be >= 2");
    if (s.max_iters < 0) return fail(PLAS_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (s.trace_cap < 0) return fail(PLAS_ERR_INVALID_ARG, "trace_cap must be >= 0");
    return PLAS_OK;
}

}  // namespace plas

using namespace plas;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int plas_version(void) { return 100; }

const char* plas_last_error(void) { return g_last_error.c_str(); }

const char* plas_status_string(int status) {
    switch (status) {
        case PLAS_OK: return "ok";
        case PLAS_ERR_INVALID_ARG: return "invalid argument";
        case PLAS_ERR_OOM: return "out of device memory";
        case PLAS_ERR_CUDA: return "CUDA error";
        case PLAS_ERR_TIMEOUT: return "device wait timed out";
        case PLAS_ERR_NONFINITE: return "input holds NaN or Inf";
        case PLAS_ERR_BUDGET: return "batch exceeds its memory budget";
        case PLAS_ERR_INTERNAL: return "internal error";
        default: return "unknown status";
    }
}

int plas_default_schedule(plas_schedule* out) {
    if (!out) return fail(PLAS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    out->phi0 = 0.0;
    out->shrink = 0.95;
    out->phi_min = 1.0;
    out->tol = 1e-4;
    out->sigma_ratio = 0.5;
    out->min_block = 16;
    out->shuffle_init = 1;
    out->normalize = 1;
    out->iters_per_poll = 8;
    out->max_iters = 0;
    out->profile = 0;
    return PLAS_OK;
}

int plas_num_levels(int H, int W, const plas_schedule* sched) {
    if (H < 1 || W < 1) return fail(PLAS_ERR_INVALID_ARG, "grid sides must be >= 1");
    plas_schedule s;
    if (sched) s = *sched; else plas_default_schedule(&s);
    if (int e = validate_schedule(s)) return e;
    return count_levels(s, H, W);
}

size_t plas_sort_workspace_bytes(int H, int W, int D) {
    if (H < 1 || W < 1 || !channels_supported(D) || (long long)H * W > (1LL << 26)) return 0;
    plas_schedule s;
    plas_default_schedule(&s);
    return sort_workspace_bytes(H, W, D, s);
}

int plas_sort(const float* x, int H, int W, int D, const float* weights, const float* carried,
              int C, uint64_t seed, const plas_schedule* sched, const int32_t* perm_init,
              plas_state* state_io, int32_t* perm_out, float* carried_out, float* sorted_out,
              void* workspace, size_t ws_bytes, plas_stats* stats, void* stream) {
    g_last_error.clear();
    if (H < 0 || W < 0) return fail(PLAS_ERR_INVALID_ARG, "grid sides must be >= 0");
    if (!channels_supported(D))
        return fail(PLAS_ERR_INVALID_ARG, "D=%d not supported (1..16, 20, 24, 32, 48, 64)", D);
    const long long N = (long long)H * W;
    if (N > (1LL << 26)) return fail(PLAS_ERR_INVALID_ARG, "N=%lld exceeds 2^26", N);
    if (C < 0 || (C > 0 && (!carried || !carried_out)))
        return fail(PLAS_ERR_INVALID_ARG, "carried/carried_out required when C > 0");
    plas_schedule s;
    if (sched) s = *sched; else plas_default_schedule(&s);
    if (int e = validate_schedule(s)) return e;
    if (N == 0) {
        if (state_io) { memset(state_io, 0, sizeof(*state_io)); state_io->done = 1; }
        if (stats) memset(stats, 0, sizeof(*stats));
        return PLAS_OK;
    }
    if (!x || !perm_out) return fail(PLAS_ERR_INVALID_ARG, "x and perm_out are required");
    if (!aligned(x, 4) || !aligned(perm_out, 4)) return fail(PLAS_ERR_INVALID_ARG, "misaligned pointer");
    const bool resume = state_io && (state_io->it > 0 || state_io->level > 0);
    if (resume && !perm_init) return fail(PLAS_ERR_INVALID_ARG, "resuming needs perm_init");
    if (resume && (state_io->level < 0 || state_io->it < 0))
        return fail(PLAS_ERR_INVALID_ARG, "invalid resume state");
    SortArgs a{};
    a.x = x; a.H = H; a.W = W; a.D = D;
    for (int d = 0; d < kMaxD; ++d) a.w.w[d] = (d < D) ? (weights ? weights[d] : 1.0f) : 0.0f;
    for (int d = 0; d < D; ++d)
        if (!std::isfinite(a.w.w[d])) return fail(PLAS_ERR_INVALID_ARG, "weights must be finite");
    a.carried = carried; a.C = C; a.seed = seed; a.s = s; a.perm_init = perm_init;
    a.state_io = state_io; a.perm_out = perm_out; a.carried_out = carried_out;
    a.sorted_out = sorted_out; a.stats = stats; a.stream = (cudaStream_t)stream;

    const size_t need = sort_workspace_bytes(H, W, D, s);
    if (workspace) {
        if (ws_bytes < need) return fail(PLAS_ERR_INVALID_ARG, "workspace too small (%zu < %zu)", ws_bytes, need);
        if (!aligned(workspace, 256)) return fail(PLAS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        return run_sort(a, (char*)workspace);
    }
    void* mem = nullptr;
    cudaError_t e = cudaMallocAsync(&mem, need, a.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "workspace allocation of %zu bytes failed: %s", need, cudaGetErrorString(e));
    }
    const int rc = run_sort(a, (char*)mem);
    cudaFreeAsync(mem, a.stream);
    return rc;
}

int plas_gather_rows(const float* src, int N, int C, const int32_t* perm, float* dst, void* stream) {
    g_last_error.clear();
    if (N < 0 || C < 1) return fail(PLAS_ERR_INVALID_ARG, "N >= 0 and C >= 1 required");
    if (N == 0) return PLAS_OK;
    if (!src || !perm || !dst) return fail(PLAS_ERR_INVALID_ARG, "NULL pointer");
    launch_gather_rows(src, N, C, perm, dst, (cudaStream_t)stream);
    return check_launch("gather_rows");
}

int plas_target(const float* x, int H, int W, int D, const float* weights, int normalize,
                const int32_t* perm, double phi, double sigma_ratio, float* T, void* stream) {
    g_last_error.clear();
    if (H < 1 || W < 1 || !channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "bad sizes");
    if (!x || !perm || !T) return fail(PLAS_ERR_INVALID_ARG, "NULL pointer");
    if (!(phi >= 0.0) || !(sigma_ratio > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "bad phi/sigma");
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = (long long)H * W;
    plas_schedule s;
    plas_default_schedule(&s);
    s.phi0 = phi > 0.0 ? phi : 1.0;
    s.phi_min = s.phi0;  // exactly one level, at phi
    s.sigma_ratio = sigma_ratio;
    s.normalize = normalize;
    Geometry g = build_geometry(s, H, W);
    Workspace ws{};
    const size_t need = workspace_layout(H, W, D, 1, g.table_floats, nullptr, nullptr);
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "workspace allocation failed");
    }
    workspace_layout(H, W, D, 1, g.table_floats, &ws, (char*)mem);
    Weights w{};
    for (int d = 0; d < D; ++d) w.w[d] = weights ? weights[d] : 1.0f;
    DevState init{};
    int rc = PLAS_OK;
    do {
        if (cudaMemcpyAsync(ws.st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(ws.lv, g.lv.data(), sizeof(LevelDesc), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(ws.table, g.table.data(), sizeof(float) * g.table_floats,
                            cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = fail(PLAS_ERR_CUDA, "upload failed");
            break;
        }
        launch_state_reset(ws.st, st);
        launch_minmax(x, N, D, ws.st, num_sms(), st);
        launch_finalize_prep(ws.st, N, D, w, normalize, st);
        launch_pack(x, (int)N, D, w, normalize, ws.st, 2, perm, 0, ws.G, st);
        launch_norms(ws.lv, 1, H, W, ws.table, st);
        const RowPlan rp = plan_rows(W, D, g.lv[0].ntpx);
        launch_blur_rows(ws.G, grid_stride(D), H, W, D, ws.H1, ws.st, 0, g.lv[0], ws.table, rp, st);
        launch_blur_cols(ws.H1, H, W, D, target_stride(D), ws.T, ws.st, 0, g.lv[0], ws.table,
                         plan_cols(H), st);
        launch_copy_features(ws.T, (int)N, D, target_stride(D), T, st);
        rc = check_launch("target");
        if (rc != PLAS_OK) break;
        DevState chk{};
        if (cudaMemcpyAsync(&chk, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(PLAS_ERR_CUDA, "status readback failed");
            break;
        }
        if (chk.bad_index) rc = fail(PLAS_ERR_INVALID_ARG, "perm holds an index outside [0, N)");
        else if (chk.nonfinite) rc = fail(PLAS_ERR_NONFINITE, "x holds NaN or Inf");
    } while (0);
    cudaFreeAsync(mem, st);
    return rc;
}

int plas_group_permutation(uint64_t seed, uint32_t tag, uint64_t counter, uint32_t n,
                           uint32_t* out, void* stream) {
    g_last_error.clear();
    if (n < 1 || n > (1u << 26) || !out) return fail(PLAS_ERR_INVALID_ARG, "bad n or NULL out");
    launch_keyed_permutation(seed, tag, counter, n, out, num_sms(), (cudaStream_t)stream);
    return check_launch("group_permutation");
}

int plas_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n, uint32_t* out,
                void* stream) {
    g_last_error.clear();
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(PLAS_ERR_INVALID_ARG, "bad arguments");
    launch_philox(ctr, key0, key1, n, out, (cudaStream_t)stream);
    return check_launch("philox");
}

int plas_grid_metrics(const float* grid, int H, int W, int D, double scale, double* out,
                      void* stream) {
    g_last_error.clear();
    if (H < 1 || W < 1 || D < 1 || !grid || !out) return fail(PLAS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    double* acc = nullptr;
    if (cudaMallocAsync((void**)&acc, sizeof(double) * 3, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "allocation failed");
    }
    double h[3] = {0, 0, 0};
    int rc = PLAS_OK;
    if (cudaMemsetAsync(acc, 0, sizeof(double) * 3, st) != cudaSuccess) rc = fail(PLAS_ERR_CUDA, "memset failed");
    if (rc == PLAS_OK) {
        launch_neighbour_metrics(grid, D, H, W, D, scale, acc, num_sms(), st);
        rc = check_launch("metrics");
    }
    if (rc == PLAS_OK && (cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaStreamSynchronize(st) != cudaSuccess))
        rc = fail(PLAS_ERR_CUDA, "readback failed");
    cudaFreeAsync(acc, st);
    if (rc != PLAS_OK) return rc;
    const double npairs = (double)H * (W - 1) + (double)(H - 1) * W;
    const double nv = npairs * D;
    out[0] = npairs > 0 ? h[0] / npairs : 0.0;
    out[1] = npairs > 0 ? h[2] / nv - (h[1] / nv) * (h[1] / nv) : 0.0;
    out[2] = npairs > 0 ? h[1] / nv : 0.0;
    return PLAS_OK;
}

}  // extern "C"
