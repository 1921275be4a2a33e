// plas_api.cu -- host helpers of the C ABI (errors, schedule geometry, the
// per-grid workspace layout) and the small entry points of include/plas.h:
// defaults, level count, row gather, the standalone target / grouping /
// Philox entry points used for per-step parity, and grid metrics.  The sort
// itself (single, batched and served) lives in engine.cu.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "plas_host.h"

namespace plas {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

std::atomic<long long> g_alloc_fail_at{0};  // 0: none; n: the n-th allocation from now fails
std::atomic<long long> g_stall_polls{0};    // read-backs still to be frozen

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    long long n = g_alloc_fail_at.load();
    while (n > 0) {
        if (g_alloc_fail_at.compare_exchange_weak(n, n - 1)) {
            if (n == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMallocAsync(p, bytes, s);
}

std::atomic<long long> g_persist_zero{0};  // persistent launches still to get a zero wait limit

unsigned long long persist_wait_limit_ns() {
    long long n = g_persist_zero.load();
    while (n > 0)
        if (g_persist_zero.compare_exchange_weak(n, n - 1)) return 0ull;
    return 2000000000ull;  // two seconds
}

std::atomic<long long> g_guard_damage{0};  // checked runs still to get a damaged guard band

bool injected_guard_damage() {
    long long n = g_guard_damage.load();
    while (n > 0)
        if (g_guard_damage.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

bool injected_stall() {
    long long n = g_stall_polls.load();
    while (n > 0)
        if (g_stall_polls.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PLAS_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return PLAS_OK;
}

int num_sms() {
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

int validate_schedule(const plas_schedule& s) {
    if (!(s.shrink > 0.0 && s.shrink < 1.0)) return fail(PLAS_ERR_INVALID_ARG, "shrink must be in (0,1)");
    if (!(s.phi_min > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "phi_min must be > 0");
    if (!(s.tol >= 0.0)) return fail(PLAS_ERR_INVALID_ARG, "tol must be >= 0");
    if (!(s.sigma_ratio > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "sigma_ratio must be > 0");
    if (s.min_block < 2) return fail(PLAS_ERR_INVALID_ARG, "min_block must be >= 2");
    if (s.max_iters < 0) return fail(PLAS_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (s.trace_cap < 0) return fail(PLAS_ERR_INVALID_ARG, "trace_cap must be >= 0");
    if (!(s.phi0 <= 1e7)) return fail(PLAS_ERR_INVALID_ARG, "phi0 too large");
    if (s.target_mode != 0 && s.target_mode != 1) return fail(PLAS_ERR_INVALID_ARG, "target_mode must be 0 or 1");
    if (s.persistent < -1 || s.persistent > 1) return fail(PLAS_ERR_INVALID_ARG, "persistent must be -1, 0 or 1");
    return PLAS_OK;
}

// ---------------------------------------------------------------------------
// schedule geometry
// ---------------------------------------------------------------------------
double start_radius(const plas_schedule& s, int H, int W) {
    double p = s.phi0 > 0.0 ? s.phi0 : (double)std::min(H, W) / 2.0 - 1.0;
    if (p < s.phi_min) p = s.phi_min;
    return p;
}

int count_levels(const plas_schedule& s, int H, int W) {
    double p = start_radius(s, H, W);
    int n = 0;
    while (p >= s.phi_min && n < 100000) {
        ++n;
        p = s.shrink * p;
    }
    return n;
}

// Taps of one pass: pairs (k_j, k_j) for j = -rr..rr at pair index rp + j,
// with rp = rr (the first tap at step 0) and zero pairs after, up to ntp, a
// whole number of 8-step blocks.  (Any rp >= rr gives the same FMA chains,
// since zero taps leave them unchanged; rp = rr needs the fewest blocks.)
static void padded_tap_pairs(int r, int rcap, double sigma, int* rr_out, int* rp, int* ntp,
                             std::vector<float>& out) {
    const int X = kFirX;
    const int rr = std::min(r, rcap);
    *rr_out = rr;
    *rp = rr;
    *ntp = (2 * rr + 1 + X - 1) / X * X;
    out.assign((size_t)2 * *ntp, 0.0f);
    for (int j = -rr; j <= rr; ++j) {
        double q = (double)j * (double)j;
        double den = 2.0 * sigma * sigma;
        const float k = (float)std::exp(-q / den);
        out[(size_t)2 * (*rp + j)] = k;
        out[(size_t)2 * (*rp + j) + 1] = k;
    }
}

Geometry build_geometry(const plas_schedule& s, int H, int W) {
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
        padded_tap_pairs(d.r, W - 1, sigma, &d.rx, &d.rpx, &d.ntpx, tx);
        padded_tap_pairs(d.r, H - 1, sigma, &d.ry, &d.rpy, &d.ntpy, ty);
        g.max_steps = std::max({g.max_steps, d.ntpx, d.ntpy});
        d.off_tx = (long long)off; off += align_up((size_t)2 * d.ntpx, 4);
        d.off_ty = (long long)off; off += align_up((size_t)2 * d.ntpy, 4);
        // border norms, then their reciprocals, per axis
        d.off_nx = (long long)off; off += 2 * align_up((size_t)W, 4);
        d.off_ny = (long long)off; off += 2 * align_up((size_t)H, 4);
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
// per-grid workspace
// ---------------------------------------------------------------------------
size_t workspace_layout(int H, int W, int D, int nlev, size_t table_floats, Workspace* ws,
                        char* base, bool sat) {
    const long long N = (long long)H * W;
    size_t off = 0;
    Workspace w{};
    // every region is followed by a guard band (filled and verified by
    // checked runs; otherwise unused)
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        if (w.guards.n < kMaxGuards) w.guards.at[w.guards.n++] = base ? (unsigned char*)(base + off) : nullptr;
        off += kGuardBytes;
        return base ? (void*)(base + o) : nullptr;
    };
    w.st = (DevState*)take(sizeof(DevState));
    w.ref = (GridRef*)take(sizeof(GridRef));
    w.G = (float*)take(sizeof(float) * (size_t)N * grid_stride(D));
    w.T = (float*)take(sizeof(float) * (size_t)N * target_stride(D));
    w.H1 = (float*)take(sizeof(float) * (size_t)W * h1_stride(H, D));
    w.pi = (uint32_t*)take(sizeof(uint32_t) * (size_t)std::max<long long>(N, 4));
    w.lv = (LevelDesc*)take(sizeof(LevelDesc) * (size_t)nlev);
    w.table = (float*)take(sizeof(float) * table_floats);
    w.macc = (double*)take(sizeof(double) * 4);
    w.pctl = (PersistCtl*)take(sizeof(PersistCtl));
    w.sat = sat ? (long long*)take(sizeof(long long) * (size_t)N * ((D + 1) & ~1)) : nullptr;
    if (ws) *ws = w;
    return off;
}

size_t sort_workspace_bytes(int H, int W, int D, const plas_schedule& s) {
    Geometry g = build_geometry(s, H, W);
    return workspace_layout(H, W, D, (int)g.lv.size(), g.table_floats, nullptr, nullptr,
                            s.target_mode == 1);
}

// ---------------------------------------------------------------------------
// pinned staging for state polls: one buffer and two events per host thread,
// allocated on first use and kept for the life of the thread
// ---------------------------------------------------------------------------
struct PollBuf {
    void* h = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int device = -1;
};
static thread_local PollBuf g_poll;

int poll_buffers(size_t bytes, void** host, cudaEvent_t* ev2) {
    int dev = 0;
    PLAS_CUDA(cudaGetDevice(&dev));
    if (g_poll.device != dev || g_poll.bytes < bytes) {
        // a buffer of another device or too small is replaced (the old one is
        // left to process teardown: its device context may be in use)
        void* p = nullptr;
        const size_t nb = std::max<size_t>(bytes, 4096);
        PLAS_CUDA(cudaMallocHost(&p, nb));
        g_poll.h = p;
        g_poll.bytes = nb;
        PLAS_CUDA(cudaEventCreateWithFlags(&g_poll.ev[0], cudaEventDisableTiming));
        PLAS_CUDA(cudaEventCreateWithFlags(&g_poll.ev[1], cudaEventDisableTiming));
        g_poll.device = dev;
    }
    *host = g_poll.h;
    ev2[0] = g_poll.ev[0];
    ev2[1] = g_poll.ev[1];
    return PLAS_OK;
}

// ---- launch-shape tuning table --------------------------------------------------
namespace {
struct TuneEntry {
    int device, H, W, D;
    Tuning t;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
}  // namespace

Tuning tuning_for(int H, int W, int D) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const TuneEntry* best = nullptr;
    double best_d = 0.0;
    const double ln = std::log((double)std::max(1, H) * std::max(1, W));
    for (const auto& e : g_tune) {
        if (e.device != dev || e.D != D) continue;
        const double d = std::fabs(std::log((double)e.H * e.W) - ln);
        if (!best || d < best_d) {
            best = &e;
            best_d = d;
        }
    }
    return best ? best->t : Tuning{};
}

void install_tuning(int H, int W, int D, const Tuning* t) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.erase(std::remove_if(g_tune.begin(), g_tune.end(),
                                [&](const TuneEntry& e) {
                                    return e.device == dev && e.H == H && e.W == W && e.D == D;
                                }),
                 g_tune.end());
    if (t) g_tune.push_back(TuneEntry{dev, H, W, D, *t});
}

}  // namespace plas

using namespace plas;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int plas_version(void) { return 200; }

// Host-side fault injection.  kind 0 clears everything; kind 1 makes the
// count-th device allocation from now on fail (count >= 1); kind 2 freezes
// the next count state read-backs of the sweep engine, so that its progress
// check sees a grid that does not advance.
int plas_debug_inject(int kind, long long count) {
    if (kind == 0) {
        plas::g_alloc_fail_at.store(0);
        plas::g_stall_polls.store(0);
        plas::g_persist_zero.store(0);
        plas::g_guard_damage.store(0);
        return PLAS_OK;
    }
    if (count < 1) return plas::fail(PLAS_ERR_INVALID_ARG, "count must be >= 1");
    if (kind == 1) {
        plas::g_alloc_fail_at.store(count);
        return PLAS_OK;
    }
    if (kind == 2) {
        plas::g_stall_polls.store(count);
        return PLAS_OK;
    }
    if (kind == 3) {
        plas::g_persist_zero.store(count);
        return PLAS_OK;
    }
    if (kind == 4) {
        plas::g_guard_damage.store(count);
        return PLAS_OK;
    }
    return plas::fail(PLAS_ERR_INVALID_ARG, "unknown injection kind %d", kind);
}

int plas_set_tuning(int H, int W, int D, const plas_tuning* t) {
    set_last_error("");
    if (H < 1 || W < 1 || !channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "bad shape");
    if (!t) {
        install_tuning(H, W, D, nullptr);
        return PLAS_OK;
    }
    if (t->fir_small_below < 0 || t->fir_medium_below < 0 || t->assign_ctas_per_sm < 1 ||
        t->assign_ctas_per_sm > kAssignMaxPerSm)
        return fail(PLAS_ERR_INVALID_ARG,
                    "fir_small_below and fir_medium_below must be >= 0, assign_ctas_per_sm 1..%d",
                    kAssignMaxPerSm);
    Tuning tu;
    tu.small_below = t->fir_small_below;
    tu.medium_below = t->fir_medium_below;
    tu.assign_per_sm = t->assign_ctas_per_sm;
    tu.large_tma = t->large_tma ? 1 : 0;
    tu.small_fused = t->small_fused ? 1 : 0;
    install_tuning(H, W, D, &tu);
    return PLAS_OK;
}

int plas_get_tuning(int H, int W, int D, plas_tuning* out) {
    set_last_error("");
    if (!out) return fail(PLAS_ERR_INVALID_ARG, "out is NULL");
    if (H < 1 || W < 1 || !channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "bad shape");
    memset(out, 0, sizeof(*out));
    const Tuning t = tuning_for(H, W, D);
    out->fir_small_below = t.small_below;
    out->fir_medium_below = t.medium_below;
    out->assign_ctas_per_sm = t.assign_per_sm;
    out->large_tma = t.large_tma;
    out->small_fused = t.small_fused;
    return PLAS_OK;
}

const char* plas_last_error(void) { return g_last_error.c_str(); }

const char* plas_status_string(int status) {
    switch (status) {
        case PLAS_OK: return "ok";
        case PLAS_ERR_INVALID_ARG: return "invalid argument";
        case PLAS_ERR_OOM: return "out of device memory";
        case PLAS_ERR_CUDA: return "CUDA error";
        case PLAS_ERR_TIMEOUT: return "device wait timed out";
        case PLAS_ERR_NONFINITE: return "input holds NaN or Inf";
        case PLAS_ERR_BUDGET: return "request exceeds the memory budget";
        case PLAS_ERR_INTERNAL: return "internal error";
        case PLAS_ERR_NOT_PERMUTATION: return "not a permutation";
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
    out->sigma_ratio = 2.0;
    out->min_block = 16;
    out->shuffle_init = 1;
    out->normalize = 1;
    out->iters_per_poll = 8;
    out->max_iters = 0;
    out->profile = 0;
    out->graphs = 1;
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
    if (H < 1 || W < 1 || !channels_supported(D) || !grid_fits(H, W, D)) return 0;
    plas_schedule s;
    plas_default_schedule(&s);
    return sort_workspace_bytes(H, W, D, s);
}

size_t plas_sort_workspace_bytes_ex(int H, int W, int D, const plas_schedule* sched) {
    if (H < 1 || W < 1 || !channels_supported(D) || !grid_fits(H, W, D)) return 0;
    plas_schedule s;
    if (sched) s = *sched; else plas_default_schedule(&s);
    if (validate_schedule(s) != PLAS_OK) return 0;
    return sort_workspace_bytes(H, W, D, s);
}

int plas_gather_rows(const float* src, int N, int C, const int32_t* perm, float* dst, void* stream) {
    g_last_error.clear();
    if (N < 0 || C < 1) return fail(PLAS_ERR_INVALID_ARG, "N >= 0 and C >= 1 required");
    if (N == 0) return PLAS_OK;
    if (!src || !perm || !dst) return fail(PLAS_ERR_INVALID_ARG, "NULL pointer");
    launch_gather_rows(src, N, C, perm, dst, (cudaStream_t)stream);
    return check_launch("gather_rows");
}

int plas_select_rows(const float* src, long long n_src, int C, const int32_t* idx, long long n_out,
                     float* dst, void* stream) {
    g_last_error.clear();
    if (n_src < 0 || n_out < 0 || C < 1) return fail(PLAS_ERR_INVALID_ARG, "sizes must be >= 0, C >= 1");
    if (n_out == 0) return PLAS_OK;
    if (!src || !idx || !dst) return fail(PLAS_ERR_INVALID_ARG, "NULL pointer");
    launch_gather_rows(src, n_out, C, idx, dst, (cudaStream_t)stream, n_src);
    return check_launch("select_rows");
}

static int target_impl(const float* x, int H, int W, int D, const float* weights, int normalize,
                       const int32_t* perm, double phi, double sigma_ratio, float* T, void* stream,
                       int mode) {
    g_last_error.clear();
    if (H < 1 || W < 1 || !channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "bad sizes");
    if (!grid_fits(H, W, D)) return fail(PLAS_ERR_INVALID_ARG, "grid too large (H*W and max(H, W)*D must be <= 2^26)");
    if (!x || !perm || !T) return fail(PLAS_ERR_INVALID_ARG, "NULL pointer");
    if (!(phi >= 0.0 && phi <= 1e7) || !(sigma_ratio > 0.0)) return fail(PLAS_ERR_INVALID_ARG, "bad phi/sigma");
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
    const size_t need = workspace_layout(H, W, D, 1, g.table_floats, nullptr, nullptr, mode == 1);
    void* mem = nullptr;
    if (dev_alloc(&mem, need, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "workspace allocation failed");
    }
    workspace_layout(H, W, D, 1, g.table_floats, &ws, (char*)mem, mode == 1);
    Weights w{};
    for (int d = 0; d < D; ++d) w.w[d] = weights ? weights[d] : 1.0f;
    DevState init{};
    GridRef ref{};
    ref.G = ws.G; ref.T = ws.T; ref.H1 = ws.H1; ref.pi = ws.pi; ref.st = ws.st;
    ref.lv = ws.lv; ref.table = ws.table; ref.H = H; ref.W = W; ref.nlev = 1;
    ref.target_mode = mode;
    ref.sat = ws.sat;
    ref.edge_blocks = 1;
    int rc = PLAS_OK;
    do {
        if (cudaMemcpyAsync(ws.st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(ws.ref, &ref, sizeof(GridRef), cudaMemcpyHostToDevice, st) != cudaSuccess ||
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
        if (mode == 1) {
            launch_box_target(ws.ref, H, W, D, num_sms(), st);
        } else {
            const Tuning tu = tuning_for(H, W, D);
            const int var = fir_variant(g.lv[0].r, D, tu);
            FirTma tma;
            if (tu.large_tma) make_fir_tma(ws.G, ws.H1, H, W, D, g.max_steps, &tma);
            launch_fir(0, ws.ref, nullptr, fir_pass_ctas(0, H, W, D, var), D, var, st, &tma);
            launch_fir(1, ws.ref, nullptr, fir_pass_ctas(1, H, W, D, var), D, var, st, &tma);
        }
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

int plas_target(const float* x, int H, int W, int D, const float* weights, int normalize,
                const int32_t* perm, double phi, double sigma_ratio, float* T, void* stream) {
    return target_impl(x, H, W, D, weights, normalize, perm, phi, sigma_ratio, T, stream, 0);
}

int plas_target_box(const float* x, int H, int W, int D, const float* weights, int normalize,
                    const int32_t* perm, double phi, float* T, void* stream) {
    return target_impl(x, H, W, D, weights, normalize, perm, phi, 2.0, T, stream, 1);
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

int plas_check_permutation(const int32_t* perm, int N, int* first_bad, void* stream) {
    g_last_error.clear();
    if (first_bad) *first_bad = -1;
    if (N < 0 || N > (1 << 30) || (N > 0 && !perm))
        return fail(PLAS_ERR_INVALID_ARG, "0 <= N <= 2^30 and a non-NULL perm required");
    if (N == 0) return PLAS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = ((size_t)N + 31) / 32;
    const size_t bytes = 16 + 2 * words * sizeof(uint32_t);
    char* mem = nullptr;
    if (dev_alloc((void**)&mem, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PLAS_ERR_OOM, "allocation failed");
    }
    int* res = reinterpret_cast<int*>(mem);
    uint32_t* seen = reinterpret_cast<uint32_t*>(mem + 16);
    uint32_t* dup = seen + words;
    const int init = 0x7fffffff;
    int h = init;
    int rc = PLAS_OK;
    if (cudaMemsetAsync(seen, 0, 2 * words * sizeof(uint32_t), st) != cudaSuccess ||
        cudaMemcpyAsync(res, &init, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = fail(PLAS_ERR_CUDA, "initialisation failed");
    if (rc == PLAS_OK) {
        launch_check_permutation(perm, N, seen, dup, res, num_sms(), st);
        rc = check_launch("check_permutation");
    }
    if (rc == PLAS_OK && (cudaMemcpyAsync(&h, res, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaStreamSynchronize(st) != cudaSuccess))
        rc = fail(PLAS_ERR_CUDA, "readback failed");
    cudaFreeAsync(mem, st);
    if (rc != PLAS_OK) return rc;
    if (h == init) return PLAS_OK;
    if (first_bad) *first_bad = h;
    return fail(PLAS_ERR_NOT_PERMUTATION,
                "position %d holds a value outside [0, %d) or one that occurs more than once", h, N);
}

int plas_grid_metrics(const float* grid, int H, int W, int D, double scale, double* out,
                      void* stream) {
    g_last_error.clear();
    if (H < 1 || W < 1 || D < 1 || !grid || !out) return fail(PLAS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    double* acc = nullptr;
    if (dev_alloc((void**)&acc, sizeof(double) * 3, st) != cudaSuccess) {
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
