// engine.cu -- the sweep engine behind plas_sort, plas_batch_sort and the
// served-sort API (include/plas.h).
//
// A sweep advances every admitted grid by one PLAS iteration (Sec. 3.1 of
// Morgenstern et al., arXiv 2312.13299): grouping table, target pass along y,
// target pass along x, assignment + schedule step -- one launch per kernel
// class for all grids.  The schedule runs on the device, so the host only
// enqueues batches of sweeps and reads each grid's 128-byte state header back
// once per batch, one batch behind (the GPU never waits for the host inside a
// level).  A grid whose schedule has ended takes no work in later sweeps; its
// outputs (permutation, carried attributes) are gathered when the host sees
// it finished, and its workspace can then be given to a new request.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <vector>

#include "plas_host.h"

namespace plas {

namespace {

// kernel classes of a sweep (the grouping table is written by the FIR pass-0 launch)
enum { kClsFirY = 0, kClsFirX = 1, kClsAssign = 2, kClsCount = 3 };

struct Job {
    const float* x = nullptr;
    int H = 0, W = 0;
    const float* carried = nullptr;
    int C = 0;
    uint64_t seed = 0;
    const int32_t* perm_init = nullptr;
    plas_state init{};
    bool resume = false;
    int32_t* perm_out = nullptr;
    float* carried_out = nullptr;
    float* sorted_out = nullptr;
    plas_state* state_out = nullptr;
    long long* trace_S = nullptr;
    int* trace_level = nullptr;
    long long trace_cap = 0;
    long long ticket = 0;
};

struct Slot {
    Job job;
    Geometry geo;
    Workspace ws{};
    char* mem = nullptr;
    size_t bytes = 0;
    bool owns = false;
    long long N = 0;
    int nlev = 0;
    int ctas[kClsCount] = {0, 0, 0};
    Tuning tune;  // FIR tiling choice
    int fvar = kFirLargeRadius;  // FIR variant this grid's CTA maps hold (multi-grid sweeps)
    FirTma tma;   // the large tiling's tensor maps (one-grid sweeps)
    bool active = false;
    bool cancel = false;  // served request cancelled while admitted
    DevState last{};
    long long last_it = -1;
    int stuck = 0;
    // served scheduling: estimated device time of one iteration at each level
    // and of the rest of the sort from each level on (ns)
    std::vector<double> it_ns;
    std::vector<double> rem_ns;
};

bool finished(const Slot& s, const plas_schedule& sch) {
    return s.last.done || s.last.status != 0 || (sch.max_iters > 0 && s.last.it >= sch.max_iters);
}

struct EventPair {
    cudaEvent_t a, b;
    int cls;
};

// Launch parameters of one batch of sweeps.
struct SweepPlan {
    int k;
    int var;
    const GridRef* grids;
    const CtaMap* map[kClsCount];
    int ctas[kClsCount];
    // multi-grid sweeps: one launch per FIR variant group and pass (the grids
    // of a group share a variant; pass 1 of the one-launch variants is empty)
    int nfg = 0;
    int fvar[kFirTilings] = {};
    int fctas[2][kFirTilings] = {};
    const CtaMap* fmap[2][kFirTilings] = {};
    bool operator==(const SweepPlan& o) const {
        if (k != o.k || var != o.var || grids != o.grids || nfg != o.nfg) return false;
        for (int c = 0; c < kClsCount; ++c)
            if (map[c] != o.map[c] || ctas[c] != o.ctas[c]) return false;
        for (int g = 0; g < nfg; ++g)
            if (fvar[g] != o.fvar[g] || fctas[0][g] != o.fctas[0][g] || fctas[1][g] != o.fctas[1][g] ||
                fmap[0][g] != o.fmap[0][g] || fmap[1][g] != o.fmap[1][g])
                return false;
        return true;
    }
    // kernel launches of one sweep
    int launches() const {
        int n = 1;  // assignment
        if (nfg == 0) return n + (ctas[kClsFirY] > 0) + (ctas[kClsFirX] > 0);
        for (int g = 0; g < nfg; ++g) n += (fctas[0][g] > 0) + (fctas[1][g] > 0);
        return n;
    }
};

struct Graph {
    cudaGraphExec_t exec = nullptr;
    SweepPlan plan{};
};

class Engine {
   public:
    Engine(int D, const Weights& w, const plas_schedule& s, cudaStream_t st)
        : D_(D), w_(w), s_(s), st_(st), nsm_(num_sms()) {}
    ~Engine() {
        for (auto& p : marks_) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : pool_) cudaEventDestroy(e);
        for (auto e : ev_)
            if (e) cudaEventDestroy(e);
        if (dmaps_ && dmaps_owned_) cudaFreeAsync(dmaps_, st_);
        for (auto& g : graph_)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap_) cudaStreamDestroy(cap_);
        if (!owned_host_.empty()) {
            cudaStreamSynchronize(st_);  // no read-back may still target them
            for (void* h : owned_host_) cudaFreeHost(h);
        }
    }

    // Poll into pinned buffers of this engine instead of the calling
    // thread's shared one (for engines that outlive a single call).
    void own_host_buffers() { own_host_ = true; }

    // Continue this engine's work on stream s, after everything already
    // enqueued on its current stream (graphs launch into any stream).
    int move_to_stream(cudaStream_t s) {
        cudaEvent_t e = nullptr;
        PLAS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        PLAS_CUDA(cudaEventRecord(e, st_));
        PLAS_CUDA(cudaStreamWaitEvent(s, e, 0));
        cudaEventDestroy(e);
        st_ = s;
        return PLAS_OK;
    }

    // Multi-grid descriptor arrays come from this arena when given (no
    // allocation), else from stream-ordered allocations.
    void set_arena(char* base, size_t bytes) {
        arena_ = base;
        arena_bytes_ = bytes;
    }

    static size_t map_bytes(size_t grids, size_t ctas) {
        return align_up(grids * sizeof(GridRef), 256) + align_up(ctas * sizeof(CtaMap), 256);
    }

    int admit(Slot* sl) {
        const Job& j = sl->job;
        const int H = j.H, W = j.W;
        sl->N = (long long)H * W;
        sl->geo = build_geometry(s_, H, W);
        sl->nlev = (int)sl->geo.lv.size();
        workspace_layout(H, W, D_, sl->nlev, sl->geo.table_floats, &sl->ws, sl->mem,
                         s_.target_mode == 1);
        make_fir_tma(sl->ws.G, sl->ws.H1, H, W, D_, sl->geo.max_steps, &sl->tma);
        DevState init{};
        if (j.resume) {
            init.it = j.init.it;
            init.epoch = j.init.epoch;
            init.redraws = j.init.redraws;
            init.level = j.init.level;
            init.stall = j.init.stall;
            init.has_prev = j.init.has_prev;
            init.done = j.init.done;
            init.d_prev = j.init.d_prev;
            init.d_last = j.init.d_last;
        }
        init.max_iters = s_.max_iters;
        if (init.level >= sl->nlev) init.done = 1;
        GridRef ref{};
        ref.G = sl->ws.G; ref.T = sl->ws.T; ref.H1 = sl->ws.H1; ref.pi = sl->ws.pi;
        ref.st = sl->ws.st; ref.lv = sl->ws.lv; ref.table = sl->ws.table;
        ref.H = H; ref.W = W; ref.nlev = sl->nlev; ref.seed = j.seed;
        ref.trace_S = j.trace_S; ref.trace_level = j.trace_level; ref.trace_cap = j.trace_cap;
        ref.target_mode = s_.target_mode;
        ref.sat = sl->ws.sat;
        ref.checked = s_.checked;
        ref.edge_blocks = s_.whole_blocks ? 0 : 1;
        if (s_.checked) {
            launch_fill_guards(sl->ws.guards, st_);
            if (injected_guard_damage() && sl->ws.guards.n > 0)  // a planted overwrite (tests)
                PLAS_CUDA(cudaMemsetAsync(sl->ws.guards.at[0] + 17, 0, 1, st_));
        }
        PLAS_CUDA(cudaMemcpyAsync(sl->ws.st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st_));
        PLAS_CUDA(cudaMemcpyAsync(sl->ws.ref, &ref, sizeof(GridRef), cudaMemcpyHostToDevice, st_));
        PLAS_CUDA(cudaMemcpyAsync(sl->ws.lv, sl->geo.lv.data(), sizeof(LevelDesc) * sl->nlev,
                                  cudaMemcpyHostToDevice, st_));
        PLAS_CUDA(cudaMemcpyAsync(sl->ws.table, sl->geo.table.data(),
                                  sizeof(float) * sl->geo.table_floats, cudaMemcpyHostToDevice, st_));
        cudaEvent_t e0 = begin();
        launch_state_reset(sl->ws.st, st_);
        launch_minmax(j.x, sl->N, D_, sl->ws.st, nsm_, st_);
        launch_finalize_prep(sl->ws.st, sl->N, D_, w_, s_.normalize, st_);
        const int mode = j.perm_init ? 2 : (s_.shuffle_init ? 1 : 0);
        launch_pack(j.x, (int)sl->N, D_, w_, s_.normalize, sl->ws.st, mode, j.perm_init, j.seed,
                    sl->ws.G, st_);
        launch_norms(sl->ws.lv, sl->nlev, H, W, sl->ws.table, st_);
        end(e0, -1);
        launches_ += 5;
        if (int e = check_launch("preparation")) return e;
        const Tuning tu = tuning_for(H, W, D_);
        sl->tune = tu;
        sl->ctas[kClsFirY] = fir_ctas(H, W * D_, kFirLargeRadius);
        sl->ctas[kClsFirX] = fir_ctas(W, H * D_, kFirLargeRadius);
        sl->ctas[kClsAssign] = assign_ctas(H, W, nsm_, tu.assign_per_sm);
        sl->last = init;
        sl->active = true;
        active_.push_back(sl);
        dirty_ = true;
        return PLAS_OK;
    }

    // Enqueue k sweeps over the active grids.
    // FIR variant of a grid at the radius it last reported
    int grid_variant(const Slot* sl) const {
        const int L = std::min(std::max(sl->last.level, 0), sl->nlev - 1);
        return fir_variant(sl->geo.lv[L].r, D_, sl->tune);
    }

    int sweeps(int k) {
        if (active_.empty()) return PLAS_OK;
        if (!dirty_ && active_.size() > 1 && !want_persist()) {
            // a grid whose radius now takes another FIR variant: new CTA maps
            for (const Slot* sl : active_)
                if (grid_variant(sl) != sl->fvar) {
                    dirty_ = true;
                    break;
                }
        }
        if (dirty_)
            if (int e = rebuild()) return e;
        SweepPlan p{};
        p.k = k;
        const bool one = active_.size() == 1;
        p.grids = one ? active_[0]->ws.ref : dgrids_;
        // FIR tiling: one grid follows the radius it last reported (all tilings
        // give the same bits; a stale choice only costs time); many grids use
        // the large-radius tiling their CTA maps were built for
        p.var = kFirLargeRadius;
        for (int c = 0; c < kClsCount; ++c) {
            p.map[c] = one ? nullptr : dmap_[c];
            p.ctas[c] = one ? active_[0]->ctas[c] : total_[c];
        }
        if (!one && !want_persist()) {
            p.nfg = nfg_;
            for (int g = 0; g < nfg_; ++g) {
                p.fvar[g] = fvar_[g];
                for (int pass = 0; pass < 2; ++pass) {
                    p.fctas[pass][g] = fcnt_[pass][g];
                    p.fmap[pass][g] = dmap_[pass == 0 ? kClsFirY : kClsFirX] + foff_[pass][g];
                }
            }
        }
        if (one) {
            const Slot* sl = active_[0];
            const int L = std::min(std::max(sl->last.level, 0), sl->nlev - 1);
            p.var = fir_variant(sl->geo.lv[L].r, D_, sl->tune);
            p.ctas[kClsFirY] = fir_pass_ctas(0, sl->job.H, sl->job.W, D_, p.var);
            p.ctas[kClsFirX] = fir_pass_ctas(1, sl->job.H, sl->job.W, D_, p.var);
        }
        if (one) persist_ = want_persist();
        if (persist_) {
            // one cooperative launch for the k sweeps: the work items of each
            // phase are the medium tiling's FIR tiles and the assignment slices
            const int ny = one ? fir_ctas(active_[0]->job.H, active_[0]->job.W * D_, kFirMediumRadius)
                               : total_[kClsFirY];
            const int nx = one ? fir_ctas(active_[0]->job.W, active_[0]->job.H * D_, kFirMediumRadius)
                               : total_[kClsFirX];
            const int rc = launch_persist(p.grids, (int)active_.size(), p.map[kClsFirY], ny,
                                          p.map[kClsFirX], nx, p.map[kClsAssign], p.ctas[kClsAssign], D_,
                                          k, s_.tol, active_[0]->ws.pctl, persist_wait_limit_ns(), st_);
            launches_ += 1;
            persist_launches_ += 1;
            if (rc != 0) {
                const cudaError_t e = cudaGetLastError();
                return fail(rc == -1 ? PLAS_ERR_INVALID_ARG : PLAS_ERR_CUDA,
                            "persistent sweep launch failed: %s", cudaGetErrorString(e));
            }
            return check_launch("persistent sweep");
        }
        launches_ += (long long)k * (s_.target_mode == 1 ? kClsCount : p.launches());
        if (s_.graphs && !s_.profile && !graphs_failed_) {
            // every kernel reads its grid's level from device state, so a batch
            // captured once replays unchanged until the grid set, the tiling or
            // k changes
            Graph& g = graph_[p.var];
            if (!g.exec || !(g.plan == p)) {
                if (int e = capture(p, &g)) return e;
            }
            if (g.exec) {
                PLAS_CUDA(cudaGraphLaunch(g.exec, st_));
                graph_launches_ += 1;
                return PLAS_OK;
            }
        }
        enqueue(p, st_, true);
        return check_launch("sweep");
    }

    // Enqueue a read-back of every active grid's state header into host
    // buffer 'buf' (0 or 1) and record its event.
    int poll(int buf) {
        const size_t hb = kStateHeaderBytes;
        if (active_.size() > host_cap_ || host_ == nullptr) {
            // a grown buffer replaces the old one, which stays allocated, so
            // a read-back still in flight keeps a valid destination
            host_cap_ = std::max<size_t>({active_.size(), 2 * host_cap_, 8});
            if (int e = host_buffers(2 * host_cap_ * hb)) return e;
        }
        polled_[buf] = active_;
        polled_base_[buf] = host_ + buf * host_cap_ * hb;
        for (size_t i = 0; i < active_.size(); ++i)
            PLAS_CUDA(cudaMemcpyAsync(polled_base_[buf] + i * hb, active_[i]->ws.st, hb,
                                      cudaMemcpyDeviceToHost, st_));
        PLAS_CUDA(cudaEventRecord(ev_[buf], st_));
        return PLAS_OK;
    }

    // Whether the next sweeps run as one persistent cooperative launch (on
    // request only: graph-replayed launches measured faster for every grid
    // size and batch tried, so they stay the default).
    bool want_persist() const {
        return s_.persistent > 0 && s_.target_mode == 0 && !s_.profile;
    }

    // Whether poll 'buf' has landed (wait() then returns without blocking),
    // and a wait for it that does not consume it.
    bool poll_ready(int buf) const { return cudaEventQuery(ev_[buf]) != cudaErrorNotReady; }
    void sync_poll(int buf) const { cudaEventSynchronize(ev_[buf]); }

    // Wait for poll 'buf' and store each polled grid's state.
    int wait(int buf) {
        PLAS_CUDA(cudaEventSynchronize(ev_[buf]));
        const size_t hb = kStateHeaderBytes;
        for (size_t i = 0; i < polled_[buf].size(); ++i) {
            Slot* sl = polled_[buf][i];
            if (!injected_stall()) memcpy(&sl->last, polled_base_[buf] + i * hb, hb);
            if (!finished(*sl, s_)) {
                sl->stuck = (sl->last.it == sl->last_it) ? sl->stuck + 1 : 0;
                sl->last_it = sl->last.it;
                if (sl->stuck > 4)
                    return fail(PLAS_ERR_INTERNAL, "grid made no progress at iteration %lld", sl->last.it);
            }
        }
        return PLAS_OK;
    }

    // Take a grid out of the sweeps without outputs (a cancelled request).
    // Sweeps already enqueued still run on its workspace; the caller frees
    // that memory stream-ordered after them.
    void drop(Slot* sl) {
        sl->active = false;
        active_.erase(std::remove(active_.begin(), active_.end(), sl), active_.end());
        dirty_ = true;
    }

    // Enqueue the outputs of a finished grid and take it out of the sweeps.
    int retire(Slot* sl) {
        const Job& j = sl->job;
        if (sl->last.status == 0) {
            launch_extract_perm(sl->ws.G, (int)sl->N, D_, j.perm_out, st_);
            launches_ += 1;
            if (j.carried && j.carried_out && j.C > 0) {
                launch_gather_rows(j.carried, sl->N, j.C, j.perm_out, j.carried_out, st_);
                launches_ += 1;
            }
            if (j.sorted_out) {
                launch_gather_rows(j.x, sl->N, D_, j.perm_out, j.sorted_out, st_);
                launches_ += 1;
            }
        }
        sl->active = false;
        active_.erase(std::remove(active_.begin(), active_.end(), sl), active_.end());
        dirty_ = true;
        return check_launch("outputs");
    }

    // Per-class event times (call after the stream is synchronised).
    void harvest() {
        for (auto& m : marks_) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, m.a, m.b);
            const int k = m.cls < 0 ? PLAS_K_PREP : class_to_stat(m.cls);
            ks_[k].launches += (m.cls < 0) ? 5 : 1;
            ks_[k].ms += ms;
            pool_.push_back(m.a);
            pool_.push_back(m.b);
        }
        marks_.clear();
    }

    static int class_to_stat(int c) {
        switch (c) {
            case kClsFirY: return PLAS_K_BLUR_COLS;
            case kClsFirX: return PLAS_K_BLUR_ROWS;
            default: return PLAS_K_ASSIGN;
        }
    }

    std::vector<Slot*>& active() { return active_; }
    // Replace the set of grids the next sweeps advance (admitted slots only).
    void select(const std::vector<Slot*>& run) {
        if (run != active_) {
            active_ = run;
            dirty_ = true;
        }
    }
    const std::vector<Slot*>& polled(int buf) const { return polled_[buf]; }
    plas_kernel_stat ks_[PLAS_K_COUNT] = {};
    long long launches_ = 0;

   private:
    cudaEvent_t begin() {
        if (!s_.profile) return nullptr;
        cudaEvent_t e = get_event();
        cudaEventRecord(e, st_);
        return e;
    }
    void end(cudaEvent_t a, int cls) {
        if (!s_.profile || !a) return;
        cudaEvent_t b = get_event();
        cudaEventRecord(b, st_);
        marks_.push_back({a, b, cls});
    }
    cudaEvent_t get_event() {
        if (!pool_.empty()) {
            cudaEvent_t e = pool_.back();
            pool_.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    // Tensor maps of the one grid a sweep advances (none for many grids).
    const FirTma* tma_of(const SweepPlan& p) const {
        return p.map[kClsFirY] == nullptr && active_.size() == 1 && active_[0]->tune.large_tma
                   ? &active_[0]->tma
                   : nullptr;
    }

    // The launches of k sweeps (events only when profiling directly).
    void enqueue(const SweepPlan& p, cudaStream_t st, bool events) {
        for (int i = 0; i < p.k; ++i) {
            for (int c = 0; c < kClsCount; ++c) {
                cudaEvent_t e0 = events ? begin() : nullptr;
                switch (c) {
                    case kClsFirY:
                    case kClsFirX: {
                        const int pass = c == kClsFirY ? 0 : 1;
                        if (s_.target_mode == 1) {  // box target (single grid): all of it here
                            if (pass == 0)
                                launch_box_target(p.grids, active_[0]->job.H, active_[0]->job.W, D_, nsm_, st);
                        } else if (p.nfg == 0) {
                            launch_fir(pass, p.grids, p.map[c], p.ctas[c], D_, p.var, st, tma_of(p));
                        } else {  // one launch per variant group of the grids
                            for (int g = 0; g < p.nfg; ++g)
                                launch_fir(pass, p.grids, p.fmap[pass][g], p.fctas[pass][g], D_, p.fvar[g], st);
                        }
                        break;
                    }
                    default: launch_assign(p.grids, p.map[c], p.ctas[c], D_, s_.tol, st, s_.checked != 0); break;
                }
                if (events) end(e0, c);
            }
        }
    }

    // Capture the launches of plan p on a private stream (nothing runs) and
    // instantiate them.  A capture the runtime refuses leaves g empty and
    // switches this engine to direct launches; a launch error fails.
    int capture(const SweepPlan& p, Graph* g) {
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
        if (!cap_) PLAS_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
        prepare_fir_launches();
        prepare_box_launches();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            graphs_failed_ = true;
            return PLAS_OK;
        }
        enqueue(p, cap_, false);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(cap_, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(PLAS_ERR_CUDA, "sweep launch failed: %s", cudaGetErrorString(le));
        }
        if (ce != cudaSuccess || !graph) {
            cudaGetLastError();
            graphs_failed_ = true;
            return PLAS_OK;
        }
        const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            g->exec = nullptr;
            graphs_failed_ = true;
            return PLAS_OK;
        }
        g->plan = p;
        captures_ += 1;
        return PLAS_OK;
    }

    int host_buffers(size_t bytes) {
        void* h = nullptr;
        if (own_host_) {
            // a buffer of this engine alone (engines that live side by side in
            // one thread must not share the per-thread staging buffer); a
            // grown buffer replaces the old one, which is freed with the engine
            PLAS_CUDA(cudaMallocHost(&h, std::max<size_t>(bytes, 4096)));
            owned_host_.push_back(h);
        } else {
            cudaEvent_t unused[2];
            if (int e = poll_buffers(bytes, &h, unused)) return e;
        }
        host_ = (char*)h;
        if (!ev_[0]) {
            PLAS_CUDA(cudaEventCreateWithFlags(&ev_[0], cudaEventDisableTiming));
            PLAS_CUDA(cudaEventCreateWithFlags(&ev_[1], cudaEventDisableTiming));
        }
        return PLAS_OK;
    }

    // Descriptor array and CTA maps of the active grids (multi-grid sweeps).
    int rebuild() {
        dirty_ = false;
        if (active_.size() <= 1) return PLAS_OK;
        std::vector<GridRef> refs(active_.size());
        for (size_t i = 0; i < active_.size(); ++i) {
            Slot* sl = active_[i];
            GridRef& r = refs[i];
            r.G = sl->ws.G; r.T = sl->ws.T; r.H1 = sl->ws.H1; r.pi = sl->ws.pi; r.st = sl->ws.st;
            r.lv = sl->ws.lv; r.table = sl->ws.table; r.H = sl->job.H; r.W = sl->job.W;
            r.nlev = sl->nlev; r.seed = sl->job.seed;
            r.trace_S = sl->job.trace_S; r.trace_level = sl->job.trace_level;
            r.trace_cap = sl->job.trace_cap;
            r.target_mode = s_.target_mode;
            r.sat = sl->ws.sat;
            r.checked = s_.checked;
            r.edge_blocks = s_.whole_blocks ? 0 : 1;
        }
        // the persistent sweep runs the medium FIR tiling for every grid;
        // separate launches give each grid the variant its last reported
        // radius takes, one launch per variant group and pass
        persist_ = want_persist();
        for (Slot* sl : active_) sl->fvar = persist_ ? kFirMediumRadius : grid_variant(sl);
        nfg_ = 0;
        for (int v = 0; v < kFirTilings; ++v)
            for (const Slot* sl : active_)
                if (sl->fvar == v) {
                    fvar_[nfg_++] = v;
                    break;
                }
        std::vector<CtaMap> maps;
        for (int c = 0; c < kClsCount; ++c) {
            total_[c] = 0;
            if (c == kClsAssign) {
                for (size_t i = 0; i < active_.size(); ++i) {
                    const int n = active_[i]->ctas[c];
                    for (int l = 0; l < n; ++l) maps.push_back(CtaMap{(int)i, l, n, 0});
                    total_[c] += n;
                }
                continue;
            }
            const int pass = c == kClsFirY ? 0 : 1;
            for (int g = 0; g < nfg_; ++g) {
                foff_[pass][g] = total_[c];
                fcnt_[pass][g] = 0;
                for (size_t i = 0; i < active_.size(); ++i) {
                    if (active_[i]->fvar != fvar_[g]) continue;
                    const Job& j = active_[i]->job;
                    const int n = fir_pass_ctas(pass, j.H, j.W, D_, fvar_[g]);
                    for (int l = 0; l < n; ++l) maps.push_back(CtaMap{(int)i, l, n, 0});
                    fcnt_[pass][g] += n;
                    total_[c] += n;
                }
            }
        }
        const size_t need = map_bytes(refs.size(), maps.size());
        if (need > dmaps_cap_) {
            if (arena_) {
                if (need > arena_bytes_) return fail(PLAS_ERR_INTERNAL, "descriptor arena too small");
                dmaps_ = arena_;
                dmaps_cap_ = arena_bytes_;
            } else {
                if (dmaps_ && dmaps_owned_) cudaFreeAsync(dmaps_, st_);  // stream-ordered
                void* p = nullptr;
                if (dev_alloc(&p, need * 2, st_) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(PLAS_ERR_OOM, "descriptor allocation failed");
                }
                dmaps_ = (char*)p;
                dmaps_cap_ = need * 2;
                dmaps_owned_ = true;
            }
        }
        dgrids_ = (GridRef*)dmaps_;
        CtaMap* m = (CtaMap*)(dmaps_ + align_up(refs.size() * sizeof(GridRef), 256));
        size_t o = 0;
        for (int c = 0; c < kClsCount; ++c) {
            dmap_[c] = m + o;
            o += total_[c];
        }
        // Stream-ordered: sweeps already enqueued read the arrays before the
        // copies land.  The sources are pageable, so each copy is staged before
        // the call returns and the vectors may go out of scope.
        PLAS_CUDA(cudaMemcpyAsync(dgrids_, refs.data(), refs.size() * sizeof(GridRef),
                                  cudaMemcpyHostToDevice, st_));
        PLAS_CUDA(cudaMemcpyAsync(m, maps.data(), maps.size() * sizeof(CtaMap),
                                  cudaMemcpyHostToDevice, st_));
        return PLAS_OK;
    }

    int D_;
    Weights w_;
    plas_schedule s_;
    cudaStream_t st_;
    int nsm_;
    std::vector<Slot*> active_;
    std::vector<Slot*> polled_[2];
    bool dirty_ = true;
    char* arena_ = nullptr;
    size_t arena_bytes_ = 0;
    char* dmaps_ = nullptr;
    size_t dmaps_cap_ = 0;
    bool dmaps_owned_ = false;
    GridRef* dgrids_ = nullptr;
    CtaMap* dmap_[kClsCount] = {nullptr, nullptr, nullptr};
    int total_[kClsCount] = {0, 0, 0};
    // FIR variant groups of the multi-grid CTA maps: variant, and per pass the
    // offset into the class's maps and the CTA count
    int nfg_ = 0;
    int fvar_[kFirTilings] = {};
    int foff_[2][kFirTilings] = {};
    int fcnt_[2][kFirTilings] = {};
    bool persist_ = false;  // the next sweeps run as one persistent launch
    char* host_ = nullptr;
    size_t host_cap_ = 0;
    char* polled_base_[2] = {nullptr, nullptr};
    cudaEvent_t ev_[2] = {nullptr, nullptr};
    std::vector<EventPair> marks_;
    std::vector<cudaEvent_t> pool_;
    cudaStream_t cap_ = nullptr;
    Graph graph_[kFirTilings];  // one per FIR tiling
    bool graphs_failed_ = false;
    bool own_host_ = false;
    std::vector<void*> owned_host_;

   public:
    long long captures_ = 0;
    long long graph_launches_ = 0;
    long long persist_launches_ = 0;
};

// Checked runs: every guard band must still hold its pattern.
int verify_guards(const Workspace& ws, cudaStream_t st) {
    unsigned int* bad = reinterpret_cast<unsigned int*>(ws.macc);  // scratch, before the metrics
    unsigned int h = 0;
    PLAS_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), st));
    launch_check_guards(ws.guards, bad, st);
    PLAS_CUDA(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, st));
    PLAS_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(PLAS_ERR_INTERNAL, "checked run: %u guard bytes between workspace regions were overwritten", h);
    return PLAS_OK;
}

int status_error(const DevState& st) {
    if (st.nonfinite) return fail(PLAS_ERR_NONFINITE, "sort input holds NaN or Inf");
    if (st.bad_index) return fail(PLAS_ERR_INVALID_ARG, "perm_init holds an index outside [0, N)");
    if (st.status == PLAS_ERR_TIMEOUT)
        return fail(PLAS_ERR_TIMEOUT, "a bounded device wait gave up (no progress for 2 s)");
    if (st.status == PLAS_ERR_INTERNAL)
        return fail(PLAS_ERR_INTERNAL, "checked run: a grouping entry or cell position outside the grid");
    return fail(PLAS_ERR_INTERNAL, "device status %d", st.status);
}

void to_public(const DevState& d, plas_state* o) {
    o->it = d.it;
    o->epoch = d.epoch;
    o->redraws = d.redraws;
    o->level = d.level;
    o->stall = d.stall;
    o->has_prev = d.has_prev;
    o->done = d.done;
    o->d_prev = d.d_prev;
    o->d_last = d.d_last;
    o->scale_exp = d.scale_exp;
    o->status = d.status;
}

int check_job(const plas_job& j, int D, int* skip) {
    *skip = 0;
    if (j.H < 0 || j.W < 0) return fail(PLAS_ERR_INVALID_ARG, "grid sides must be >= 0");
    const long long N = (long long)j.H * j.W;
    if (!grid_fits(j.H, j.W, D)) return fail(PLAS_ERR_INVALID_ARG, "grid %lldx%lld x %d: needs H*W <= 2^26 and max(H, W)*D <= 2^26", (long long)j.H, (long long)j.W, (int)D);
    if (N == 0) {
        *skip = 1;
        return PLAS_OK;
    }
    if (!j.x || !j.perm_out) return fail(PLAS_ERR_INVALID_ARG, "job needs x and perm_out");
    if (!aligned(j.x, 4) || !aligned(j.perm_out, 4)) return fail(PLAS_ERR_INVALID_ARG, "misaligned pointer");
    if (j.C < 0 || (j.C > 0 && (!j.carried || !j.carried_out)))
        return fail(PLAS_ERR_INVALID_ARG, "carried/carried_out required when C > 0");
    (void)D;
    return PLAS_OK;
}

Job job_from(const plas_job& j) {
    Job o;
    o.x = j.x; o.H = j.H; o.W = j.W; o.carried = j.carried; o.C = j.C; o.seed = j.seed;
    o.perm_out = j.perm_out; o.carried_out = j.carried_out; o.state_out = j.state_out;
    return o;
}

int make_weights(const float* weights, int D, Weights* w) {
    for (int d = 0; d < kMaxD; ++d) w->w[d] = (d < D) ? (weights ? weights[d] : 1.0f) : 0.0f;
    for (int d = 0; d < D; ++d)
        if (!std::isfinite(w->w[d])) return fail(PLAS_ERR_INVALID_ARG, "weights must be finite");
    return PLAS_OK;
}

// Run every admitted grid of 'eng' to completion (batches of k sweeps, one
// batch of look-ahead), retiring grids as they finish.
int run_all(Engine& eng, const plas_schedule& s) {
    const int k = s.iters_per_poll > 0 ? s.iters_per_poll : 8;
    int buf = 0;
    bool pending = false;
    int first_error = PLAS_OK;
    // grids that are finished before the first sweep (e.g. resumed at the end)
    for (auto* sl : std::vector<Slot*>(eng.active()))
        if (finished(*sl, s)) {
            if (sl->last.status && !first_error) first_error = status_error(sl->last);
            if (int e = eng.retire(sl)) return e;
        }
    while (!eng.active().empty()) {
        if (int e = eng.sweeps(k)) return e;
        if (int e = eng.poll(buf)) return e;
        if (pending) {
            if (int e = eng.wait(buf ^ 1)) return e;
            for (auto* sl : std::vector<Slot*>(eng.active()))
                if (finished(*sl, s)) {
                    if (sl->last.status && !first_error) first_error = status_error(sl->last);
                    if (int e = eng.retire(sl)) return e;
                }
        }
        pending = true;
        buf ^= 1;
    }
    if (pending)
        if (int e = eng.wait(buf ^ 1)) return e;  // the last poll
    return first_error;
}

}  // namespace

}  // namespace plas

using namespace plas;

// ===========================================================================
// the sort
// ===========================================================================
extern "C" int plas_sort(const float* x, int H, int W, int D, const float* weights,
                         const float* carried, int C, uint64_t seed, const plas_schedule* sched,
                         const int32_t* perm_init, plas_state* state_io, int32_t* perm_out,
                         float* carried_out, float* sorted_out, void* workspace, size_t ws_bytes,
                         plas_stats* stats, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    set_last_error("");
    if (H < 0 || W < 0) return fail(PLAS_ERR_INVALID_ARG, "grid sides must be >= 0");
    if (!channels_supported(D))
        return fail(PLAS_ERR_INVALID_ARG, "D=%d not supported (1..16, 20, 24, 32, 48, 64)", D);
    const long long N = (long long)H * W;
    if (!grid_fits(H, W, D)) return fail(PLAS_ERR_INVALID_ARG, "grid %lldx%lld x %d: needs H*W <= 2^26 and max(H, W)*D <= 2^26", (long long)H, (long long)W, (int)D);
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
    Weights w{};
    if (int e = make_weights(weights, D, &w)) return e;
    cudaStream_t st = (cudaStream_t)stream;

    Slot sl;
    Job& j = sl.job;
    j.x = x; j.H = H; j.W = W; j.carried = carried; j.C = C; j.seed = seed;
    j.perm_init = perm_init; j.resume = resume;
    if (resume) j.init = *state_io;
    j.perm_out = perm_out; j.carried_out = carried_out; j.sorted_out = sorted_out;
    j.trace_S = s.trace_S; j.trace_level = s.trace_level; j.trace_cap = s.trace_cap;

    const size_t need = sort_workspace_bytes(H, W, D, s);
    if (workspace) {
        if (ws_bytes < need) return fail(PLAS_ERR_INVALID_ARG, "workspace too small (%zu < %zu)", ws_bytes, need);
        if (!aligned(workspace, 256)) return fail(PLAS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        sl.mem = (char*)workspace;
    } else {
        void* mem = nullptr;
        if (dev_alloc(&mem, need, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(PLAS_ERR_OOM, "workspace allocation of %zu bytes failed", need);
        }
        sl.mem = (char*)mem;
        sl.owns = true;
    }
    int rc = PLAS_OK;
    {
        Engine eng(D, w, s, st);
        rc = eng.admit(&sl);
        if (rc == PLAS_OK) rc = run_all(eng, s);
        if (rc == PLAS_OK && s.checked) rc = verify_guards(sl.ws, st);
        if (rc == PLAS_OK && stats) {
            memset(stats, 0, sizeof(*stats));
            double macc[4] = {0, 0, 0, 0};
            if (cudaMemsetAsync(sl.ws.macc, 0, sizeof(double) * 4, st) != cudaSuccess) rc = fail(PLAS_ERR_CUDA, "memset failed");
            launch_neighbour_metrics(sl.ws.G, grid_stride(D), H, W, D, 1.0, sl.ws.macc, num_sms(), st);
            eng.launches_ += 1;
            DevState fin{};
            if (rc == PLAS_OK &&
                (cudaMemcpyAsync(macc, sl.ws.macc, sizeof(double) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(&fin, sl.ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaStreamSynchronize(st) != cudaSuccess))
                rc = fail(PLAS_ERR_CUDA, "stats readback failed");
            if (rc == PLAS_OK) {
                eng.harvest();
                const long long npairs = (long long)H * (W - 1) + (long long)(H - 1) * W;
                stats->iterations = fin.it;
                stats->redraws = fin.redraws;
                stats->grouped_cells = fin.grouped;
                stats->levels = sl.nlev;
                stats->status = fin.status;
                stats->final_l2_to_target = fin.d_last;
                stats->neighbour_l2 = npairs > 0 ? macc[0] / (double)npairs : 0.0;
                for (int c = 0; c < PLAS_K_COUNT; ++c) stats->kernel[c] = eng.ks_[c];
                const double its = (double)(fin.it - (resume ? state_io->it : 0));
                stats->kernel[PLAS_K_PREP].bytes = (double)N * D * 8 + (double)N * grid_stride(D) * 4;
                // target: read the features, write the target (8 N D bytes per
                // iteration); the Gaussian takes two passes, each counted in full,
                // except in iterations whose pass-0 launch ran both passes (fused
                // small-radius kernel): their work is all in BLUR_COLS
                stats->kernel[PLAS_K_BLUR_COLS].bytes = its * 8.0 * (double)N * D;
                stats->kernel[PLAS_K_BLUR_COLS].flops = 2.0 * (fin.fmas_y + fin.fmas_xf);
                stats->kernel[PLAS_K_BLUR_ROWS].bytes =
                    s.target_mode == 1 ? 0.0 : (its - (double)fin.fused_its) * 8.0 * (double)N * D;
                stats->kernel[PLAS_K_BLUR_ROWS].flops = 2.0 * fin.fmas_x;
                // the grouping table is written by the pass-0 launches
                stats->kernel[PLAS_K_BLUR_COLS].bytes += 4.0 * fin.beta2_sum;
                stats->kernel[PLAS_K_ASSIGN].bytes =
                    (double)fin.grouped * (12.0 * D + 8.0) + (its * N - (double)fin.grouped) * 8.0 * D;
                stats->kernel[PLAS_K_GATHER].bytes = (double)N * 8 + (carried_out ? (double)N * C * 8 : 0.0) +
                                                     (sorted_out ? (double)N * D * 8 : 0.0);
                stats->launches = eng.launches_;
                stats->graph_launches = eng.graph_launches_;
                stats->graph_captures = eng.captures_;
            }
        } else if (rc == PLAS_OK) {
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = fail(PLAS_ERR_CUDA, "stream sync failed");
        }
        if (rc == PLAS_OK && state_io) to_public(sl.last, state_io);
        if (rc != PLAS_OK && state_io && sl.last.status) to_public(sl.last, state_io);
    }
    if (sl.owns) cudaFreeAsync(sl.mem, st);
    if (stats && rc == PLAS_OK)
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

// ===========================================================================
// launch-shape autotuning
// ===========================================================================
namespace {

// Mean device time (us) of 'reps' runs of fn, after one warm-up run.
template <class F>
int time_us(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int reps, F fn, float* us) {
    fn();
    PLAS_CUDA(cudaEventRecord(a, st));
    for (int i = 0; i < reps; ++i) fn();
    PLAS_CUDA(cudaEventRecord(b, st));
    PLAS_CUDA(cudaEventSynchronize(b));
    if (int e = check_launch("autotune")) return e;
    float ms = 0.0f;
    PLAS_CUDA(cudaEventElapsedTime(&ms, a, b));
    *us = ms * 1000.0f / (float)reps;
    return PLAS_OK;
}

int autotune_run(int H, int W, int D, cudaStream_t st, float* x, char* ws, cudaEvent_t a,
                 cudaEvent_t b, plas_tuning* out) {
    plas_schedule s;
    plas_default_schedule(&s);
    s.graphs = 0;
    const int rtop = std::max(1, (int)std::floor(start_radius(s, H, W)));
    std::vector<int> radii;
    for (int r : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512})
        if (r <= rtop && (int)radii.size() < PLAS_TUNE_MAX_RADII - 1) radii.push_back(r);
    if (radii.back() != rtop) radii.push_back(rtop);
    const int assign_r[2] = {rtop, std::min(8, rtop)};
    const int per_sm[PLAS_TUNE_ASSIGN_CANDIDATES] = {2, 4, 8, 16};
    float assign_us[PLAS_TUNE_ASSIGN_CANDIDATES] = {0, 0, 0, 0};
    Weights w{};
    if (int e = make_weights(nullptr, D, &w)) return e;
    const int nsm = num_sms();
    constexpr int kReps = 5;
    out->n_radii = (int)radii.size();
    for (size_t i = 0; i < radii.size(); ++i) {
        const int r = radii[i];
        plas_schedule sr = s;
        sr.phi0 = (double)r;  // level 0 has radius r
        Engine eng(D, w, sr, st);
        Slot sl;
        sl.job.x = x;
        sl.job.H = H;
        sl.job.W = W;
        sl.job.seed = 1;
        sl.mem = ws;
        if (int e = eng.admit(&sl)) return e;
        out->radius[i] = r;
        for (int var : {kFirLargeRadius + 100, kFirLargeRadius, kFirMediumRadius, kFirSmallRadius}) {
            if (var == kFirSmallRadius && r > kDirectTuneMaxR) {  // correct, but slow there
                out->fir_small_us[i] = -1.0f;
                continue;
            }
            if (var == kFirLargeRadius + 100) {  // the large tiling with tensor copies
                out->fir_large_tma_us[i] = -1.0f;
                if (!sl.tma.ok) continue;
                const int c0 = fir_ctas(H, W * D, kFirLargeRadius), c1 = fir_ctas(W, H * D, kFirLargeRadius);
                float us = 0.0f;
                if (int e = time_us(st, a, b, kReps, [&] {
                        launch_fir(0, sl.ws.ref, nullptr, c0, D, kFirLargeRadius, st, &sl.tma);
                        launch_fir(1, sl.ws.ref, nullptr, c1, D, kFirLargeRadius, st, &sl.tma);
                    }, &us))
                    return e;
                out->fir_large_tma_us[i] = us;
                continue;
            }
            // the small-radius path: the one-launch kernel where it applies
            Tuning small_only;
            small_only.small_below = r + 1;
            const int kv = var == kFirSmallRadius ? fir_variant(r, D, small_only) : var;
            const int c0 = fir_pass_ctas(0, H, W, D, kv), c1 = fir_pass_ctas(1, H, W, D, kv);
            float us = 0.0f;
            if (int e = time_us(st, a, b, kReps, [&] {
                    launch_fir(0, sl.ws.ref, nullptr, c0, D, kv, st);
                    launch_fir(1, sl.ws.ref, nullptr, c1, D, kv, st);
                }, &us))
                return e;
            (var == kFirSmallRadius ? out->fir_small_us
             : var == kFirMediumRadius ? out->fir_medium_us : out->fir_large_us)[i] = us;
        }
        for (int k = 0; k < 2; ++k) {
            if (r != assign_r[k] || (k == 1 && assign_r[1] == assign_r[0])) continue;
            for (int c = 0; c < PLAS_TUNE_ASSIGN_CANDIDATES; ++c) {
                const int ctas = assign_ctas(H, W, nsm, per_sm[c]);
                float us = 0.0f;
                if (int e = time_us(st, a, b, kReps, [&] {
                        launch_assign(sl.ws.ref, nullptr, ctas, D, s.tol, st);
                    }, &us))
                    return e;
                assign_us[c] += us;
            }
        }
    }
    // the large tiling: tensor copies where they are faster summed over the
    // measured radii (both variants give the same bits)
    double ring_sum = 0.0, tma_sum = 0.0;
    bool tma_all = true;
    for (size_t i = 0; i < radii.size(); ++i) {
        out->fir_large_ring_us[i] = out->fir_large_us[i];
        ring_sum += out->fir_large_us[i];
        tma_sum += out->fir_large_tma_us[i];
        tma_all = tma_all && out->fir_large_tma_us[i] > 0.0f;
    }
    const int large_tma = tma_all && tma_sum < ring_sum ? 1 : 0;
    if (large_tma)
        for (size_t i = 0; i < radii.size(); ++i) out->fir_large_us[i] = out->fir_large_tma_us[i];
    // the two thresholds (small <= medium) that minimise the summed time over
    // the measured radii
    Tuning best;
    double best_cost = -1.0;
    for (size_t j = 0; j <= radii.size(); ++j) {
        for (size_t m = j; m <= radii.size(); ++m) {
            Tuning t;
            t.small_below = j < radii.size() ? radii[j] : rtop + 1;
            t.medium_below = m < radii.size() ? radii[m] : rtop + 1;
            double cost = 0.0;
            for (size_t i = 0; i < radii.size(); ++i) {
                const int v = fir_tiling(radii[i], t);
                const float us = v == kFirSmallRadius ? out->fir_small_us[i]
                                 : v == kFirMediumRadius ? out->fir_medium_us[i] : out->fir_large_us[i];
                cost += us < 0.0f ? 1e30 : us;  // not measured: never chosen
            }
            if (best_cost < 0.0 || cost < best_cost) {
                best_cost = cost;
                best = t;
            }
        }
    }
    int best_c = 0;
    for (int c = 0; c < PLAS_TUNE_ASSIGN_CANDIDATES; ++c) {
        out->assign_per_sm[c] = per_sm[c];
        out->assign_us[c] = assign_us[c];
        if (assign_us[c] < assign_us[best_c]) best_c = c;
    }
    out->fir_small_below = best.small_below;
    out->fir_medium_below = best.medium_below;
    out->assign_ctas_per_sm = per_sm[best_c];
    out->large_tma = large_tma;
    out->small_fused = 1;
    Tuning tu = best;
    tu.assign_per_sm = per_sm[best_c];
    tu.large_tma = large_tma;
    install_tuning(H, W, D, &tu);
    return PLAS_OK;
}

}  // namespace

extern "C" int plas_autotune(int H, int W, int D, void* stream, plas_tuning* out) {
    set_last_error("");
    if (!out) return fail(PLAS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    if (H < 1 || W < 1 || !channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "bad shape");
    const long long N = (long long)H * W;
    if (!grid_fits(H, W, D)) return fail(PLAS_ERR_INVALID_ARG, "grid %lldx%lld x %d: needs H*W <= 2^26 and max(H, W)*D <= 2^26", (long long)H, (long long)W, (int)D);
    cudaStream_t st = (cudaStream_t)stream;
    plas_schedule s;
    plas_default_schedule(&s);
    const size_t ws_bytes = sort_workspace_bytes(H, W, D, s);
    void* x = nullptr;
    void* ws = nullptr;
    if (dev_alloc(&x, (size_t)N * D * sizeof(float), st) != cudaSuccess ||
        dev_alloc(&ws, ws_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        if (x) cudaFreeAsync(x, st);
        return fail(PLAS_ERR_OOM, "autotune buffers");
    }
    launch_fill_uniform((float*)x, N * D, 0x7475ull, st);
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = PLAS_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        rc = fail(PLAS_ERR_CUDA, "event creation failed");
    if (rc == PLAS_OK) rc = autotune_run(H, W, D, st, (float*)x, (char*)ws, a, b, out);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(x, st);
    cudaFreeAsync(ws, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == PLAS_OK)
        rc = fail(PLAS_ERR_CUDA, "stream sync failed");
    return rc;
}

// ===========================================================================
// batched sort
// ===========================================================================
static size_t batch_bytes(int n, const plas_job* jobs, int D, const plas_schedule& s,
                          std::vector<size_t>* per_job, size_t* maps_at) {
    size_t total = 0, grids = 0, ctas = 0;
    const int nsm = num_sms();
    if (per_job) per_job->assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const int H = jobs[i].H, W = jobs[i].W;
        if (H < 1 || W < 1) continue;
        const size_t b = align_up(sort_workspace_bytes(H, W, D, s), 256);
        if (per_job) (*per_job)[i] = b;
        total += b;
        grids += 1;
        // CTA maps sized for the FIR variant with the most tiles (a grid's
        // variant follows its radius)
        for (int pass = 0; pass < 2; ++pass) {
            int m = 0;
            for (int v = 0; v < kFirTilings; ++v)
                if (v < kFirFused || D <= kFusedMaxD) m = std::max(m, fir_pass_ctas(pass, H, W, D, v));
            ctas += m;
        }
        ctas += assign_ctas(H, W, nsm, kAssignMaxPerSm);
    }
    if (maps_at) *maps_at = total;
    return total + Engine::map_bytes(grids, ctas);
}

extern "C" size_t plas_batch_workspace_bytes(int n, const plas_job* jobs, int D) {
    if (n < 0 || (n > 0 && !jobs) || !channels_supported(D)) return 0;
    plas_schedule s;
    plas_default_schedule(&s);
    return batch_bytes(n, jobs, D, s, nullptr, nullptr);
}

struct plas_server;
namespace {
int run_lane_batch(int n, const plas_job* jobs, int D, const Weights& w, const plas_schedule& s,
                   char* base, const std::vector<size_t>& per, cudaStream_t st);
}  // namespace

extern "C" int plas_batch_sort(int n, const plas_job* jobs, int D, const float* weights,
                               const plas_schedule* sched, void* workspace, size_t ws_bytes,
                               void* stream) {
    set_last_error("");
    if (n < 0 || (n > 0 && !jobs)) return fail(PLAS_ERR_INVALID_ARG, "bad job list");
    if (!channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "D=%d not supported", D);
    plas_schedule s;
    if (sched) s = *sched; else plas_default_schedule(&s);
    s.trace_S = nullptr;  // traces are a single-sort facility
    s.trace_level = nullptr;
    s.trace_cap = 0;
    if (int e = validate_schedule(s)) return e;
    Weights w{};
    if (int e = make_weights(weights, D, &w)) return e;
    for (int i = 0; i < n; ++i) {
        int skip = 0;
        if (int e = check_job(jobs[i], D, &skip)) return e;
        if (skip && jobs[i].state_out) {
            memset(jobs[i].state_out, 0, sizeof(plas_state));
            jobs[i].state_out->done = 1;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<size_t> per;
    size_t maps_at = 0;
    const size_t need = batch_bytes(n, jobs, D, s, &per, &maps_at);
    char* base = nullptr;
    bool owns = false;
    if (workspace) {
        if (ws_bytes < need) return fail(PLAS_ERR_INVALID_ARG, "batch workspace too small (%zu < %zu)", ws_bytes, need);
        if (!aligned(workspace, 256)) return fail(PLAS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        base = (char*)workspace;
    } else {
        void* p = nullptr;
        if (dev_alloc(&p, need, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(PLAS_ERR_OOM, "batch workspace allocation of %zu bytes failed", need);
        }
        base = (char*)p;
        owns = true;
    }
    int rc = PLAS_OK;
    if (s.target_mode == 1) {
        // the box target: the inputs are ready on the caller's stream, each
        // grid then runs on a lane of its own
        rc = run_lane_batch(n, jobs, D, w, s, base, per, st);
        if (owns) cudaFreeAsync(base, st);
        return rc;
    }
    {
        std::vector<std::unique_ptr<Slot>> slots;
        Engine eng(D, w, s, st);
        eng.set_arena(base + maps_at, need - maps_at);
        size_t off = 0;
        for (int i = 0; i < n && rc == PLAS_OK; ++i) {
            if (per[i] == 0) continue;
            auto sl = std::make_unique<Slot>();
            sl->job = job_from(jobs[i]);
            sl->mem = base + off;
            off += per[i];
            rc = eng.admit(sl.get());
            slots.push_back(std::move(sl));
        }
        if (rc == PLAS_OK) rc = run_all(eng, s);
        if (rc == PLAS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(PLAS_ERR_CUDA, "stream sync failed");
        if (rc == PLAS_OK)
            for (auto& sl : slots)
                if (sl->job.state_out) to_public(sl->last, sl->job.state_out);
    }
    if (owns) cudaFreeAsync(base, st);
    return rc;
}

// ===========================================================================
// served sorts (continuous batching)
// ===========================================================================
struct plas_server {
    int D = 0;
    Weights w{};
    plas_schedule s{};
    size_t budget = 0;
    size_t in_use = 0;
    cudaStream_t st = nullptr;
    int policy = PLAS_SERVE_FIFO_FILL;
    std::unique_ptr<Engine> eng;
    std::deque<std::unique_ptr<Slot>> queue;
    std::vector<std::unique_ptr<Slot>> running;  // admitted, in admission order
    struct Retiring {
        cudaEvent_t ev;
        Slot* sl;
    };
    std::vector<Retiring> retiring;  // outputs enqueued, not yet known complete
    // host records of finished requests, kept until no read-back in flight
    // can name them
    std::vector<std::pair<long long, std::unique_ptr<Slot>>> graveyard;
    std::vector<cudaEvent_t> events;
    std::vector<long long> completed;  // finished, not yet reported
    long long next_ticket = 0;
    long long step_no = 0;
    int buf = 0;
    bool pending = false;  // a state read-back is in flight
    // PLAS_SERVE_CONCURRENT: one lane (stream + engine) per admitted request
    struct Lane {
        std::unique_ptr<Slot> sl;
        cudaStream_t st = nullptr;
        std::unique_ptr<Engine> eng;
        int buf = 0;
        int inflight = 0;        // batches whose state read-back is not consumed
        cudaEvent_t done = nullptr;  // after the outputs, once retired
        bool head = false;       // on the high-priority stream
        std::vector<cudaStream_t> old_streams;  // left when promoted (destroyed with the lane)
    };
    std::vector<std::unique_ptr<Lane>> lanes;
    int prio_least = 0, prio_greatest = 0;
    int first_error = 0;  // a lane's grid that ended with a device status
};

namespace {

// Estimated device time of the rest of a sort from each level on: per level
// about 53 iterations (the mean of measured full schedules), each costing the
// two target passes (4 flops per in-range tap and channel, at the ~43 TFLOP/s
// the FIR kernel sustains), the assignment (~0.06 ns per cell) and a launch
// floor of 15 us.  Only the order of these numbers matters.
void plan_slot(Slot* sl, int D) {
    const double N = (double)sl->N;
    const int H = sl->job.H, W = sl->job.W;
    sl->it_ns.assign(sl->nlev, 0.0);
    sl->rem_ns.assign(sl->nlev + 1, 0.0);
    for (int L = sl->nlev - 1; L >= 0; --L) {
        const int r = sl->geo.lv[L].r;
        const double ty = std::min(2.0 * r + 1, (double)H), tx = std::min(2.0 * r + 1, (double)W);
        sl->it_ns[L] = N * D * (tx + ty) * 4.0 / 43.0 + N * 0.06 + 15000.0;
        sl->rem_ns[L] = sl->rem_ns[L + 1] + 53.0 * sl->it_ns[L];
    }
}

int level_of(const Slot* sl) {
    return std::min(std::max(sl->last.level, 0), (int)sl->it_ns.size() - 1);
}

// The grids the next batch of sweeps advances.  FIFO_FILL: admission order;
// SHORTEST_FIRST: least estimated work left first; both take grids until the
// estimated time of one sweep over them reaches kFillNs (a grid at a large
// radius fills a sweep alone; grids at small radii, whose launches are too
// short to fill the GPU, share one).  ALL: every admitted grid.  The window
// was measured at 0.6, 1.5 and 3 ms per sweep on 64 served requests: 3 ms
// gave the highest throughput and the lowest p99 of the three (Poisson
// arrivals and overload).
constexpr double kFillNs = 3000000.0;

// ADAPTIVE: FIFO_FILL while fewer than kBacklog requests are admitted (the
// oldest request runs nearly alone, as on the plain path), ALL under a
// backlog, where sweeping many grids together raises throughput.
constexpr size_t kBacklog = 8;

std::vector<Slot*> choose(plas_server* srv) {
    std::vector<Slot*> cand;
    for (auto& p : srv->running)
        if (p->active && !finished(*p, srv->s)) cand.push_back(p.get());
    if (srv->policy == PLAS_SERVE_ALL) return cand;
    if (srv->policy == PLAS_SERVE_ADAPTIVE && cand.size() >= kBacklog) return cand;
    if (srv->policy == PLAS_SERVE_SHORTEST_FIRST)
        std::stable_sort(cand.begin(), cand.end(), [](const Slot* a, const Slot* b) {
            return a->rem_ns[level_of(a)] < b->rem_ns[level_of(b)];
        });
    std::vector<Slot*> run;
    double t = 0.0;
    for (Slot* sl : cand) {
        run.push_back(sl);
        t += sl->it_ns[level_of(sl)];
        if (t >= kFillNs) break;
    }
    return run;
}

}  // namespace

extern "C" int plas_server_create(int D, const float* weights, const plas_schedule* sched,
                                  size_t mem_budget, void* stream, plas_server** out) {
    set_last_error("");
    if (!out) return fail(PLAS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!channels_supported(D)) return fail(PLAS_ERR_INVALID_ARG, "D=%d not supported", D);
    auto srv = std::make_unique<plas_server>();
    srv->D = D;
    if (int e = make_weights(weights, D, &srv->w)) return e;
    if (sched) srv->s = *sched; else plas_default_schedule(&srv->s);
    srv->s.trace_S = nullptr;
    srv->s.trace_level = nullptr;
    srv->s.trace_cap = 0;
    if (int e = validate_schedule(srv->s)) return e;
    // the box target runs one grid per launch: its requests take the
    // concurrent policy, one lane (stream + engine) each
    if (srv->s.target_mode == 1) srv->policy = PLAS_SERVE_CONCURRENT;
    srv->budget = mem_budget;
    srv->st = (cudaStream_t)stream;
    srv->eng = std::make_unique<Engine>(D, srv->w, srv->s, srv->st);
    srv->eng->own_host_buffers();
    if (cudaDeviceGetStreamPriorityRange(&srv->prio_least, &srv->prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        srv->prio_least = srv->prio_greatest = 0;
    }
    *out = srv.release();
    return PLAS_OK;
}

extern "C" int plas_server_set_policy(plas_server* srv, int policy) {
    set_last_error("");
    if (!srv) return fail(PLAS_ERR_INVALID_ARG, "NULL server");
    if (policy < PLAS_SERVE_FIFO_FILL || policy > PLAS_SERVE_ADAPTIVE)
        return fail(PLAS_ERR_INVALID_ARG, "unknown policy %d", policy);
    if (srv->s.target_mode == 1 && policy != PLAS_SERVE_CONCURRENT)
        return fail(PLAS_ERR_INVALID_ARG, "the box target is served by the concurrent policy only");
    const bool lanes_now = srv->policy == PLAS_SERVE_CONCURRENT;
    const bool lanes_next = policy == PLAS_SERVE_CONCURRENT;
    if (lanes_now != lanes_next && (!srv->running.empty() || !srv->lanes.empty()))
        return fail(PLAS_ERR_INVALID_ARG,
                    "switching to or from the concurrent policy needs a server with nothing admitted");
    srv->policy = policy;
    return PLAS_OK;
}

extern "C" int plas_server_submit(plas_server* srv, const plas_job* job, long long* ticket) {
    set_last_error("");
    if (!srv || !job) return fail(PLAS_ERR_INVALID_ARG, "NULL server or job");
    int skip = 0;
    if (int e = check_job(*job, srv->D, &skip)) return e;
    auto sl = std::make_unique<Slot>();
    sl->job = job_from(*job);
    sl->job.ticket = srv->next_ticket++;
    if (ticket) *ticket = sl->job.ticket;
    if (skip) {
        if (job->state_out) {
            memset(job->state_out, 0, sizeof(plas_state));
            job->state_out->done = 1;
        }
        srv->completed.push_back(sl->job.ticket);
        return PLAS_OK;
    }
    sl->bytes = align_up(sort_workspace_bytes(job->H, job->W, srv->D, srv->s), 256);
    if (srv->budget && sl->bytes > srv->budget)
        return fail(PLAS_ERR_BUDGET, "request needs %zu bytes, budget is %zu", sl->bytes, srv->budget);
    srv->queue.push_back(std::move(sl));
    return PLAS_OK;
}

// One server step.  The host never waits for the sweeps it has just
// enqueued: it reads the state of the previous step's batch (one batch
// behind, as plas_sort does), so the GPU always has a batch queued while the
// host retires, admits and chooses.
namespace {

// PLAS_SERVE_CONCURRENT: every admitted request advances on its own stream
// with its own one-grid engine (graph-replayed batches of sweeps, two batches
// in flight, state read one batch behind), so requests progress at their own
// pace.  The oldest admitted request runs on a stream of the highest
// priority, the others at the lowest: the block scheduler gives the oldest
// request's CTAs the SMs first, as the plain one-at-a-time path would, and
// the younger requests fill the SMs it leaves idle (small grids and small
// radii do not fill the GPU).  When the oldest finishes, the next oldest moves
// to the high-priority stream.
int step_concurrent(plas_server* srv, int sweeps, long long* done, int cap, int* n_done) {
    constexpr size_t kMaxLanes = 16;
    const plas_schedule& s = srv->s;
    const int k = sweeps > 0 ? sweeps : 1;
    // cancellations
    for (auto& ln : srv->lanes) {
        Slot* sl = ln->sl.get();
        if (!sl->cancel || ln->done) continue;
        ln->eng->drop(sl);
        if (sl->owns) cudaFreeAsync(sl->mem, ln->st);
        sl->mem = nullptr;
        srv->in_use -= sl->bytes;
        PLAS_CUDA(cudaEventCreateWithFlags(&ln->done, cudaEventDisableTiming));
        PLAS_CUDA(cudaEventRecord(ln->done, ln->st));
    }
    // admission: FIFO into free lanes while the budget allows
    while (!srv->queue.empty() && srv->lanes.size() < kMaxLanes) {
        Slot* sl = srv->queue.front().get();
        if (srv->budget && srv->in_use + sl->bytes > srv->budget) break;
        auto ln = std::make_unique<plas_server::Lane>();
        sl->N = (long long)sl->job.H * sl->job.W;
        sl->geo = build_geometry(srv->s, sl->job.H, sl->job.W);
        sl->nlev = (int)sl->geo.lv.size();
        plan_slot(sl, srv->D);
        const bool head = srv->lanes.empty();
        PLAS_CUDA(cudaStreamCreateWithPriority(&ln->st, cudaStreamNonBlocking,
                                               head ? srv->prio_greatest : srv->prio_least));
        ln->head = head;
        // the request's inputs were written on the server's stream
        cudaEvent_t ready = nullptr;
        PLAS_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        PLAS_CUDA(cudaEventRecord(ready, srv->st));
        PLAS_CUDA(cudaStreamWaitEvent(ln->st, ready, 0));
        cudaEventDestroy(ready);
        if (!sl->mem) {  // (a batch hands its requests carved workspaces)
            void* mem = nullptr;
            if (dev_alloc(&mem, sl->bytes, ln->st) != cudaSuccess) {
                cudaGetLastError();
                cudaStreamDestroy(ln->st);
                if (srv->lanes.empty()) return fail(PLAS_ERR_OOM, "workspace allocation failed");
                break;
            }
            sl->mem = (char*)mem;
            sl->owns = true;
        }
        srv->in_use += sl->bytes;
        // lanes run side by side: no cooperative launches (they would compete
        // for co-residency)
        plas_schedule ls = srv->s;
        ls.persistent = -1;
        ln->eng = std::make_unique<Engine>(srv->D, srv->w, ls, ln->st);
        ln->eng->own_host_buffers();
        if (int e = ln->eng->admit(sl)) return e;
        ln->sl = std::move(srv->queue.front());
        srv->queue.pop_front();
        srv->lanes.push_back(std::move(ln));
    }
    // feed every lane up to two batches; consume landed read-backs
    bool progress = false;
    for (auto& lp : srv->lanes) {
        plas_server::Lane& ln = *lp;
        if (ln.done) continue;
        Slot* sl = ln.sl.get();
        if (ln.inflight > 0 && ln.eng->poll_ready(ln.buf ^ (ln.inflight == 2 ? 0 : 1))) {
            const int oldest = ln.inflight == 2 ? ln.buf : ln.buf ^ 1;
            if (int e = ln.eng->wait(oldest)) return e;
            ln.inflight -= 1;
            progress = true;
            if (finished(*sl, s)) {
                if (int e = ln.eng->retire(sl)) return e;
                if (sl->owns) cudaFreeAsync(sl->mem, ln.st);
                sl->mem = nullptr;
                srv->in_use -= sl->bytes;
                PLAS_CUDA(cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming));
                PLAS_CUDA(cudaEventRecord(ln.done, ln.st));
                continue;
            }
        }
        while (ln.inflight < 2) {
            if (int e = ln.eng->sweeps(k)) return e;
            if (int e = ln.eng->poll(ln.buf)) return e;
            ln.buf ^= 1;
            ln.inflight += 1;
            progress = true;
        }
    }
    // completions (a lane's stream has finished its outputs)
    for (size_t i = 0; i < srv->lanes.size();) {
        plas_server::Lane& ln = *srv->lanes[i];
        if (!ln.done) {
            ++i;
            continue;
        }
        const cudaError_t q = cudaEventQuery(ln.done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess) return fail(PLAS_ERR_CUDA, "output copies failed: %s", cudaGetErrorString(q));
        Slot* sl = ln.sl.get();
        if (!sl->cancel) {
            if (sl->job.state_out) to_public(sl->last, sl->job.state_out);
            if (sl->last.status && !srv->first_error) srv->first_error = status_error(sl->last);
            srv->completed.push_back(sl->job.ticket);
        }
        cudaEventDestroy(ln.done);
        ln.eng.reset();
        cudaStreamDestroy(ln.st);
        for (cudaStream_t o : ln.old_streams) cudaStreamDestroy(o);
        srv->lanes.erase(srv->lanes.begin() + i);
        progress = true;
    }
    // the oldest unfinished request takes the high-priority stream
    for (auto& lp : srv->lanes) {
        if (lp->done) continue;
        if (!lp->head) {
            cudaStream_t hs = nullptr;
            PLAS_CUDA(cudaStreamCreateWithPriority(&hs, cudaStreamNonBlocking, srv->prio_greatest));
            if (int e = lp->eng->move_to_stream(hs)) return e;
            lp->old_streams.push_back(lp->st);
            lp->st = hs;
            lp->head = true;
        }
        break;
    }
    // nothing moved: wait for the oldest read-back rather than spin
    if (!progress) {
        for (auto& lp : srv->lanes) {
            if (lp->done) {
                cudaEventSynchronize(lp->done);
                break;
            }
            if (lp->inflight > 0) {
                lp->eng->sync_poll(lp->inflight == 2 ? lp->buf : lp->buf ^ 1);
                break;
            }
        }
    }
    const int n = std::min<int>(cap, (int)srv->completed.size());
    for (int i = 0; i < n; ++i) done[i] = srv->completed[i];
    srv->completed.erase(srv->completed.begin(), srv->completed.begin() + n);
    *n_done = n;
    return PLAS_OK;
}

}  // namespace

namespace {

// A batch under the box target: every grid on a lane of its own (the box
// kernels run one grid per launch), in the carved workspaces of the batch.
int run_lane_batch(int n, const plas_job* jobs, int D, const Weights& w, const plas_schedule& s,
                   char* base, const std::vector<size_t>& per, cudaStream_t st) {
    plas_server srv;
    srv.D = D;
    srv.w = w;
    srv.s = s;
    srv.st = st;
    srv.policy = PLAS_SERVE_CONCURRENT;
    if (cudaDeviceGetStreamPriorityRange(&srv.prio_least, &srv.prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        srv.prio_least = srv.prio_greatest = 0;
    }
    size_t off = 0;
    int pending = 0;
    for (int i = 0; i < n; ++i) {
        if (per[i] == 0) continue;
        auto sl = std::make_unique<Slot>();
        sl->job = job_from(jobs[i]);
        sl->job.ticket = i;
        sl->mem = base + off;
        sl->bytes = per[i];
        off += per[i];
        srv.queue.push_back(std::move(sl));
        ++pending;
    }
    std::vector<long long> done((size_t)std::max(n, 1));
    int rc = PLAS_OK;
    while (pending > 0) {
        int got = 0;
        rc = step_concurrent(&srv, s.iters_per_poll > 0 ? s.iters_per_poll : 8, done.data(), n, &got);
        if (rc != PLAS_OK) break;
        pending -= got;
    }
    // the lanes' work is ordered before anything later on the caller's stream
    for (auto& ln : srv.lanes) {
        cudaStreamSynchronize(ln->st);
        if (ln->done) cudaEventDestroy(ln->done);
        ln->eng.reset();
        cudaStreamDestroy(ln->st);
        for (cudaStream_t o : ln->old_streams) cudaStreamDestroy(o);
    }
    srv.lanes.clear();
    if (rc == PLAS_OK) rc = srv.first_error;
    return rc;
}

}  // namespace

extern "C" int plas_server_step(plas_server* srv, int sweeps, long long* done, int cap,
                                int* n_done) {
    set_last_error("");
    if (!srv || !n_done || sweeps < 0 || cap < 0 || (cap > 0 && !done))
        return fail(PLAS_ERR_INVALID_ARG, "bad arguments");
    *n_done = 0;
    srv->step_no += 1;
    if (srv->policy == PLAS_SERVE_CONCURRENT) return step_concurrent(srv, sweeps, done, cap, n_done);
    Engine& eng = *srv->eng;
    // cancelled requests leave the sweeps; their memory is released after
    // the work already queued on them, and their host records are kept while
    // a read-back in flight can name them
    for (size_t i = 0; i < srv->running.size();) {
        Slot* sl = srv->running[i].get();
        if (!sl->cancel) {
            ++i;
            continue;
        }
        eng.drop(sl);
        cudaFreeAsync(sl->mem, srv->st);
        sl->mem = nullptr;
        srv->in_use -= sl->bytes;
        srv->graveyard.emplace_back(srv->step_no, std::move(srv->running[i]));
        srv->running.erase(srv->running.begin() + i);
    }
    // admission: FIFO, while the next request fits the budget
    while (!srv->queue.empty()) {
        Slot* sl = srv->queue.front().get();
        if (srv->budget && srv->in_use + sl->bytes > srv->budget) break;
        void* mem = nullptr;
        if (dev_alloc(&mem, sl->bytes, srv->st) != cudaSuccess) {
            cudaGetLastError();
            if (srv->running.empty()) return fail(PLAS_ERR_OOM, "workspace allocation failed");
            break;  // wait for running requests to release memory
        }
        sl->mem = (char*)mem;
        sl->owns = true;
        srv->in_use += sl->bytes;
        if (int e = eng.admit(sl)) return e;
        plan_slot(sl, srv->D);
        srv->running.push_back(std::move(srv->queue.front()));
        srv->queue.pop_front();
    }
    // sweeps over the chosen grids, then a read-back of their state
    const std::vector<Slot*> run = choose(srv);
    eng.select(run);
    const bool swept = !run.empty();
    if (swept) {
        if (int e = eng.sweeps(sweeps > 0 ? sweeps : 1)) return e;
        if (int e = eng.poll(srv->buf)) return e;
    }
    // the previous read-back: retire the grids it shows finished
    if (srv->pending) {
        const int pb = srv->buf ^ 1;  // this step's read-back, if any, went to buf
        if (int e = eng.wait(pb)) return e;
        for (Slot* sl : std::vector<Slot*>(eng.polled(pb))) {
            if (!sl->active || !finished(*sl, srv->s)) continue;
            if (int e = eng.retire(sl)) return e;
            cudaEvent_t ev = nullptr;
            if (!srv->events.empty()) {
                ev = srv->events.back();
                srv->events.pop_back();
            } else {
                PLAS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            }
            PLAS_CUDA(cudaEventRecord(ev, srv->st));
            // stream-ordered: the memory is reused only by work queued later
            cudaFreeAsync(sl->mem, srv->st);
            sl->mem = nullptr;
            srv->in_use -= sl->bytes;
            srv->retiring.push_back({ev, sl});
        }
    }
    srv->pending = swept;
    if (swept) srv->buf ^= 1;
    // completions: outputs whose copies have finished (wait only when no
    // other work is queued, so an idle server does not spin)
    const bool block = !swept;
    for (size_t i = 0; i < srv->retiring.size();) {
        auto& r = srv->retiring[i];
        const cudaError_t q = block ? cudaEventSynchronize(r.ev) : cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess) return fail(PLAS_ERR_CUDA, "output copies failed: %s", cudaGetErrorString(q));
        Slot* sl = r.sl;
        if (sl->job.state_out) to_public(sl->last, sl->job.state_out);
        srv->completed.push_back(sl->job.ticket);
        srv->events.push_back(r.ev);
        auto it = std::find_if(srv->running.begin(), srv->running.end(),
                               [sl](const std::unique_ptr<Slot>& p) { return p.get() == sl; });
        srv->graveyard.emplace_back(srv->step_no, std::move(*it));
        srv->running.erase(it);
        srv->retiring.erase(srv->retiring.begin() + i);
    }
    // a finished slot can be named by at most the read-back of the step that
    // retired it, which the next step consumes
    srv->graveyard.erase(std::remove_if(srv->graveyard.begin(), srv->graveyard.end(),
                                        [srv](const std::pair<long long, std::unique_ptr<Slot>>& g) {
                                            return !srv->pending || g.first + 2 <= srv->step_no;
                                        }),
                         srv->graveyard.end());
    const int n = std::min<int>(cap, (int)srv->completed.size());
    for (int i = 0; i < n; ++i) done[i] = srv->completed[i];
    srv->completed.erase(srv->completed.begin(), srv->completed.begin() + n);
    *n_done = n;
    return PLAS_OK;
}

extern "C" int plas_server_cancel(plas_server* srv, long long ticket) {
    set_last_error("");
    if (!srv) return fail(PLAS_ERR_INVALID_ARG, "NULL server");
    for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
        if ((*it)->job.ticket == ticket) {
            srv->queue.erase(it);
            return PLAS_OK;
        }
    for (auto& p : srv->running)
        if (p->job.ticket == ticket) {
            if (!p->active || p->cancel)
                return fail(PLAS_ERR_INVALID_ARG, "request %lld has finished or was cancelled", ticket);
            p->cancel = true;
            return PLAS_OK;
        }
    for (auto& ln : srv->lanes)
        if (ln->sl->job.ticket == ticket) {
            if (ln->done || ln->sl->cancel)
                return fail(PLAS_ERR_INVALID_ARG, "request %lld has finished or was cancelled", ticket);
            ln->sl->cancel = true;
            return PLAS_OK;
        }
    return fail(PLAS_ERR_INVALID_ARG, "request %lld is not queued or running", ticket);
}

extern "C" int plas_server_status(plas_server* srv, int* queued, int* active, size_t* mem_in_use) {
    if (!srv) return fail(PLAS_ERR_INVALID_ARG, "NULL server");
    if (queued) *queued = (int)srv->queue.size();
    if (active) *active = (int)(srv->running.size() + srv->lanes.size());
    if (mem_in_use) *mem_in_use = srv->in_use;
    return PLAS_OK;
}

extern "C" int plas_server_destroy(plas_server* srv) {
    if (!srv) return PLAS_OK;
    cudaStreamSynchronize(srv->st);
    for (auto& ln : srv->lanes) {
        cudaStreamSynchronize(ln->st);
        if (ln->sl->owns && ln->sl->mem) cudaFreeAsync(ln->sl->mem, ln->st);
        cudaStreamSynchronize(ln->st);
        if (ln->done) cudaEventDestroy(ln->done);
        ln->eng.reset();
        cudaStreamDestroy(ln->st);
        for (cudaStream_t o : ln->old_streams) cudaStreamDestroy(o);
    }
    srv->lanes.clear();
    for (auto& sl : srv->running)
        if (sl->owns && sl->mem) cudaFreeAsync(sl->mem, srv->st);
    for (auto& r : srv->retiring) cudaEventDestroy(r.ev);
    for (auto e : srv->events) cudaEventDestroy(e);
    srv->eng.reset();
    cudaStreamSynchronize(srv->st);
    delete srv;
    return PLAS_OK;
}
