// plas_host.h -- host-side helpers shared by the C ABI translation units
// (internal to the CUDA library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/plas.h"
#include "plas_kernels.h"

namespace plas {

// ---- errors -------------------------------------------------------------------
int fail(int code, const char* fmt, ...);

// ---- host-side fault injection (plas_debug_inject; tests only) -----------------
// Every device allocation of the library goes through dev_alloc, which fails
// with cudaErrorMemoryAllocation when an injected failure is due.  A frozen
// read-back makes the progress check see no advance.  Neither touches the GPU.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
bool injected_stall();
// Wait limit of the persistent sweep's grid barriers: two seconds, or 0 while
// an injected zero limit is due (plas_debug_inject kind 3).
unsigned long long persist_wait_limit_ns();
// A planted overwrite of a checked run's first guard band is due
// (plas_debug_inject kind 4).
bool injected_guard_damage();
int check_launch(const char* what);
int num_sms();

#define PLAS_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::plas::fail(PLAS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,             \
                                cudaGetErrorString(e_), __FILE__, __LINE__);               \
    } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline bool channels_supported(int D) {
    return (D >= 1 && D <= 16) || D == 20 || D == 24 || D == 32 || D == 48 || D == 64;
}
int validate_schedule(const plas_schedule& s);
// Grid sizes the kernels index with 32-bit arithmetic: N = H * W <= 2^26 and
// max(H, W) * D <= 2^26 (a target pass's columns); 0 when they fit.
inline bool grid_fits(long long H, long long W, int D) {
    return H * W <= (1LL << 26) && (H > W ? H : W) * D <= (1LL << 26);
}

// ---- schedule geometry (Sec. 3.1) -----------------------------------------------
// phi_L = phi0 * shrink^L while >= phi_min; r = floor(phi); beta = min(max(r +
// 1, min_block), H, W); sigma = sigma_ratio * phi; taps k_j = (float) exp(-j^2 /
// (2 sigma^2)) in FP64, stored twice each (pairs for the packed FMA).
struct Geometry {
    std::vector<LevelDesc> lv;
    int max_steps = 0;  // largest padded tap-step count of any level and pass
    std::vector<float> table;  // padded tap pairs per level (norms filled on the device)
    size_t table_floats = 0;
};
double start_radius(const plas_schedule& s, int H, int W);
int count_levels(const plas_schedule& s, int H, int W);
Geometry build_geometry(const plas_schedule& s, int H, int W);

// ---- per-grid device workspace ----------------------------------------------------
struct Workspace {
    DevState* st;
    GridRef* ref;  // the grid's own descriptor (one-grid sweeps)
    float* G;
    float* T;
    float* H1;
    uint32_t* pi;
    LevelDesc* lv;
    float* table;
    double* macc;
    PersistCtl* pctl;  // control block of persistent sweeps over this grid
    long long* sat;  // box target: summed-area table, N x round_up(D, 2) int64 (else null)
    Guards guards;   // the guard band after each region (checked runs fill them)
};
size_t workspace_layout(int H, int W, int D, int nlev, size_t table_floats, Workspace* ws,
                        char* base, bool sat = false);
size_t sort_workspace_bytes(int H, int W, int D, const plas_schedule& s);

// ---- launch-shape tuning (plas_api.cu) ---------------------------------------------------
// What a sort of this shape on the current device uses: the installed entry
// for (D, H, W), else the entry with the same D and the nearest cell count,
// else the defaults.
constexpr int kDirectTuneMaxR = 32;  // the tuner times the direct FIR kernel up to this radius
constexpr int kDefaultSmallBelow = 12;
constexpr int kDefaultMediumBelow = 96;
constexpr int kDefaultAssignPerSm = 4;
struct Tuning {
    int small_below = kDefaultSmallBelow;    // small-radius path (one launch, or direct) below this radius
    int medium_below = kDefaultMediumBelow;  // else 64-row below this one, else 128-row
    int assign_per_sm = kDefaultAssignPerSm;
    int large_tma = 0;  // 1: the large tiling streams rows with tensor copies where a grid allows
                        // (measured slower than the ring everywhere; the tuner may pick it)
    int small_fused = 1;  // small radii run both passes in one launch where eligible
};
inline int fir_tiling(int r, const Tuning& t) {
    return r < t.small_below ? kFirSmallRadius : r < t.medium_below ? kFirMediumRadius : kFirLargeRadius;
}
// The FIR variant a level of radius r runs for D channels: the small-radius
// path takes the one-launch kernel up to kFusedMaxR and 16 channels (radii
// only shrink within a sort, so a plan made at radius r stays eligible).
inline int fir_variant(int r, int D, const Tuning& t) {
    const int v = fir_tiling(r, t);
    return v == kFirSmallRadius && t.small_fused && D <= kFusedMaxD && r <= kFusedMaxR ? fused_variant(r)
                                                                                      : v;
}
Tuning tuning_for(int H, int W, int D);
void install_tuning(int H, int W, int D, const Tuning* t);  // nullptr removes

// ---- pinned host staging for state polls (per host thread) ----------------------------
int poll_buffers(size_t bytes, void** host, cudaEvent_t* ev2);

}  // namespace plas
