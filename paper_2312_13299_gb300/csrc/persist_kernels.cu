// persist_kernels.cu -- the persistent sweep: one cooperative launch that
// advances every grid of a sweep by k iterations of the PLAS sort (Sec. 3.1
// of Morgenstern et al., arXiv 2312.13299).
//
// Each iteration has three phases, separated by a grid-wide barrier: the
// target pass along y (its work items also write the grouping table), the
// pass along x, and the assignment with its exact residual sum (the last
// work item of a grid to finish runs that grid's schedule step, as in the
// one-launch-per-class kernels).  The work items of a phase are the same
// (grid, tile) pairs a per-class launch would run as CTAs, from the same CTA
// maps; resident CTAs take them round robin and run the same bodies
// (sweep_bodies.cuh), so the results are bit-identical.  Data written in one
// phase is read in the next through ordinary loads after the barrier's
// gpu-scope fences (no read-only-path loads of the target or the grouping
// table).
//
// The barrier's wait is bounded: after limit_ns without the last arrival, the
// CTA records PLAS_ERR_TIMEOUT in the launch's control block and in every
// grid's status word; every CTA that sees the flag stops, so the launch ends
// and the host reads the error.  No wait is unbounded and nothing traps.
#include <algorithm>

#include "sweep_bodies.cuh"

namespace plas {

namespace {

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Sense-counting grid barrier over gridDim.x co-resident CTAs.  false: the
// launch gave up (a wait ran past limit_ns here or in another CTA).
__device__ bool grid_barrier(PersistCtl* c, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &c->gen;
        volatile int* vstat = &c->status;
        int ok = 1;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&c->arrive, 1u) + 1u == gridDim.x) {
            atomicExch(&c->arrive, 0u);
            __threadfence();
            atomicAdd(&c->gen, 1u);
        } else {
            const unsigned long long t0 = now_ns();
            while (*vgen == g) {
                if (*vstat) {
                    ok = 0;
                    break;
                }
                if (now_ns() - t0 > limit_ns) {
                    atomicCAS(&c->status, 0, -4);  // PLAS_ERR_TIMEOUT
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && *vstat == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ CtaRef item_of(const CtaMap* __restrict__ map, int w, int n) {
    if (map == nullptr) return CtaRef{0, w, n};
    const CtaMap m = map[w];
    return CtaRef{m.grid, m.local, m.count};
}

// The phase bodies as separate functions, so that each gets its own register
// allocation (one call per work item).
__device__ __noinline__ void fir_item(int pass, const GridRef* __restrict__ grids, CtaRef cr, int D,
                                      int gs, int ts, ulonglong2* ring) {
    fir_ring_body<FirMedium>(pass, grids, cr, D, gs, ts, ring);
}
template <int D>
__device__ __noinline__ void assign_item(const GridRef* __restrict__ grids, CtaRef cr, double tol) {
    assign_body<D, false>(grids, cr, tol);
}

template <int D>
__global__ void __launch_bounds__(kAssignThreads, 2) persist_sweep_kernel(
    const GridRef* __restrict__ grids, int ngrids, const CtaMap* __restrict__ map_y, int n_y,
    const CtaMap* __restrict__ map_x, int n_x, const CtaMap* __restrict__ map_a, int n_a, int k,
    double tol, PersistCtl* ctl, unsigned long long limit_ns) {
    static_assert(FirMedium::THREADS == kAssignThreads, "one CTA shape for every phase");
    extern __shared__ __align__(16) ulonglong2 ring[];  // FirMedium::RING x 32 lanes x 4 columns
    constexpr int GS = (D + 1 + 3) & ~3, TS = (D + 3) & ~3;
    bool ok = true;
    for (int it = 0; it < k && ok; ++it) {
        for (int w = blockIdx.x; w < n_y; w += gridDim.x)
            fir_item(0, grids, item_of(map_y, w, n_y), D, GS, TS, ring);
        ok = grid_barrier(ctl, limit_ns);
        if (!ok) break;
        for (int w = blockIdx.x; w < n_x; w += gridDim.x)
            fir_item(1, grids, item_of(map_x, w, n_x), D, GS, TS, ring);
        ok = grid_barrier(ctl, limit_ns);
        if (!ok) break;
        for (int w = blockIdx.x; w < n_a; w += gridDim.x)
            assign_item<D>(grids, item_of(map_a, w, n_a), tol);
        ok = grid_barrier(ctl, limit_ns);
    }
    if (!ok && threadIdx.x == 0)
        for (int g = blockIdx.x; g < ngrids; g += gridDim.x) atomicCAS(&grids[g].st->status, 0, -4);
}

template <int D>
int launch_persist_t(const GridRef* grids, int ngrids, const CtaMap* my, int ny, const CtaMap* mx,
                     int nx, const CtaMap* ma, int na, int k, double tol, PersistCtl* ctl,
                     unsigned long long limit_ns, cudaStream_t s) {
    const size_t smem = sizeof(ulonglong2) * FirMedium::RING * 32;
    static int per_sm[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -3;
    if (per_sm[dev] == 0) {
        if (cudaFuncSetAttribute(persist_sweep_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -3;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persist_sweep_kernel<D>, kAssignThreads,
                                                          smem) != cudaSuccess ||
            n < 1)
            return -3;
        per_sm[dev] = n;
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
    const int work = std::max({ny, nx, na, 1});
    const int blocks = std::min(work, per_sm[dev] * nsm);
    if (cudaMemsetAsync(ctl, 0, sizeof(PersistCtl), s) != cudaSuccess) return -3;
    void* args[] = {(void*)&grids, (void*)&ngrids, (void*)&my, (void*)&ny, (void*)&mx, (void*)&nx,
                    (void*)&ma, (void*)&na, (void*)&k, (void*)&tol, (void*)&ctl, (void*)&limit_ns};
    if (cudaLaunchCooperativeKernel((const void*)persist_sweep_kernel<D>, dim3(blocks),
                                    dim3(kAssignThreads), args, smem, s) != cudaSuccess)
        return -3;
    return 0;
}

}  // namespace

int launch_persist(const GridRef* grids, int ngrids, const CtaMap* map_y, int n_y,
                   const CtaMap* map_x, int n_x, const CtaMap* map_a, int n_a, int D, int k,
                   double tol, PersistCtl* ctl, unsigned long long limit_ns, cudaStream_t s) {
    switch (D) {
#define PLAS_CASE(d) \
    case d:          \
        return launch_persist_t<d>(grids, ngrids, map_y, n_y, map_x, n_x, map_a, n_a, k, tol, ctl, limit_ns, s);
        PLAS_CASE(1) PLAS_CASE(2) PLAS_CASE(3) PLAS_CASE(4) PLAS_CASE(5) PLAS_CASE(6)
        PLAS_CASE(7) PLAS_CASE(8) PLAS_CASE(9) PLAS_CASE(10) PLAS_CASE(11) PLAS_CASE(12)
        PLAS_CASE(13) PLAS_CASE(14) PLAS_CASE(15) PLAS_CASE(16) PLAS_CASE(20) PLAS_CASE(24)
        PLAS_CASE(32) PLAS_CASE(48) PLAS_CASE(64)
#undef PLAS_CASE
        default: return -1;
    }
}

}  // namespace plas
