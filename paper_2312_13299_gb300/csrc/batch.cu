// batch.cu -- plas_batch_sort: many independent grids with one schedule.
//
// Every grid keeps its own random streams (seeded per job) and its own
// schedule state, so each result equals plas_sort on that grid alone.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/plas.h"
#include "plas_kernels.h"

extern "C" {

size_t plas_batch_workspace_bytes(int n, const plas_job* jobs, int D) {
    if (n < 0 || (n > 0 && !jobs)) return 0;
    size_t need = 256;
    for (int i = 0; i < n; ++i) {
        if (jobs[i].H < 1 || jobs[i].W < 1) continue;
        need = std::max(need, plas_sort_workspace_bytes(jobs[i].H, jobs[i].W, D));
    }
    return need;
}

int plas_batch_sort(int n, const plas_job* jobs, int D, const float* weights,
                    const plas_schedule* sched, void* workspace, size_t ws_bytes, void* stream) {
    if (n < 0 || (n > 0 && !jobs)) {
        plas::set_last_error("bad job list");
        return PLAS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const plas_job& j = jobs[i];
        if (j.H < 0 || j.W < 0 || !j.x || !j.perm_out || (j.C > 0 && (!j.carried || !j.carried_out))) {
            plas::set_last_error("invalid job descriptor");
            return PLAS_ERR_INVALID_ARG;
        }
    }
    const size_t need = plas_batch_workspace_bytes(n, jobs, D);
    if (workspace && ws_bytes < need) {
        plas::set_last_error("batch workspace too small");
        return PLAS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const plas_job& j = jobs[i];
        plas_state st;
        memset(&st, 0, sizeof(st));
        const int rc = plas_sort(j.x, j.H, j.W, D, weights, j.carried, j.C, j.seed, sched, nullptr,
                                 &st, j.perm_out, j.carried_out, nullptr, workspace, ws_bytes,
                                 nullptr, stream);
        if (rc != PLAS_OK) return rc;
        if (j.state_out) *j.state_out = st;
    }
    return PLAS_OK;
}

}  // extern "C"
