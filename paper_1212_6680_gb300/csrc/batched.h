// batched.h -- many independent systems on uneven grids solved together: one persistent
// V-cycle kernel for all systems, batched FP64 Krylov kernels, one CUDA graph per iteration.
#pragma once

#include <cuda_runtime.h>

#include "smg_internal.h"

namespace smg {

// One unit of work of the persistent V-cycle kernel.
enum : int { TASK_RELAX = 0, TASK_RELAX_F64 = 1, TASK_RESTRICT = 2, TASK_PROLONG = 3 };

struct BTask {
    int type;  // TASK_*
    int arg;   // index into the relax-args or transfer-args table
    int idx;   // plane index within the colour (relax), coarse plane (restrict), fine plane (prolong)
    int sys;   // system (its active flag gates the task)
};

// Arguments of the grid transfers of one (system, level).
struct BTransfer {
    int nx, ny, nzf;
    const void *f;     // level f (storage type)
    void *u;           // level u
    void *fc;          // next level's f (restriction output)
    const void *uc;    // next level's u (prolongation input)
    const double *zc64;
    const float *zc32;
};

struct PersistArgs {
    const PlaneRelaxArgs *relax;
    const BTransfer *xfer;
    const BTask *tasks;
    const int *step_begin;  // [nsteps + 1]
    int nsteps;
    const int *active;      // per system: 1 while it is being iterated
    unsigned *bar_count;    // grid barrier state
    unsigned *bar_gen;
    int *err;               // SMG_ERR_TIMEOUT when a barrier wait gives up
    long long spin_limit;   // iterations of the barrier wait before giving up
    int expected_blocks;    // CTAs the barrier waits for (gridDim.x in normal use)
};

// Launch the persistent V-cycle over all steps (storage precision, x-line chunk K <= 4).
cudaError_t launch_persistent_vcycle(Prec storage, int K, int blocks, int threads, size_t smem,
                                     const PersistArgs &p, cudaStream_t st, bool cooperative);
int set_persistent_smem(Prec storage, int K, size_t smem);
int persistent_blocks_per_sm(Prec storage, int K, int threads, size_t smem);

// Barrier self-test: a persistent kernel of `blocks` CTAs whose barrier waits for
// blocks + extra CTAs; writes the error status (0 or SMG_ERR_TIMEOUT) to *err.
cudaError_t launch_barrier_selftest(int blocks, int extra, long long spin_limit, unsigned *count, unsigned *gen,
                                    int *err, cudaStream_t st);

}  // namespace smg
