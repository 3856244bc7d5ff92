// batched.cuh -- the persistent multi-system V-cycle kernel.
//
// All the V-cycle steps of all systems run in one launch: CTAs walk a device-resident task
// list step by step (a step = one colour of plane relaxation, one restriction or one
// prolongation per system and z-level, the levels of different systems aligned from the
// finest), with a grid-wide barrier between steps.  The barrier's wait is bounded: after
// `spin_limit` polls it records SMG_ERR_TIMEOUT and every CTA returns, so a barrier that can
// never complete (a CTA that is not resident) ends the kernel with an error status instead of
// hanging.
#pragma once

#include "../../include/smg.h"
#include "batched.h"
#include "grid_sync.cuh"
#include "plane_lean.cuh"
#include "plane_relax.cuh"
#include "transfer.cuh"

namespace smg {

template <class S, int K>
__global__ void __launch_bounds__(512, 1) persistent_vcycle_kernel(const __grid_constant__ PersistArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using CL = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
    for (int s = 0; s < p.nsteps; ++s) {
        for (int t = p.step_begin[s] + static_cast<int>(blockIdx.x); t < p.step_begin[s + 1];
             t += static_cast<int>(gridDim.x)) {
            const BTask tk = p.tasks[t];
            if (!p.active[tk.sys]) continue;
            if (tk.type == TASK_RELAX) {
                const PlaneRelaxArgs &a = p.relax[tk.arg];
                if (a.lean) plane_lean_task<S, CL, K, false>(a, tk.idx, 0, blockIdx.x, 0, smem_raw);
                else plane_task<S, CL, K, false>(a, tk.idx, 0, blockIdx.x, 0, smem_raw);
            } else if (tk.type == TASK_RELAX_F64) {
                const PlaneRelaxArgs &a = p.relax[tk.arg];
                if (a.lean) plane_lean_task<S, double, K, false>(a, tk.idx, 0, blockIdx.x, 0, smem_raw);
                else plane_task<S, double, K, false>(a, tk.idx, 0, blockIdx.x, 0, smem_raw);
            } else if (tk.type == TASK_RESTRICT) {
                const BTransfer &x = p.xfer[tk.arg];
                const CL *zc = coef_table<CL>(x.zc64, x.zc32);
                for (int ip = threadIdx.x; ip < x.nx * x.ny; ip += blockDim.x)
                    restrict_point<S, CL>(x.nx, x.ny, x.nzf, static_cast<const S *>(x.f), static_cast<const S *>(x.u),
                                          static_cast<S *>(x.fc), zc, tk.idx, ip);
            } else {
                const BTransfer &x = p.xfer[tk.arg];
                const CL *zc = coef_table<CL>(x.zc64, x.zc32);
                for (int ip = threadIdx.x; ip < x.nx * x.ny; ip += blockDim.x)
                    prolong_point<S, CL>(x.nx, x.ny, x.nzf, static_cast<S *>(x.u), static_cast<const S *>(x.uc), zc,
                                         tk.idx, ip);
            }
            __syncthreads();  // the next task reuses the shared memory
        }
        if (!grid_barrier(p.bar_count, p.bar_gen, p.err, p.spin_limit, static_cast<unsigned>(p.expected_blocks)))
            return;
    }
}

}  // namespace smg
