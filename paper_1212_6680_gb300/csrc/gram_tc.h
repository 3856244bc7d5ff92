// gram_tc.h -- FP64-accurate Gram products of tall-skinny blocks on the tcgen05 tensor cores
// (BF16 digit splitting with exact FP32 accumulation; see gram_tc.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace smg {

// Device workspace gram_tc needs for n rows (column maxima and per-CTA partials).
size_t gram_tc_workspace_bytes(long long n);

// G (device, k1 x k2 row-major) = U^T V, U: n x k1 (column j at U + j ldu), V: n x k2; 1 <= k1,
// k2 <= 64.  work: gram_tc_workspace_bytes(n) bytes of device memory.  Asynchronous on st.
// reuse_u_cmax: U and work are those of the previous call on this stream and U has not changed
// since, so U's column maxima left in work are reused instead of recomputed.
cudaError_t gram_tc(long long n, int k1, const double *U, long long ldu, int k2, const double *V, long long ldv,
                    double *G, void *work, int num_sms, cudaStream_t st, bool reuse_u_cmax = false);

// Reads and clears the flag a CTA sets when its bounded wait for its MMAs gave up (1), else 0.
cudaError_t gram_tc_status(int *err);

}  // namespace smg
