// krylov.h -- device scalars and launchers of the FP64 Krylov recurrences (Algorithm 1).
#pragma once

#include <cuda_runtime.h>

#include "smg_internal.h"

namespace smg {

constexpr int kMaxReduceBlocks = 1216;  // CTAs of a reduction kernel on HBM-resident vectors (8 x 152 SMs)
constexpr int kReduceBlocks = 304;      // CTAs of a reduction kernel on L2-resident vectors (2 x 152 SMs)

// Scalars of Algorithm 1 kept on the device between kernels.
struct KrylovScalars {
    double rho;       // (s_k, r_k)
    double rho_prev;  // (s_{k-1}, r_{k-1})
    double sdr;       // (s_k, r_k - r_{k-1})
    double beta, pq, alpha;
    double rr;        // ||r_k||^2 (recurrence)
    double bb;        // ||b||^2
    double tt;        // ||b - A x||^2 (true residual)
    int restart;      // 1: next beta = 0 (first step, or continuing from a true residual)
    int status;       // 0 or an SMG_ERR_* code raised on the device
    int variant;      // SMG_PCG, SMG_FPCG, SMG_PSD
    int it;           // iterations done (the x/r update of each increments it)
    int maxit;        // the solve's iteration limit
    int pad;
    double tol2;      // tol^2: the device-side loop continues while rr > tol2 * bb
    double *hist;     // when set: hist[it] = sqrt(rr / bb) after every x/r update
};

struct DSum;

struct KrylovWork {
    KrylovScalars *sc = nullptr;   // device
    DSum *part = nullptr;          // device, kMaxReduceBlocks * 2 partial sums
    unsigned *counter = nullptr;   // device, 1 counter (reset by the last block)
    unsigned *bar = nullptr;       // device, grid-barrier count and generation, then an error word
    bool fused = false;            // the iteration tail as one cooperative kernel where it fits
};

int reduction_blocks(long long n);
cudaError_t kry_init_residual(Prec st_prec, int nx, int ny, int nz, const double *b, const double *x, double *r,
                              void *f0, KrylovWork &w, cudaStream_t st);
cudaError_t kry_true_residual(int nx, int ny, int nz, const double *b, const double *x, KrylovWork &w,
                              cudaStream_t st);
// One iteration after s = T r: dots + beta, p update, q = A p + alpha, x/r update + ||r||^2.
// With use_cond, the x/r update's last CTA also sets the conditional node `cond` of the CUDA
// graph that repeats the iteration: 1 (run another) while status == 0, rr > tol2 bb and
// it < maxit, else 0.
cudaError_t kry_iteration_tail(Prec st_prec, int nx, int ny, int nz, const void *s, double *x, double *r, double *p,
                               double *q, double *dr, void *f0, KrylovWork &w, cudaStream_t st,
                               cudaGraphConditionalHandle cond = 0, int use_cond = 0);

}  // namespace smg
