// lobpcg.h -- block LOBPCG preconditioned by SMG (section "Preconditioning of LOBPCG with SMG"
// of arXiv:1212.6680; the method itself is Knyazev's locally optimal block preconditioned
// conjugate gradient, which the paper cites and runs through BLOPEX).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

namespace smg {

struct LobpcgOps {
    long long n = 0;
    // out = A u for nb column-major vectors (column stride n)
    std::function<int(int nb, const double *u, double *out, cudaStream_t st)> apply_A;
    // S = T R for nb vectors (one batched V-cycle)
    std::function<int(int nb, const double *r, double *s, cudaStream_t st)> apply_T;
};

struct LobpcgWork {
    long long n = 0;
    int m = 0;
    double *S = nullptr, *AS = nullptr;   // n x 3m each: [X | W | P]
    double *T1 = nullptr, *T2 = nullptr;  // n x 3m temporaries
    double *part = nullptr;               // Gram partial sums
    long long part_tiles = 0;             // capacity of part in 16 x 16 tiles
    int num_sms = 0;                      // SMs of the device (sizes the Gram grids)
    double *gram = nullptr;               // reduced Gram matrices
    double *coef = nullptr;               // small coefficient matrices (k x k)
    double *h_buf = nullptr;              // pinned host buffer
    void *tc_work = nullptr;              // workspace of the tensor-core Gram products
    int gram_tc_min = 16;                 // products with k1, k2 >= this (and <= 64) run on the
                                          // tensor cores (gram_tc.cu); 0 = never
};

int lobpcg_run(const LobpcgOps &ops, LobpcgWork &w, int m, double *X, double *lambda, double tol, int maxit,
               int *iters, cudaStream_t st, std::string &msg);
void lobpcg_free(LobpcgWork &w);

// Dense FP64 helpers (host), exposed for the unit tests of the Rayleigh-Ritz step.
// Symmetric eigen-decomposition by cyclic Jacobi: A (k x k, row-major, symmetric) ->
// eigenvalues ascending in w, eigenvectors as columns of V (row-major k x k).
void jacobi_eigh(int k, const double *A, double *w, double *V);
// Cholesky A = L L^T (row-major, lower L); returns false if A is not positive definite.
bool cholesky(int k, const double *A, double *L);

}  // namespace smg
