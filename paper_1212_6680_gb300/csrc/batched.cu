// batched.cu -- krylov_solve_batched: many independent 7-point Laplacian systems on uneven
// grids solved together by Algorithm 1 of arXiv:1212.6680 (PCG eq. (1), flexible PCG eq. (2),
// PSD) with the SMG preconditioner.
//
// Per iteration, one CUDA graph:
//   1. the persistent V-cycle kernel (batched.cuh): every relaxation / transfer step of every
//      system's V-cycle in one launch, the z-levels of all systems aligned from the finest;
//   2. the FP64 Krylov kernels over all systems at once: vectors are concatenated, every CTA
//      works on one chunk of one system, per-system sums are finished by one thread per system
//      (compensated), and the per-system scalars (alpha, beta, norms) live on the device;
//   3. an 4-byte copy of the number of systems still iterating.
// A system whose recurrence residual meets the tolerance is masked out on the device (its
// tasks and chunks are skipped); when none is left, the true residuals are checked and any
// system that fails continues from its true residual with beta = 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/smg.h"
#include "batched.h"
#include "plane_relax.cuh"

namespace smg {

// ---- persistent-kernel dispatch over K -----------------------------------------------------------
#define SMG_DECL_BK(k)                                                                                 \
    cudaError_t launch_persistent_vcycle_k##k(Prec, int, int, size_t, const PersistArgs &, cudaStream_t, bool); \
    int set_persistent_smem_k##k(Prec, size_t);                                                        \
    int persistent_blocks_per_sm_k##k(Prec, int, size_t);
SMG_DECL_BK(1)
SMG_DECL_BK(2)
SMG_DECL_BK(3)
SMG_DECL_BK(4)

cudaError_t launch_persistent_vcycle(Prec storage, int K, int blocks, int threads, size_t smem, const PersistArgs &p,
                                     cudaStream_t st, bool cooperative) {
    switch (K) {
    case 1: return launch_persistent_vcycle_k1(storage, blocks, threads, smem, p, st, cooperative);
    case 2: return launch_persistent_vcycle_k2(storage, blocks, threads, smem, p, st, cooperative);
    case 3: return launch_persistent_vcycle_k3(storage, blocks, threads, smem, p, st, cooperative);
    case 4: return launch_persistent_vcycle_k4(storage, blocks, threads, smem, p, st, cooperative);
    }
    return cudaErrorInvalidValue;
}
int set_persistent_smem(Prec storage, int K, size_t smem) {
    switch (K) {
    case 1: return set_persistent_smem_k1(storage, smem);
    case 2: return set_persistent_smem_k2(storage, smem);
    case 3: return set_persistent_smem_k3(storage, smem);
    case 4: return set_persistent_smem_k4(storage, smem);
    }
    return static_cast<int>(cudaErrorInvalidValue);
}
int persistent_blocks_per_sm(Prec storage, int K, int threads, size_t smem) {
    switch (K) {
    case 1: return persistent_blocks_per_sm_k1(storage, threads, smem);
    case 2: return persistent_blocks_per_sm_k2(storage, threads, smem);
    case 3: return persistent_blocks_per_sm_k3(storage, threads, smem);
    case 4: return persistent_blocks_per_sm_k4(storage, threads, smem);
    }
    return 0;
}

namespace {

// ---- barrier self-test ------------------------------------------------------------------------------
__device__ __forceinline__ bool test_barrier(unsigned *count, unsigned *gen, int *err, long long limit,
                                             unsigned expected) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = *reinterpret_cast<volatile unsigned *>(gen);
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*reinterpret_cast<volatile unsigned *>(gen) == g) {
                if (*reinterpret_cast<volatile int *>(err) != 0) break;
                if (++spins > limit) {
                    atomicCAS(err, 0, SMG_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*reinterpret_cast<volatile int *>(err) == 0);
    }
    __syncthreads();
    return ok != 0;
}

__global__ void barrier_selftest_kernel(unsigned expected, long long limit, unsigned *count, unsigned *gen, int *err) {
    for (int s = 0; s < 4; ++s)
        if (!test_barrier(count, gen, err, limit, expected)) return;
}

// ---- batched FP64 Krylov kernels --------------------------------------------------------------------
constexpr int kChunk = 4096;
constexpr int kBThreads = 256;

struct BSys {
    int nx, ny, nz;
    long long off;        // offset of this system in the concatenated FP64 vectors
    long long f0_off;     // offset of its level-0 f in the storage array
    long long u0_off;     // offset of its level-0 u
    int c0, c1;           // its chunks [c0, c1)
};

struct BScal {
    double rho, rho_prev, beta, alpha, rr, bb;
    int restart, status, iters, pad;
};

// Per-solve controls, read from device memory so that a captured graph serves every solve.
struct BCtl {
    double tol2;  // tol^2
    int maxit;
    int variant;  // SMG_PCG, SMG_FPCG or SMG_PSD
};

struct BKrylov {
    const BSys *sys;
    const int *ch_sys;
    const long long *ch_start;  // global offset of the chunk
    const int *ch_len;
    double *r, *p, *q, *dr;
    const double *const *bptr;
    double *const *xptr;
    void *fstore, *ustore;      // storage arrays (level vectors of every system)
    double *part;               // 2 per chunk
    BScal *sc;
    int *active;
    int *nactive;
    const BCtl *ctl;            // tolerance, maxit, variant of the current solve (device)
    int nsys;
};

__device__ __forceinline__ double stencil_at(const double *__restrict__ v, long long i, int x, int y, int z, int nx,
                                             int ny, int nz) {
    const long long np = static_cast<long long>(nx) * ny;
    double nb = 0.0;
    if (x > 0) nb += v[i - 1];
    if (x < nx - 1) nb += v[i + 1];
    if (y > 0) nb += v[i - nx];
    if (y < ny - 1) nb += v[i + nx];
    if (z > 0) nb += v[i - np];
    if (z < nz - 1) nb += v[i + np];
    return 6.0 * v[i] - nb;
}

__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sh[2][kBThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int k = 0; k < kBThreads / 32; ++k) {
            a += sh[0][k];
            b += sh[1][k];
        }
    }
}

// r = b - A x, f0 = (S) r, partial ||r||^2, ||b||^2   (mode 1: only systems whose active flag is 2)
template <class S>
__global__ void __launch_bounds__(kBThreads) kb_init(BKrylov k, int only_flagged) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    const BSys sy = k.sys[s];
    double a0 = 0.0, a1 = 0.0;
    if (!only_flagged || k.active[s] == 2) {
        const long long g0 = k.ch_start[c];
        const int len = k.ch_len[c];
        const double *x = k.xptr[s];
        const double *b = k.bptr[s];
        S *f0 = static_cast<S *>(k.fstore) + sy.f0_off;
        const int npi = sy.nx * sy.ny;
        for (int t = threadIdx.x; t < len; t += kBThreads) {
            const long long gi = g0 + t;
            const int li = static_cast<int>(gi - sy.off);
            const int z = li / npi, ip = li - z * npi, y = ip / sy.nx, xx = ip - y * sy.nx;
            const double ri = b[li] - stencil_at(x, li, xx, y, z, sy.nx, sy.ny, sy.nz);
            k.r[gi] = ri;
            stv<S, double>(f0 + li, ri);
            a0 = fma(ri, ri, a0);
            a1 = fma(b[li], b[li], a1);
        }
    }
    block_sum2(a0, a1);
    if (threadIdx.x == 0) {
        k.part[2 * c] = a0;
        k.part[2 * c + 1] = a1;
    }
}

__device__ __forceinline__ void sum_chunks(const BKrylov &k, int s, double &v0, double &v1) {
    const BSys sy = k.sys[s];
    double s0 = 0.0, c0 = 0.0, s1 = 0.0, c1 = 0.0;
    for (int c = sy.c0; c < sy.c1; ++c) {
        const double a = k.part[2 * c], b = k.part[2 * c + 1];
        double t = s0 + a, bp = t - s0;
        c0 += (s0 - (t - bp)) + (a - bp);
        s0 = t;
        t = s1 + b;
        bp = t - s1;
        c1 += (s1 - (t - bp)) + (b - bp);
        s1 = t;
    }
    v0 = s0 + c0;
    v1 = s1 + c1;
}

// after kb_init: norms; mode 0 (start): every system active unless already converged;
// mode 1 (after a true-residual check): systems flagged 2 continue (restart), others stop.
__global__ void kb_fin_init(BKrylov k, int mode) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < k.nsys; s += blockDim.x) {
        double rr, bb;
        sum_chunks(k, s, rr, bb);
        BScal &q = k.sc[s];
        if (mode == 0) {
            q = BScal{0, 0, 0, 0, rr, bb, 1, 0, 0, 0};
            const double bref = bb > 0.0 ? bb : 1.0;
            k.active[s] = (rr > k.ctl->tol2 * bref) ? 1 : 0;
            if (!isfinite(rr) || !isfinite(bb)) {
                q.status = SMG_ERR_NAN;
                k.active[s] = 0;
            }
        } else {
            if (k.active[s] == 2) {
                q.rr = rr;
                q.restart = 1;
                k.active[s] = 1;
            }
        }
        if (k.active[s] == 1) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *k.nactive = cnt;
}

template <class S>
__global__ void __launch_bounds__(kBThreads) kb_dots(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    double a0 = 0.0, a1 = 0.0;
    if (k.active[s] == 1) {
        const BSys sy = k.sys[s];
        const long long g0 = k.ch_start[c];
        const int len = k.ch_len[c];
        const S *u0 = static_cast<const S *>(k.ustore) + sy.u0_off;
        const bool want = (k.ctl->variant == SMG_FPCG) && (k.sc[s].restart == 0);
        for (int t = threadIdx.x; t < len; t += kBThreads) {
            const long long gi = g0 + t;
            const double si = ldv<double>(u0 + (gi - sy.off));
            a0 = fma(si, k.r[gi], a0);
            if (want) a1 = fma(si, k.dr[gi], a1);
        }
    }
    block_sum2(a0, a1);
    if (threadIdx.x == 0) {
        k.part[2 * c] = a0;
        k.part[2 * c + 1] = a1;
    }
}

// smg_batched_apply: every system's r (FP64, caller memory) into its level-0 f in the storage
// precision, and every system active for the V-cycle that follows.
template <class S>
__global__ void __launch_bounds__(kBThreads) kb_apply_in(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    const BSys sy = k.sys[s];
    const long long g0 = k.ch_start[c];
    const int len = k.ch_len[c];
    const double *r = k.bptr[s];
    S *f0 = static_cast<S *>(k.fstore) + sy.f0_off;
    for (int t = threadIdx.x; t < len; t += kBThreads) {
        const int li = static_cast<int>(g0 + t - sy.off);
        stv<S, double>(f0 + li, r[li]);
    }
    if (threadIdx.x == 0 && c == sy.c0) k.active[s] = 1;
}

// smg_batched_apply: every system's level-0 u (the cycle's output, storage precision) widened
// exactly to FP64 into the caller's s.
template <class S>
__global__ void __launch_bounds__(kBThreads) kb_apply_out(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    const BSys sy = k.sys[s];
    const long long g0 = k.ch_start[c];
    const int len = k.ch_len[c];
    double *out = k.xptr[s];
    const S *u0 = static_cast<const S *>(k.ustore) + sy.u0_off;
    for (int t = threadIdx.x; t < len; t += kBThreads) {
        const int li = static_cast<int>(g0 + t - sy.off);
        out[li] = ldv<double>(u0 + li);
    }
}

__global__ void kb_fin_beta(BKrylov k) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k.nsys; s += gridDim.x * blockDim.x) {
        if (k.active[s] != 1) continue;
        double rho, sdr;
        sum_chunks(k, s, rho, sdr);
        BScal &q = k.sc[s];
        double beta = 0.0;
        if (q.restart == 0 && k.ctl->variant != SMG_PSD) {
            if (q.rho_prev == 0.0) q.status = SMG_ERR_BREAKDOWN;
            else beta = (k.ctl->variant == SMG_PCG) ? rho / q.rho_prev : sdr / q.rho_prev;
        }
        if (!isfinite(rho) || !isfinite(beta)) q.status = SMG_ERR_NAN;
        q.rho = rho;
        q.beta = beta;
    }
}

template <class S>
__global__ void __launch_bounds__(kBThreads) kb_upd_p(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    if (k.active[s] != 1) return;
    const BSys sy = k.sys[s];
    const long long g0 = k.ch_start[c];
    const int len = k.ch_len[c];
    const S *u0 = static_cast<const S *>(k.ustore) + sy.u0_off;
    const double beta = k.sc[s].beta;
    for (int t = threadIdx.x; t < len; t += kBThreads) {
        const long long gi = g0 + t;
        const double si = ldv<double>(u0 + (gi - sy.off));
        k.p[gi] = (beta == 0.0) ? si : fma(beta, k.p[gi], si);
    }
}

__global__ void __launch_bounds__(kBThreads) kb_spmv(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    double a0 = 0.0, a1 = 0.0;
    if (k.active[s] == 1) {
        const BSys sy = k.sys[s];
        const long long g0 = k.ch_start[c];
        const int len = k.ch_len[c];
        const double *ps = k.p + sy.off;
        const int npi = sy.nx * sy.ny;
        for (int t = threadIdx.x; t < len; t += kBThreads) {
            const long long gi = g0 + t;
            const int li = static_cast<int>(gi - sy.off);
            const int z = li / npi, ip = li - z * npi, y = ip / sy.nx, xx = ip - y * sy.nx;
            const double qi = stencil_at(ps, li, xx, y, z, sy.nx, sy.ny, sy.nz);
            k.q[gi] = qi;
            a0 = fma(ps[li], qi, a0);
        }
    }
    block_sum2(a0, a1);
    if (threadIdx.x == 0) {
        k.part[2 * c] = a0;
        k.part[2 * c + 1] = 0.0;
    }
}

__global__ void kb_fin_alpha(BKrylov k) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < k.nsys; s += gridDim.x * blockDim.x) {
        if (k.active[s] != 1) continue;
        double pq, unused;
        sum_chunks(k, s, pq, unused);
        BScal &q = k.sc[s];
        if (!(pq > 0.0)) {
            q.status = (pq == pq) ? SMG_ERR_BREAKDOWN : SMG_ERR_NAN;
            q.alpha = 0.0;
        } else {
            q.alpha = q.rho / pq;
        }
    }
}

template <class S>
__global__ void __launch_bounds__(kBThreads) kb_upd_xr(BKrylov k) {
    const int c = blockIdx.x;
    const int s = k.ch_sys[c];
    double a0 = 0.0, a1 = 0.0;
    if (k.active[s] == 1) {
        const BSys sy = k.sys[s];
        const long long g0 = k.ch_start[c];
        const int len = k.ch_len[c];
        const double alpha = k.sc[s].alpha;
        const bool want_dr = (k.ctl->variant == SMG_FPCG);
        double *x = k.xptr[s];
        S *f0 = static_cast<S *>(k.fstore) + sy.f0_off;
        for (int t = threadIdx.x; t < len; t += kBThreads) {
            const long long gi = g0 + t;
            const long long li = gi - sy.off;
            x[li] = fma(alpha, k.p[gi], x[li]);
            const double ro = k.r[gi];
            const double rn = fma(-alpha, k.q[gi], ro);
            if (want_dr) k.dr[gi] = rn - ro;
            k.r[gi] = rn;
            stv<S, double>(f0 + li, rn);
            a0 = fma(rn, rn, a0);
        }
    }
    block_sum2(a0, a1);
    if (threadIdx.x == 0) {
        k.part[2 * c] = a0;
        k.part[2 * c + 1] = 0.0;
    }
}

__global__ void kb_fin_rr(BKrylov k) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < k.nsys; s += blockDim.x) {
        if (k.active[s] == 1) {
            double rr, unused;
            sum_chunks(k, s, rr, unused);
            BScal &q = k.sc[s];
            q.rr = rr;
            q.rho_prev = q.rho;
            q.restart = 0;
            q.iters += 1;
            const double bref = q.bb > 0.0 ? q.bb : 1.0;
            if (!isfinite(rr)) q.status = SMG_ERR_NAN;
            if (rr <= k.ctl->tol2 * bref || q.status != 0 || q.iters >= k.ctl->maxit) k.active[s] = 0;
        }
        if (k.active[s] == 1) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *k.nactive = cnt;
}

// After the loop: true residual norms (kb_init computes r = b - A x), flag systems to restart.
__global__ void kb_fin_true(BKrylov k, double *relres, int *nflag) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < k.nsys; s += blockDim.x) {
        double tt, bb;
        sum_chunks(k, s, tt, bb);
        const double bref = bb > 0.0 ? bb : 1.0;
        relres[s] = sqrt(tt / bref);
        BScal &q = k.sc[s];
        if (q.status == 0 && tt > k.ctl->tol2 * bref && q.iters < k.ctl->maxit) {
            k.active[s] = 2;  // continue from the true residual
            atomicAdd(&cnt, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *nflag = cnt;
}

// ---- host side ------------------------------------------------------------------------------------
thread_local std::string g_berr;

#define BCHK(call)                                                                      \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_last_error(std::string("batched solver: ") + #call + ": " +       \
                           cudaGetErrorString(e_));                                     \
            return SMG_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

int chunk_K(int nx) { return (nx + 31) / 32; }

struct Tuned {
    int threads = 512;
    int order = 1;  // 1: tasks of a step in decreasing cost, 0: system order
    int K = 0;      // x-line rows per lane (the line tile: 32 K rows per warp)
    int bps = 1;    // persistent CTAs per SM
};
std::mutex g_tune_mutex;
std::map<std::vector<int>, Tuned> g_tune_cache;

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
};

}  // namespace

cudaError_t launch_barrier_selftest(int blocks, int extra, long long spin_limit, unsigned *count, unsigned *gen,
                                    int *err, cudaStream_t st) {
    barrier_selftest_kernel<<<blocks, 32, 0, st>>>(static_cast<unsigned>(blocks + extra), spin_limit, count, gen, err);
    return cudaGetLastError();
}

}  // namespace smg

using namespace smg;

namespace {

struct SysPlan {
    int nx, ny, nz;
    long long N;
    HostHierarchy H;
    PlaneLayout lay, lay_d;
    size_t zoff, poff;                 // offsets into the concatenated coefficient tables
    std::vector<long long> foff;       // per level, offset into the storage arrays
    double cycle_bytes;                // algorithmic bytes of one V-cycle of this system
};

// Estimated cost of relaxing one plane (for the longest-first ordering of a step's tasks).
double plane_cost(const SysPlan &s) { return static_cast<double>(s.nx) * s.ny; }

// Algorithmic traffic of one V-cycle (npre pre-sweeps, npost post-sweeps) of one system, in
// storage words: a relaxation of a colour reads f and writes u of its planes (and reads u in
// correction form, mode 2), and reads each opposite-colour plane once when it can be nonzero;
// residual + restriction and prolongation + correction move 2.5 words per fine point each.
double vcycle_words(const SysPlan &p, int npre, int npost) {
    const double np = static_cast<double>(p.nx) * p.ny;
    double w = 0.0;
    auto colour = [&](int nzl, int col, int mode) {
        const int nplanes = col == 0 ? (nzl + 1) / 2 : nzl / 2;
        const int nother = nzl - nplanes;
        return (nplanes * (2.0 + (mode == 2 ? 1.0 : 0.0)) + (mode >= 1 ? nother : 0)) * np;
    };
    for (int l = 0; l + 1 < p.H.L; ++l) {
        const int nzl = p.H.nz_l[l];
        for (int sw = 0; sw < npre; ++sw) w += colour(nzl, 0, sw == 0 ? 0 : 2) + colour(nzl, 1, sw == 0 ? 1 : 2);
        for (int sw = 0; sw < npost; ++sw) w += colour(nzl, 1, 2) + colour(nzl, 0, 2);
        w += 5.0 * nzl * np;
    }
    w += 2.0 * np;  // the coarsest plane: read f, write u
    return w;
}

}  // namespace

// Everything one set of grids needs, built once: hierarchies, level vectors, Krylov vectors,
// the task list of the persistent V-cycle, the tuned schedule and the per-iteration graph.
struct smg_batched_ctx {
    int nsys = 0, npre = 1, npost = 0, prec = SMG_FP32;
    Prec P = Prec::F32;
    int K = 1, Lmax = 1, nsm = 0, nch = 0;
    std::vector<SysPlan> sys;
    DevBuf buf;
    PersistArgs pa{};
    BKrylov kk{};
    BCtl *d_ctl = nullptr;
    int *d_flags = nullptr;            // [0] systems still iterating, [1] barrier error, [2] systems to restart
    double *d_relres = nullptr;
    BScal *d_sc = nullptr;
    double **d_bptr = nullptr, **d_xptr = nullptr;
    int *h_pinned = nullptr;           // pinned copy of d_flags[0..1]
    size_t smem = 0;
    Tuned tune;
    int blocks = 0;
    long long ntasks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // V-cycle start, V-cycle end, iteration end
    // profiling (smg_batched_profile_read)
    int profile = 0;
    long long prof_launches[2] = {0, 0};
    double prof_ms[2] = {0.0, 0.0}, prof_bytes[2] = {0.0, 0.0};
    long long kernel_launches = 0;
    int kernels_per_iter = 0;

    ~smg_batched_ctx() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (h_pinned) cudaFreeHost(h_pinned);
    }

    cudaError_t launch_vcycle(cudaStream_t st, int threads, int nblocks) {
        pa.expected_blocks = nblocks;
        return launch_persistent_vcycle(P, K, nblocks, threads, smem, pa, st, false);
    }
    cudaError_t init(cudaStream_t st, int mode) {
        switch (P) {
        case Prec::F64: kb_init<double><<<nch, kBThreads, 0, st>>>(kk, mode); break;
        case Prec::F32: kb_init<float><<<nch, kBThreads, 0, st>>>(kk, mode); break;
        case Prec::BF16: kb_init<__nv_bfloat16><<<nch, kBThreads, 0, st>>>(kk, mode); break;
        }
        kb_fin_init<<<1, 1024, 0, st>>>(kk, mode);
        kernel_launches += 2;
        return cudaGetLastError();
    }
    cudaError_t krylov_tail(cudaStream_t st) {
        switch (P) {
        case Prec::F64: kb_dots<double><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::F32: kb_dots<float><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::BF16: kb_dots<__nv_bfloat16><<<nch, kBThreads, 0, st>>>(kk); break;
        }
        kb_fin_beta<<<(nsys + 127) / 128, 128, 0, st>>>(kk);
        switch (P) {
        case Prec::F64: kb_upd_p<double><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::F32: kb_upd_p<float><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::BF16: kb_upd_p<__nv_bfloat16><<<nch, kBThreads, 0, st>>>(kk); break;
        }
        kb_spmv<<<nch, kBThreads, 0, st>>>(kk);
        kb_fin_alpha<<<(nsys + 127) / 128, 128, 0, st>>>(kk);
        switch (P) {
        case Prec::F64: kb_upd_xr<double><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::F32: kb_upd_xr<float><<<nch, kBThreads, 0, st>>>(kk); break;
        case Prec::BF16: kb_upd_xr<__nv_bfloat16><<<nch, kBThreads, 0, st>>>(kk); break;
        }
        kb_fin_rr<<<1, 1024, 0, st>>>(kk);
        return cudaGetLastError();
    }
};

namespace {

int check_dims(int nsys, const int *dims) {
    if (nsys < 1 || nsys > 4096) {
        set_last_error("nsys must be in [1, 4096]");
        return SMG_ERR_ARG;
    }
    if (!dims) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    for (int s = 0; s < nsys; ++s) {
        const int nx = dims[3 * s], ny = dims[3 * s + 1], nz = dims[3 * s + 2];
        if (nx < 1 || ny < 1 || nz < 1 || nx > 128 || ny > kMaxNy || nz > kMaxNz) {
            set_last_error("each system needs 1 <= nx <= 128, 1 <= ny <= 512, 1 <= nz <= 4096");
            return SMG_ERR_ARG;
        }
    }
    return SMG_OK;
}

int batched_build(smg_batched_ctx &c, const int *dims, cudaStream_t st) {
    const int nsys = c.nsys;
    const Prec P = c.P;
    const size_t sb = storage_bytes(P), cb = (P == Prec::F64) ? 8 : 4;
    constexpr size_t kBudget = 227 * 1024 - 3 * 1024;  // static shared memory of the two plane cycles (~2 KB)
    DevBuf &buf = c.buf;

    // ---- per-system hierarchies and layouts ----
    c.sys.resize(nsys);
    std::vector<SysPlan> &sys = c.sys;
    int K = 1, Lmax = 1;
    size_t ztot = 0, ptot = 0;
    long long stot = 0, vtot = 0;
    for (int s = 0; s < nsys; ++s) {
        SysPlan &p = sys[s];
        p.nx = dims[3 * s];
        p.ny = dims[3 * s + 1];
        p.nz = dims[3 * s + 2];
        p.N = static_cast<long long>(p.nx) * p.ny * p.nz;
        build_hierarchy(p.nx, p.ny, p.nz, p.H);
        K = std::max(K, chunk_K(p.nx));
        Lmax = std::max(Lmax, p.H.L);
        p.zoff = ztot;
        p.poff = ptot;
        ztot += p.H.zcoef.size();
        ptot += p.H.pcoef.size();
        p.foff.resize(p.H.L);
        for (int l = 0; l < p.H.L; ++l) {
            p.foff[l] = stot;
            stot += static_cast<long long>(p.nx) * p.ny * p.H.nz_l[l];
        }
        vtot += p.N;
        p.cycle_bytes = vcycle_words(p, c.npre, c.npost) * static_cast<double>(sb);
    }
    c.K = K;
    c.Lmax = Lmax;
    // all systems use the widest chunk K (narrower lines are padded with identity rows); the
    // layouts size their factor sets for that K
    for (auto &p : sys) {
        p.lay = plan_plane_layout(p.H, cb, kBudget, K);
        p.lay_d = plan_plane_layout(p.H, 8, kBudget, K);
    }

    double *d_zc64, *d_pc64;
    float *d_zc32, *d_pc32;
    BCHK(buf.alloc(&d_zc64, ztot));
    BCHK(buf.alloc(&d_pc64, ptot));
    BCHK(buf.alloc(&d_zc32, ztot));
    BCHK(buf.alloc(&d_pc32, ptot));
    {
        std::vector<double> z64(ztot), p64(ptot);
        for (auto &p : sys) {
            std::copy(p.H.zcoef.begin(), p.H.zcoef.end(), z64.begin() + p.zoff);
            std::copy(p.H.pcoef.begin(), p.H.pcoef.end(), p64.begin() + p.poff);
        }
        std::vector<float> z32(z64.begin(), z64.end()), p32(p64.begin(), p64.end());
        BCHK(cudaMemcpyAsync(d_zc64, z64.data(), ztot * 8, cudaMemcpyHostToDevice, st));
        BCHK(cudaMemcpyAsync(d_pc64, p64.data(), ptot * 8, cudaMemcpyHostToDevice, st));
        BCHK(cudaMemcpyAsync(d_zc32, z32.data(), ztot * 4, cudaMemcpyHostToDevice, st));
        BCHK(cudaMemcpyAsync(d_pc32, p32.data(), ptot * 4, cudaMemcpyHostToDevice, st));
        BCHK(cudaStreamSynchronize(st));
    }
    void *d_f = nullptr, *d_u = nullptr;
    {
        unsigned char *pf, *pu;
        BCHK(buf.alloc(&pf, static_cast<size_t>(stot) * sb));
        BCHK(buf.alloc(&pu, static_cast<size_t>(stot) * sb));
        BCHK(cudaMemsetAsync(pf, 0, static_cast<size_t>(stot) * sb, st));
        BCHK(cudaMemsetAsync(pu, 0, static_cast<size_t>(stot) * sb, st));
        d_f = pf;
        d_u = pu;
    }
    int dev = 0;
    BCHK(cudaGetDevice(&dev));
    BCHK(cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nsm = c.nsm;

    // ---- tasks, steps ----
    struct StepTasks {
        std::vector<BTask> t;
        std::vector<double> cost;
    };
    std::vector<PlaneRelaxArgs> relax;
    std::vector<int> relax_f64;  // 1: the entry computes in FP64
    std::vector<int> relax_sys, relax_layd;  // the entry's system; 1: it uses the FP64 layout
    std::vector<int> relax_lvl;              // the entry's z-level
    std::vector<BTransfer> xfer;
    std::map<std::vector<int>, int> relax_index;  // (s, l, colour, mode, f64) -> args index
    size_t smem_max = 0;
    long long ws_bytes = 0;
    auto relax_arg = [&](int s, int l, int colour, int mode, bool f64, int iters_) -> int {
        std::vector<int> key{s, l, colour, mode, f64 ? 1 : 0};
        auto it = relax_index.find(key);
        if (it != relax_index.end()) return it->second;
        SysPlan &p = sys[s];
        const PlaneLayout &lay = f64 ? p.lay_d : p.lay;
        PlaneRelaxArgs a;
        std::memset(&a, 0, sizeof(a));
        a.solo_from = kMaxPlaneLevels;
        a.nx = p.nx;
        a.ny = p.ny;
        a.nz = p.H.nz_l[l];
        a.colour = colour;
        a.mode = mode;
        a.iters = iters_;
        a.f = static_cast<unsigned char *>(d_f) + p.foff[l] * sb;
        a.u = static_cast<unsigned char *>(d_u) + p.foff[l] * sb;
        a.vstride = 0;
        a.zcoef = d_zc64 + p.zoff + static_cast<size_t>(p.H.plane_base[l]) * kCoefPerPlane;
        a.pcoef = d_pc64 + p.poff + static_cast<size_t>(p.H.plane_base[l]) * p.H.sum_ny * kCoefPerLine;
        a.zcoef32 = d_zc32 + p.zoff + static_cast<size_t>(p.H.plane_base[l]) * kCoefPerPlane;
        a.pcoef32 = d_pc32 + p.poff + static_cast<size_t>(p.H.plane_base[l]) * p.H.sum_ny * kCoefPerLine;
        a.P = p.H.P;
        a.sum_ny = p.H.sum_ny;
        for (int m = 0; m < p.H.P; ++m) {
            a.ny_m[m] = p.H.ny_m[m];
            a.line_base[m] = p.H.line_base[m];
            a.off_u[m] = lay.off_u[m];
            a.off_g[m] = lay.off_g[m];
        }
        a.smem_u_mask = lay.smem_u_mask;
        a.smem_g_mask = lay.smem_g_mask;
        a.R = 1;
        a.MF = lay.MF;
        a.off_fs = lay.off_fs;
        a.vec = 0;
        const size_t elem = f64 ? 8 : cb;
        smem_max = std::max(smem_max, lay.smem_bytes);
        ws_bytes = std::max<long long>(ws_bytes, lay.ws_per_plane * static_cast<long long>(elem));
        a.ws_per_plane = lay.ws_per_plane;  // elements; converted to a common byte stride below
        relax.push_back(a);
        relax_f64.push_back((f64 || P == Prec::F64) ? 1 : 0);
        relax_sys.push_back(s);
        relax_layd.push_back(f64 ? 1 : 0);
        relax_lvl.push_back(l);
        relax_index[key] = static_cast<int>(relax.size()) - 1;
        return static_cast<int>(relax.size()) - 1;
    };
    auto xfer_arg = [&](int s, int l) -> int {
        SysPlan &p = sys[s];
        BTransfer t;
        t.nx = p.nx;
        t.ny = p.ny;
        t.nzf = p.H.nz_l[l];
        t.f = static_cast<unsigned char *>(d_f) + p.foff[l] * sb;
        t.u = static_cast<unsigned char *>(d_u) + p.foff[l] * sb;
        t.fc = static_cast<unsigned char *>(d_f) + p.foff[l + 1] * sb;
        t.uc = static_cast<unsigned char *>(d_u) + p.foff[l + 1] * sb;
        t.zc64 = d_zc64 + p.zoff + static_cast<size_t>(p.H.plane_base[l]) * kCoefPerPlane;
        t.zc32 = d_zc32 + p.zoff + static_cast<size_t>(p.H.plane_base[l]) * kCoefPerPlane;
        xfer.push_back(t);
        return static_cast<int>(xfer.size()) - 1;
    };
    std::vector<StepTasks> steps;
    auto add_relax_step = [&](int l, int colour, int mode_first, int sweep, bool with_coarsest) {
        StepTasks st_;
        for (int s = 0; s < nsys; ++s) {
            SysPlan &p = sys[s];
            if (l < p.H.L - 1) {
                const int nzl = p.H.nz_l[l];
                const int nplanes = colour == 0 ? (nzl + 1) / 2 : nzl / 2;
                const int mode = sweep == 0 ? mode_first : 2;
                const bool f64c = (P == Prec::F64);
                const int ai = relax_arg(s, l, colour, mode, f64c, 1);
                for (int i = 0; i < nplanes; ++i) {
                    st_.t.push_back(BTask{TASK_RELAX, ai, i, s});
                    st_.cost.push_back(plane_cost(p));
                }
            } else if (with_coarsest && l == p.H.L - 1) {
                const int ai = relax_arg(s, l, 0, 0, true, 1);
                st_.t.push_back(BTask{TASK_RELAX_F64, ai, 0, s});
                st_.cost.push_back(8.0 * plane_cost(p));  // FP64 plane cycle
            }
        }
        steps.push_back(st_);
    };
    for (int l = 0; l < Lmax; ++l) {
        for (int sw = 0; sw < c.npre; ++sw) {
            add_relax_step(l, 0, 0, sw, sw == 0);
            add_relax_step(l, 1, 1, sw, false);
        }
        StepTasks sx;
        for (int s = 0; s < nsys; ++s) {
            SysPlan &p = sys[s];
            if (l < p.H.L - 1) {
                const int xi = xfer_arg(s, l);
                for (int j = 0; j < p.H.nz_l[l + 1]; ++j) {
                    sx.t.push_back(BTask{TASK_RESTRICT, xi, j, s});
                    sx.cost.push_back(0.1 * plane_cost(p));
                }
            }
        }
        if (!sx.t.empty()) steps.push_back(sx);
    }
    for (int l = Lmax - 2; l >= 0; --l) {
        StepTasks sp;
        for (int s = 0; s < nsys; ++s) {
            SysPlan &p = sys[s];
            if (l < p.H.L - 1) {
                const int xi = xfer_arg(s, l);
                for (int z = 0; z < p.H.nz_l[l]; ++z) {
                    sp.t.push_back(BTask{TASK_PROLONG, xi, z, s});
                    sp.cost.push_back(0.05 * plane_cost(p));
                }
            }
        }
        if (!sp.t.empty()) steps.push_back(sp);
        for (int sw = 0; sw < c.npost; ++sw) {
            add_relax_step(l, 1, 2, 1, false);
            add_relax_step(l, 0, 2, 1, false);
        }
    }
    // drop empty steps
    steps.erase(std::remove_if(steps.begin(), steps.end(), [](const StepTasks &x) { return x.t.empty(); }),
                steps.end());
    // ---- candidate line tiles: x-line rows per lane from the narrowest that holds every
    // system's lines (K) up to 4; each has its own layouts, shared memory and workspace stride ----
    struct KPlan {
        int K;
        std::vector<PlaneRelaxArgs> relax;
        size_t smem;
        long long ws_stride;  // bytes per persistent CTA
    };
    std::vector<KPlan> kplans;
    for (int kc = K; kc <= 4; ++kc) {
        KPlan kp;
        kp.K = kc;
        kp.relax = relax;
        // general layouts, and the shortened-step cycle's (every factor set on chip) where it fits
        std::vector<PlaneLayout> lay(nsys), layd(nsys), lean(nsys), leand(nsys);
        for (int s = 0; s < nsys; ++s) {
            lay[s] = plan_plane_layout(sys[s].H, cb, kBudget, kc);
            layd[s] = plan_plane_layout(sys[s].H, 8, kBudget, kc);
            lean[s] = plan_plane_layout(sys[s].H, cb, kBudget, kc, true);
            leand[s] = plan_plane_layout(sys[s].H, 8, kBudget, kc, true);
        }
        size_t sm = 0;
        long long wsb = 0;
        for (size_t i = 0; i < relax.size(); ++i) {
            const int si = relax_sys[i];
            const PlaneLayout &Lg = relax_layd[i] ? layd[si] : lay[si];
            const PlaneLayout &Ll = relax_layd[i] ? leand[si] : lean[si];
            const bool use_lean = lean_supported(kc) && relax[i].iters == 1 && Ll.MF == sys[si].H.P &&
                                  Ll.smem_bytes <= kBudget && lean_uniform_level(sys[si].H, relax_lvl[i]);
            const PlaneLayout &L = use_lean ? Ll : Lg;
            PlaneRelaxArgs &a = kp.relax[i];
            a.lean = use_lean ? 1 : 0;
            for (int m = 0; m < a.P; ++m) {
                a.off_u[m] = L.off_u[m];
                a.off_g[m] = L.off_g[m];
            }
            a.smem_u_mask = L.smem_u_mask;
            a.smem_g_mask = L.smem_g_mask;
            a.MF = L.MF;
            a.off_fs = L.off_fs;
            sm = std::max(sm, L.smem_bytes);
            wsb = std::max<long long>(wsb, L.ws_per_plane * static_cast<long long>(relax_layd[i] ? 8 : cb));
        }
        kp.ws_stride = (wsb + 255) / 256 * 256;
        for (size_t i = 0; i < relax.size(); ++i)
            kp.relax[i].ws_per_plane = kp.ws_stride / (relax_f64[i] ? 8 : static_cast<long long>(cb));
        kp.smem = std::max<size_t>(sm, 1024);
        if (set_persistent_smem(P, kc, kp.smem) != 0) {
            cudaGetLastError();
            continue;  // this tile's layout does not fit: not a candidate
        }
        kplans.push_back(kp);
    }
    if (kplans.empty()) {
        set_last_error("batched solver: shared-memory configuration failed");
        return SMG_ERR_CUDA;
    }

    // ---- device buffers for the persistent kernel and the Krylov kernels ----
    PlaneRelaxArgs *d_relax;
    BTransfer *d_xfer;
    BTask *d_tasks;
    int *d_step_begin, *d_active;
    unsigned *d_bar;
    unsigned char *d_ws;
    BCHK(buf.alloc(&d_relax, relax.size()));
    BCHK(buf.alloc(&d_xfer, xfer.size()));
    BCHK(buf.alloc(&d_active, nsys));
    BCHK(buf.alloc(&c.d_flags, 4));
    BCHK(buf.alloc(&d_bar, 2));
    BCHK(buf.alloc(&c.d_ctl, 1));
    BCHK(cudaMemsetAsync(d_bar, 0, 2 * sizeof(unsigned), st));
    BCHK(cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), st));
    {
        std::vector<int> ones(nsys, 1);  // every system active while the schedule is tuned
        BCHK(cudaMemcpyAsync(d_active, ones.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st));
        BCHK(cudaStreamSynchronize(st));
    }
    size_t ntasks = 0;
    for (auto &s_ : steps) ntasks += s_.t.size();
    c.ntasks = static_cast<long long>(ntasks);
    BCHK(buf.alloc(&d_tasks, ntasks));
    BCHK(buf.alloc(&d_step_begin, steps.size() + 1));
    auto upload_tasks = [&](int order) -> int {
        std::vector<BTask> all;
        std::vector<int> begin{0};
        for (auto &s_ : steps) {
            std::vector<int> idx(s_.t.size());
            std::iota(idx.begin(), idx.end(), 0);
            if (order == 1)
                std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s_.cost[a] > s_.cost[b]; });
            for (int i : idx) all.push_back(s_.t[i]);
            begin.push_back(static_cast<int>(all.size()));
        }
        BCHK(cudaMemcpyAsync(d_tasks, all.data(), all.size() * sizeof(BTask), cudaMemcpyHostToDevice, st));
        BCHK(cudaMemcpyAsync(d_step_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        BCHK(cudaStreamSynchronize(st));
        return SMG_OK;
    };
    // workspace: one slot per CTA of the largest persistent grid any candidate schedule uses
    size_t ws_total = 0;
    int max_blocks = 0;
    for (auto &kp : kplans)
        for (int threads : {256, 512}) {
            const int b = nsm * persistent_blocks_per_sm(P, kp.K, threads, kp.smem);
            max_blocks = std::max(max_blocks, b);
            ws_total = std::max(ws_total, static_cast<size_t>(std::max<long long>(kp.ws_stride, 256)) * std::max(b, 0));
        }
    if (max_blocks < 1) {
        set_last_error("batched solver: the persistent kernel does not fit on an SM");
        return SMG_ERR_CUDA;
    }
    BCHK(buf.alloc(&d_ws, ws_total));
    for (auto &kp : kplans)
        for (auto &a : kp.relax) a.gws = d_ws;
    // the persistent kernel reads the relaxation arguments of the line tile in use
    auto use_tile = [&](const KPlan &kp) -> int {
        c.K = kp.K;
        c.smem = kp.smem;
        BCHK(cudaMemcpyAsync(d_relax, kp.relax.data(), kp.relax.size() * sizeof(PlaneRelaxArgs), cudaMemcpyHostToDevice,
                             st));
        BCHK(cudaStreamSynchronize(st));
        return SMG_OK;
    };
    BCHK(cudaMemcpyAsync(d_xfer, xfer.data(), xfer.size() * sizeof(BTransfer), cudaMemcpyHostToDevice, st));

    // Krylov data
    std::vector<BSys> hsys(nsys);
    std::vector<int> ch_sys;
    std::vector<long long> ch_start;
    std::vector<int> ch_len;
    {
        long long off = 0;
        for (int s = 0; s < nsys; ++s) {
            BSys &q = hsys[s];
            q.nx = sys[s].nx;
            q.ny = sys[s].ny;
            q.nz = sys[s].nz;
            q.off = off;
            q.f0_off = sys[s].foff[0];
            q.u0_off = sys[s].foff[0];
            q.c0 = static_cast<int>(ch_sys.size());
            for (long long cc = 0; cc < sys[s].N; cc += kChunk) {
                ch_sys.push_back(s);
                ch_start.push_back(off + cc);
                ch_len.push_back(static_cast<int>(std::min<long long>(kChunk, sys[s].N - cc)));
            }
            q.c1 = static_cast<int>(ch_sys.size());
            off += sys[s].N;
        }
    }
    c.nch = static_cast<int>(ch_sys.size());
    const int nch = c.nch;
    BSys *d_sys;
    int *d_ch_sys, *d_ch_len;
    long long *d_ch_start;
    double *d_r, *d_p, *d_q, *d_dr, *d_part;
    BCHK(buf.alloc(&d_sys, nsys));
    BCHK(buf.alloc(&d_ch_sys, nch));
    BCHK(buf.alloc(&d_ch_len, nch));
    BCHK(buf.alloc(&d_ch_start, nch));
    BCHK(buf.alloc(&d_r, vtot));
    BCHK(buf.alloc(&d_p, vtot));
    BCHK(buf.alloc(&d_q, vtot));
    BCHK(buf.alloc(&d_dr, vtot));
    BCHK(buf.alloc(&d_part, 2 * static_cast<size_t>(nch)));
    BCHK(buf.alloc(&c.d_relres, nsys));
    BCHK(buf.alloc(&c.d_sc, nsys));
    BCHK(buf.alloc(&c.d_bptr, nsys));
    BCHK(buf.alloc(&c.d_xptr, nsys));
    BCHK(cudaMemcpyAsync(d_sys, hsys.data(), nsys * sizeof(BSys), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(d_ch_sys, ch_sys.data(), nch * sizeof(int), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(d_ch_len, ch_len.data(), nch * sizeof(int), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(d_ch_start, ch_start.data(), nch * sizeof(long long), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemsetAsync(d_dr, 0, vtot * sizeof(double), st));
    BCHK(cudaMemsetAsync(d_p, 0, vtot * sizeof(double), st));

    BKrylov &kk = c.kk;
    kk.sys = d_sys;
    kk.ch_sys = d_ch_sys;
    kk.ch_start = d_ch_start;
    kk.ch_len = d_ch_len;
    kk.r = d_r;
    kk.p = d_p;
    kk.q = d_q;
    kk.dr = d_dr;
    kk.bptr = c.d_bptr;
    kk.xptr = c.d_xptr;
    kk.fstore = d_f;
    kk.ustore = d_u;
    kk.part = d_part;
    kk.sc = c.d_sc;
    kk.active = d_active;
    kk.nactive = c.d_flags;
    kk.ctl = c.d_ctl;
    kk.nsys = nsys;

    BCHK(cudaMallocHost(&c.h_pinned, 4 * sizeof(int)));
    for (cudaEvent_t &e : c.ev) BCHK(cudaEventCreate(&e));

    PersistArgs &pa = c.pa;
    pa.relax = d_relax;
    pa.xfer = d_xfer;
    pa.tasks = d_tasks;
    pa.step_begin = d_step_begin;
    pa.nsteps = static_cast<int>(steps.size());
    pa.active = d_active;
    pa.bar_count = d_bar;
    pa.bar_gen = d_bar + 1;
    pa.err = c.d_flags + 1;
    pa.spin_limit = 10000000;  // about a second of polling

    // ---- autotuned schedule: line tile (rows per lane), threads per CTA, persistent CTAs per SM
    // and task order within a step ----
    std::vector<int> key{nsys, c.prec, c.npre, c.npost};
    for (int s = 0; s < 3 * nsys; ++s) key.push_back(dims[s]);
    bool tuned = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c.tune = it->second;
            tuned = true;
        }
    }
    if (!tuned) {
        // the cost of a V-cycle does not depend on the values: time each candidate on the
        // zero-initialised level vectors with every system active
        float best = 1e30f;
        for (const auto &kp : kplans) {
            if (use_tile(kp) != SMG_OK) return SMG_ERR_CUDA;
            for (int threads : {256, 512}) {
                const int bmax = persistent_blocks_per_sm(P, kp.K, threads, kp.smem);
                for (int bps = 1; bps <= bmax; ++bps) {
                    const int nb = nsm * bps;
                    for (int order : {0, 1}) {
                        if (upload_tasks(order) != SMG_OK) return SMG_ERR_CUDA;
                        BCHK(c.launch_vcycle(st, threads, nb));  // warm-up
                        BCHK(cudaEventRecord(c.ev[0], st));
                        BCHK(c.launch_vcycle(st, threads, nb));
                        BCHK(cudaEventRecord(c.ev[1], st));
                        BCHK(cudaEventSynchronize(c.ev[1]));
                        c.kernel_launches += 2;
                        float ms = 0.0f;
                        BCHK(cudaEventElapsedTime(&ms, c.ev[0], c.ev[1]));
                        int herr = 0;
                        BCHK(cudaMemcpy(&herr, pa.err, sizeof(int), cudaMemcpyDeviceToHost));
                        if (herr != 0) {
                            set_last_error("batched solver: a V-cycle barrier wait timed out");
                            return herr;
                        }
                        if (ms < best) {
                            best = ms;
                            c.tune.K = kp.K;
                            c.tune.threads = threads;
                            c.tune.bps = bps;
                            c.tune.order = order;
                        }
                    }
                }
            }
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = c.tune;
    }
    const KPlan *chosen = &kplans[0];
    for (const auto &kp : kplans)
        if (kp.K == c.tune.K) chosen = &kp;
    if (use_tile(*chosen) != SMG_OK) return SMG_ERR_CUDA;
    if (upload_tasks(c.tune.order) != SMG_OK) return SMG_ERR_CUDA;
    const int bps = std::max(1, std::min(c.tune.bps, persistent_blocks_per_sm(P, c.K, c.tune.threads, c.smem)));
    c.blocks = std::min(max_blocks, nsm * bps);

    // ---- capture one iteration into a CUDA graph ----
    cudaStream_t cs = nullptr;
    BCHK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sguard{cs};
    BCHK(cudaStreamSynchronize(st));
    {
        BCHK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        // the events become event-record nodes, so the V-cycle and the Krylov part of every
        // replay can be timed
        cudaError_t e = cudaEventRecordWithFlags(c.ev[0], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = c.launch_vcycle(cs, c.tune.threads, c.blocks);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(c.ev[1], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = c.krylov_tail(cs);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(c.ev[2], cs, cudaEventRecordExternal);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.h_pinned, c.d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &c.graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            set_last_error(std::string("batched solver: graph capture: ") +
                           cudaGetErrorString(e != cudaSuccess ? e : e2));
            return SMG_ERR_CUDA;
        }
        BCHK(cudaGraphInstantiate(&c.exec, c.graph, 0));
    }
    c.kernels_per_iter = 1 + 8;  // persistent V-cycle + the Krylov tail
    return SMG_OK;
}

int batched_solve(smg_batched_ctx &c, int variant, const double *const *b, double *const *x, double tol, int maxit,
                  int *iters, double *relres, cudaStream_t st) {
    const int nsys = c.nsys;
    for (int s = 0; s < nsys; ++s) iters[s] = 0;
    const BCtl ctl{tol * tol, maxit, variant};
    BCHK(cudaMemcpyAsync(c.d_ctl, &ctl, sizeof(BCtl), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(c.d_bptr, b, nsys * sizeof(double *), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(c.d_xptr, x, nsys * sizeof(double *), cudaMemcpyHostToDevice, st));
    BCHK(c.init(st, 0));
    BCHK(cudaMemcpyAsync(c.h_pinned, c.d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    BCHK(cudaStreamSynchronize(st));
    int nact = c.h_pinned[0];
    for (int round = 0; round < 8; ++round) {
        for (int it = 0; it < maxit && nact > 0; ++it) {
            BCHK(cudaGraphLaunch(c.exec, st));
            BCHK(cudaStreamSynchronize(st));
            c.kernel_launches += c.kernels_per_iter;
            nact = c.h_pinned[0];
            if (c.h_pinned[1] != 0) {
                set_last_error("batched solver: a V-cycle barrier wait timed out");
                return c.h_pinned[1];
            }
            if (c.profile) {
                float m0 = 0.0f, m1 = 0.0f;
                if (cudaEventElapsedTime(&m0, c.ev[0], c.ev[1]) == cudaSuccess &&
                    cudaEventElapsedTime(&m1, c.ev[1], c.ev[2]) == cudaSuccess) {
                    c.prof_launches[0] += 1;
                    c.prof_ms[0] += m0;
                    c.prof_launches[1] += 1;
                    c.prof_ms[1] += m1;
                }
            }
        }
        // true residuals; systems that fail continue from them
        switch (c.P) {
        case Prec::F64: kb_init<double><<<c.nch, kBThreads, 0, st>>>(c.kk, 0); break;
        case Prec::F32: kb_init<float><<<c.nch, kBThreads, 0, st>>>(c.kk, 0); break;
        case Prec::BF16: kb_init<__nv_bfloat16><<<c.nch, kBThreads, 0, st>>>(c.kk, 0); break;
        }
        kb_fin_true<<<1, 1024, 0, st>>>(c.kk, c.d_relres, c.d_flags + 2);
        c.kernel_launches += 2;
        BCHK(cudaMemcpyAsync(c.h_pinned + 2, c.d_flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        BCHK(cudaStreamSynchronize(st));
        if (c.h_pinned[2] == 0) break;
        kb_fin_init<<<1, 1024, 0, st>>>(c.kk, 1);
        c.kernel_launches += 1;
        BCHK(cudaMemcpyAsync(c.h_pinned, c.d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        BCHK(cudaStreamSynchronize(st));
        nact = c.h_pinned[0];
    }
    std::vector<BScal> hs(nsys);
    std::vector<double> rel(nsys);
    BCHK(cudaMemcpy(hs.data(), c.d_sc, nsys * sizeof(BScal), cudaMemcpyDeviceToHost));
    BCHK(cudaMemcpy(rel.data(), c.d_relres, nsys * sizeof(double), cudaMemcpyDeviceToHost));
    int result = SMG_OK;
    for (int s = 0; s < nsys; ++s) {
        iters[s] = hs[s].iters;
        if (relres) relres[s] = rel[s];
        if (c.profile) c.prof_bytes[0] += hs[s].iters * c.sys[s].cycle_bytes;
        if (hs[s].status != 0 && result == SMG_OK) result = hs[s].status;
        if (result == SMG_OK && !(rel[s] <= tol)) result = SMG_ERR_NOCONV;
    }
    if (result == SMG_ERR_NOCONV) set_last_error("batched solver: a system did not converge within maxit");
    else if (result != SMG_OK) set_last_error("batched solver: breakdown or NaN in a system");
    return result;
}

}  // namespace

extern "C" int smg_batched_setup(int nsys, const int *dims, int npre, int npost, int prec, smg_batched_handle *out,
                                 void *stream) {
    if (!out) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    *out = nullptr;
    int rc = check_dims(nsys, dims);
    if (rc != SMG_OK) return rc;
    if (npre < 1 || npost < 0 || npre > 8 || npost > 8) {
        set_last_error("1 <= npre <= 8 and 0 <= npost <= 8 required");
        return SMG_ERR_ARG;
    }
    if (prec != SMG_FP32) {
        set_last_error("the batched solver runs the FP32 cycle (SMG_FP32) only");
        return SMG_ERR_ARG;
    }
    auto *c = new smg_batched_ctx();
    c->nsys = nsys;
    c->npre = npre;
    c->npost = npost;
    c->prec = prec;
    c->P = static_cast<Prec>(prec);
    rc = batched_build(*c, dims, static_cast<cudaStream_t>(stream));
    if (rc != SMG_OK) {
        const std::string msg = smg_last_error();
        delete c;
        set_last_error(msg);
        return rc;
    }
    *out = c;
    return SMG_OK;
}

extern "C" int smg_batched_solve(smg_batched_handle h, int variant, const double *const *b, double *const *x,
                                 double tol, int maxit, int *iters, double *relres, void *stream) {
    if (!h || !b || !x || !iters) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    if (variant != SMG_PCG && variant != SMG_FPCG && variant != SMG_PSD) {
        set_last_error("variant must be SMG_PCG, SMG_FPCG or SMG_PSD");
        return SMG_ERR_ARG;
    }
    if (!(tol > 0.0) || maxit < 0) {
        set_last_error("tol > 0 and maxit >= 0 required");
        return SMG_ERR_ARG;
    }
    for (int s = 0; s < h->nsys; ++s) {
        if (!b[s] || !x[s]) {
            set_last_error("null vector pointer");
            return SMG_ERR_ARG;
        }
    }
    return batched_solve(*h, variant, b, x, tol, maxit, iters, relres, static_cast<cudaStream_t>(stream));
}

extern "C" int smg_batched_apply(smg_batched_handle h, const double *const *r, double *const *out, void *stream) {
    if (!h || !r || !out) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    for (int s = 0; s < h->nsys; ++s) {
        if (!r[s] || !out[s]) {
            set_last_error("null vector pointer");
            return SMG_ERR_ARG;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    smg_batched_ctx &c = *h;
    BCHK(cudaMemcpyAsync(c.d_bptr, r, c.nsys * sizeof(double *), cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(c.d_xptr, out, c.nsys * sizeof(double *), cudaMemcpyHostToDevice, st));
    switch (c.P) {
    case Prec::F64: kb_apply_in<double><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    case Prec::F32: kb_apply_in<float><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    case Prec::BF16: kb_apply_in<__nv_bfloat16><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    }
    BCHK(cudaGetLastError());
    BCHK(c.launch_vcycle(st, c.tune.threads, c.blocks));
    switch (c.P) {
    case Prec::F64: kb_apply_out<double><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    case Prec::F32: kb_apply_out<float><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    case Prec::BF16: kb_apply_out<__nv_bfloat16><<<c.nch, kBThreads, 0, st>>>(c.kk); break;
    }
    BCHK(cudaGetLastError());
    c.kernel_launches += 3;
    int herr = 0;
    BCHK(cudaMemcpyAsync(&herr, c.pa.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCHK(cudaStreamSynchronize(st));
    if (herr != 0) {
        set_last_error("batched V-cycle: a grid-barrier wait timed out");
        return herr;
    }
    return SMG_OK;
}

extern "C" int smg_batched_destroy(smg_batched_handle h) {
    if (h) {
        cudaDeviceSynchronize();
        delete h;
    }
    return SMG_OK;
}

extern "C" int smg_batched_info(smg_batched_handle h, int *threads, int *order, int *blocks, long long *tasks,
                                long long *launches, int *rows_per_lane) {
    if (!h || !threads || !order || !blocks || !tasks || !launches || !rows_per_lane) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    *threads = h->tune.threads;
    *order = h->tune.order;
    *rows_per_lane = h->K;
    *blocks = h->blocks;
    *tasks = h->ntasks;
    *launches = h->kernel_launches;
    return SMG_OK;
}

extern "C" int smg_batched_set_profile(smg_batched_handle h, int on) {
    if (!h || on < 0 || on > 1) {
        set_last_error("a handle and on in {0, 1} required");
        return SMG_ERR_ARG;
    }
    h->profile = on;
    return SMG_OK;
}

extern "C" int smg_batched_profile_read(smg_batched_handle h, int which, long long *launches, double *ms,
                                        double *bytes) {
    if (!h || which < 0 || which > 1 || !launches || !ms || !bytes) {
        set_last_error("bad arguments");
        return SMG_ERR_ARG;
    }
    *launches = h->prof_launches[which];
    *ms = h->prof_ms[which];
    *bytes = h->prof_bytes[which];
    h->prof_launches[which] = 0;
    h->prof_ms[which] = 0.0;
    h->prof_bytes[which] = 0.0;
    return SMG_OK;
}

extern "C" int krylov_solve_batched(int nsys, const int *dims, int npre, int npost, int prec, const double *const *b,
                                    double *const *x, double tol, int maxit, int *iters, void *stream) {
    if (!b || !x || !iters || !dims) {
        set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    if (!(tol > 0.0) || maxit < 0) {
        set_last_error("npre >= 1, npost >= 0, tol > 0, maxit >= 0 required");
        return SMG_ERR_ARG;
    }
    if (nsys >= 1 && nsys <= 4096)
        for (int s = 0; s < nsys; ++s) iters[s] = 0;
    smg_batched_handle h = nullptr;
    int rc = smg_batched_setup(nsys, dims, npre, npost, prec, &h, stream);
    if (rc != SMG_OK) return rc;
    rc = smg_batched_solve(h, SMG_FPCG, b, x, tol, maxit, iters, nullptr, stream);
    const std::string msg = rc != SMG_OK ? std::string(smg_last_error()) : std::string();
    smg_batched_destroy(h);
    if (rc != SMG_OK) set_last_error(msg);
    return rc;
}

extern "C" int smg_barrier_selftest(int extra_blocks, double limit_seconds, int *status, void *stream) {
    if (!status || extra_blocks < 0 || !(limit_seconds > 0.0) || limit_seconds > 10.0) {
        set_last_error("status must be non-null, extra_blocks >= 0, 0 < limit_seconds <= 10");
        return SMG_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 4 * sizeof(unsigned));
    if (e != cudaSuccess) {
        set_last_error(std::string("smg_barrier_selftest: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), st);
    // one poll takes at least the 100 ns sleep: the limit is a lower bound on the wait
    const long long spins = static_cast<long long>(limit_seconds * 1e7);
    e = launch_barrier_selftest(4, extra_blocks, spins, d, d + 1, reinterpret_cast<int *>(d + 2), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, d + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_last_error(std::string("smg_barrier_selftest: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    return SMG_OK;
}
