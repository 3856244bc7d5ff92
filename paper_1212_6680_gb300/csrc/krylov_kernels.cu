// krylov_kernels.cu -- FP64 kernels of Algorithm 1 (section "PSD and PCG methods" of
// arXiv:1212.6680): s_k = T r_k, p_k = s_k + beta_k p_{k-1}, alpha_k = (s_k, r_k)/(p_k, A p_k),
// x_{k+1} = x_k + alpha_k p_k, r_{k+1} = r_k - alpha_k A p_k, with beta_k from eq. (1)
// (standard PCG), eq. (2) (flexible PCG, extra vector r_k - r_{k-1}) or 0 (PSD).
//
// The scalars live on the device (KrylovScalars); the last CTA of each reduction kernel
// combines the per-CTA partial sums and computes the scalar the next kernel needs, so one
// iteration runs without the host.  Inner products: each thread accumulates its products
// with FMA, then partials are combined with error-free TwoSum (compensated summation).
// The preconditioned residual s is read straight from the V-cycle's level-0 storage
// (FP64, FP32 or BF16): widening it to FP64 is exact, so no FP64 copy of s is made.
#include <cuda_bf16.h>

#include "grid_sync.cuh"
#include "krylov.h"
#include "plane_relax.cuh"

namespace smg {

struct DSum {
    double s, c;
};

__device__ __forceinline__ void two_sum_acc(DSum &a, double b) {
    const double t = a.s + b;
    const double bp = t - a.s;
    const double err = (a.s - (t - bp)) + (b - bp);
    a.s = t;
    a.c += err;
}
__device__ __forceinline__ DSum dsum_combine(DSum a, const DSum &b) {
    two_sum_acc(a, b.s);
    a.c += b.c;
    return a;
}
__device__ __forceinline__ DSum shfl_down_dsum(const DSum &v, int o) {
    return DSum{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
}

// Inner products: every thread accumulates its (about 2N / (threads in the grid)) products with
// FMA, the block adds the thread partials pairwise (warp shuffles, then one warp over the warp
// sums), and the last block to finish combines the block partials with error-free TwoSum
// (compensated summation).  FP64 work per element stays at one FMA, which matters on GB300
// where an FP64 operation costs as much SM time as dozens of FP32 ones.
template <int NV>
__device__ __forceinline__ void block_reduce_plain(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = (lane < nw) ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

// Write this block's partials; the last block to finish sums all of them (compensated) into
// tot[].  Returns true in every thread of the last block.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], DSum *part, unsigned *counter, double (&tot)[NV]) {
    __shared__ bool last;
    __shared__ double res[NV];
    block_reduce_plain<NV>(v);
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) part[static_cast<size_t>(blockIdx.x) * NV + k] = DSum{v[k], 0.0};
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int k = 0; k < NV; ++k) {
            DSum w{0.0, 0.0};
            for (unsigned b = lane; b < gridDim.x; b += 32) {
                const volatile DSum *vp = &part[static_cast<size_t>(b) * NV + k];
                two_sum_acc(w, vp->s);
            }
            for (int o = 16; o > 0; o >>= 1) w = dsum_combine(w, shfl_down_dsum(w, o));
            if (lane == 0) res[k] = w.s + w.c;
        }
        if (lane == 0) *counter = 0u;
    }
    __syncthreads();
    for (int k = 0; k < NV; ++k) tot[k] = res[k];
    return true;
}

__device__ __forceinline__ double stencil7(const double *__restrict__ u, long long i, int x, int y, int z, int nx,
                                           int ny, int nz, long long np) {
    double nb = 0.0;
    if (x > 0) nb += u[i - 1];
    if (x < nx - 1) nb += u[i + 1];
    if (y > 0) nb += u[i - nx];
    if (y < ny - 1) nb += u[i + nx];
    if (z > 0) nb += u[i - np];
    if (z < nz - 1) nb += u[i + np];
    return 6.0 * u[i] - nb;
}

// After the x/r update (last CTA, one thread): rr = ||r_new||^2, the iteration count, the residual
// history and, inside the CUDA graph that repeats the iteration, its loop condition.
__device__ __forceinline__ void finish_update(KrylovScalars *sc, double rr, cudaGraphConditionalHandle cond,
                                              int use_cond) {
    sc->rr = rr;
    sc->rho_prev = sc->rho;
    sc->restart = 0;
    if (!isfinite(rr)) sc->status = -6;
    const int it = sc->it + 1;
    sc->it = it;
    const double bb = sc->bb > 0.0 ? sc->bb : 1.0;
    if (sc->hist != nullptr) sc->hist[it] = sqrt(rr / bb);
    if (use_cond) {
        const bool go = sc->status == 0 && !(rr <= sc->tol2 * bb) && it < sc->maxit;
        cudaGraphSetConditional(cond, go ? 1u : 0u);
    }
}

// r = b - A x ; f0 = (S) r ; rr = ||r||^2 ; bb = ||b||^2 ; restart = 1.
template <class S>
__global__ void k_init_residual(int nx, int ny, int nz, const double *__restrict__ b, const double *__restrict__ x,
                                double *__restrict__ r, S *__restrict__ f0, KrylovScalars *sc, DSum *part,
                                unsigned *counter) {
    const long long np = static_cast<long long>(nx) * ny;
    double a0 = 0.0, a1 = 0.0;
    const int npi = nx * ny, n32 = npi * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        const int zz = i / npi, ip = i - zz * npi, yy = ip / nx, xx = ip - yy * nx;
        const double bi = b[i];
        const double ri = bi - stencil7(x, i, xx, yy, zz, nx, ny, nz, np);
        r[i] = ri;
        if (f0 != nullptr) stv<S, double>(f0 + i, ri);
        a0 = fma(ri, ri, a0);
        a1 = fma(bi, bi, a1);
    }
    double v[2] = {a0, a1};
    double tot[2];
    if (grid_reduce<2>(v, part, counter, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->bb = tot[1];
        sc->restart = 1;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) sc->status = -6;
    }
}

// tt = ||b - A x||^2 (true residual).
__global__ void k_true_residual(int nx, int ny, int nz, const double *__restrict__ b, const double *__restrict__ x,
                                KrylovScalars *sc, DSum *part, unsigned *counter) {
    const long long np = static_cast<long long>(nx) * ny;
    double a0 = 0.0;
    const int npi = nx * ny, n32 = npi * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        const int zz = i / npi, ip = i - zz * npi, yy = ip / nx, xx = ip - yy * nx;
        const double ri = b[i] - stencil7(x, i, xx, yy, zz, nx, ny, nz, np);
        a0 = fma(ri, ri, a0);
    }
    double v[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) sc->tt = tot[0];
}

// rho = (s, r), sdr = (s, r_k - r_{k-1}); beta by eq. (1), eq. (2) or 0.
template <class S>
__global__ void k_dots_beta(long long n, const S *__restrict__ s, const double *__restrict__ r,
                            const double *__restrict__ dr, KrylovScalars *sc, DSum *part, unsigned *counter) {
    pdl_trigger();
    pdl_wait();
    const int variant = sc->variant;
    const bool need_sdr = (variant == 1) && (sc->restart == 0);
    double a0 = 0.0, a1 = 0.0;
    const int n32 = static_cast<int>(n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        const double si = ldv<double>(s + i);
        a0 = fma(si, r[i], a0);
        if (need_sdr) a1 = fma(si, dr[i], a1);
    }
    double v[2] = {a0, a1};
    double tot[2];
    if (grid_reduce<2>(v, part, counter, tot) && threadIdx.x == 0) {
        const double rho = tot[0];
        double beta = 0.0;
        if (sc->restart == 0 && variant != 2) {
            if (sc->rho_prev == 0.0) {
                sc->status = -4;
            } else {
                beta = (variant == 0) ? rho / sc->rho_prev : tot[1] / sc->rho_prev;
            }
        }
        if (!isfinite(rho) || !isfinite(beta)) sc->status = -6;
        sc->rho = rho;
        sc->sdr = tot[1];
        sc->beta = beta;
    }
}

// p = s + beta p
template <class S>
__global__ void k_update_p(long long n, const S *__restrict__ s, double *__restrict__ p, const KrylovScalars *sc) {
    pdl_trigger();
    pdl_wait();
    const double beta = sc->beta;
    const int n32 = static_cast<int>(n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        const double si = ldv<double>(s + i);
        p[i] = (beta == 0.0) ? si : fma(beta, p[i], si);
    }
}

// q = A p ; pq = (p, q) ; alpha = rho / pq
__global__ void k_spmv_alpha(int nx, int ny, int nz, const double *__restrict__ p, double *__restrict__ q,
                             KrylovScalars *sc, DSum *part, unsigned *counter) {
    pdl_trigger();
    pdl_wait();
    const long long np = static_cast<long long>(nx) * ny;
    double a0 = 0.0;
    const int npi = nx * ny, n32 = npi * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        const int zz = i / npi, ip = i - zz * npi, yy = ip / nx, xx = ip - yy * nx;
        const double qi = stencil7(p, i, xx, yy, zz, nx, ny, nz, np);
        q[i] = qi;
        a0 = fma(p[i], qi, a0);
    }
    double v[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        sc->pq = pq;
        if (!(pq > 0.0)) {
            sc->status = (pq == pq) ? -4 : -6;
            sc->alpha = 0.0;
        } else {
            sc->alpha = sc->rho / pq;
        }
    }
}

// x += alpha p ; r_new = r - alpha q ; dr = r_new - r ; r = r_new ; f0 = (S) r_new ; rr = ||r_new||^2
template <class S>
__global__ void k_update_xr(long long n, double *__restrict__ x, const double *__restrict__ p, double *__restrict__ r,
                            const double *__restrict__ q, double *__restrict__ dr, S *__restrict__ f0,
                            KrylovScalars *sc, DSum *part, unsigned *counter, cudaGraphConditionalHandle cond,
                            int use_cond) {
    pdl_trigger();
    pdl_wait();
    const double alpha = sc->alpha;
    const bool want_dr = (sc->variant == 1);
    double a0 = 0.0;
    const int n32 = static_cast<int>(n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n32; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ro = r[i];
        const double rn = fma(-alpha, q[i], ro);
        if (want_dr) dr[i] = rn - ro;
        r[i] = rn;
        if (f0 != nullptr) stv<S, double>(f0 + i, rn);
        a0 = fma(rn, rn, a0);
    }
    double v[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) finish_update(sc, tot[0], cond, use_cond);
}

// ---- the same four kernels on 4-element chunks ---------------------------------------------------
// Used when nx % 4 == 0 and every vector is 16-byte aligned: each thread moves four consecutive
// elements of a vector with 16-byte loads and stores (the element values, the operations on them
// and the order of the six neighbour terms of A p are those of the scalar kernels; only the
// assignment of elements to threads, and so the partial sums' grouping, differs).
__device__ __forceinline__ void ld4(double (&v)[4], const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
template <class S> __device__ __forceinline__ void lds4(double (&v)[4], const S *p);
template <> __device__ __forceinline__ void lds4<double>(double (&v)[4], const double *p) { ld4(v, p); }
template <> __device__ __forceinline__ void lds4<float>(double (&v)[4], const float *p) {
    const float4 a = reinterpret_cast<const float4 *>(p)[0];
    v[0] = widen_f32(a.x); v[1] = widen_f32(a.y); v[2] = widen_f32(a.z); v[3] = widen_f32(a.w);
}
template <> __device__ __forceinline__ void lds4<__nv_bfloat16>(double (&v)[4], const __nv_bfloat16 *p) {
    const uint2 a = reinterpret_cast<const uint2 *>(p)[0];
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&a.x), hi = *reinterpret_cast<const __nv_bfloat162 *>(&a.y);
    v[0] = widen_f32(__low2float(lo)); v[1] = widen_f32(__high2float(lo));
    v[2] = widen_f32(__low2float(hi)); v[3] = widen_f32(__high2float(hi));
}
template <class S> __device__ __forceinline__ void sts4(S *p, const double (&v)[4]);
template <> __device__ __forceinline__ void sts4<double>(double *p, const double (&v)[4]) { st4(p, v); }
template <> __device__ __forceinline__ void sts4<float>(float *p, const double (&v)[4]) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(narrow_f64(v[0]), narrow_f64(v[1]), narrow_f64(v[2]), narrow_f64(v[3]));
}
template <> __device__ __forceinline__ void sts4<__nv_bfloat16>(__nv_bfloat16 *p, const double (&v)[4]) {
    __nv_bfloat162 lo, hi;
    lo.x = __float2bfloat16_rn(narrow_f64(v[0])); lo.y = __float2bfloat16_rn(narrow_f64(v[1]));
    hi.x = __float2bfloat16_rn(narrow_f64(v[2])); hi.y = __float2bfloat16_rn(narrow_f64(v[3]));
    uint2 a;
    a.x = *reinterpret_cast<unsigned *>(&lo);
    a.y = *reinterpret_cast<unsigned *>(&hi);
    reinterpret_cast<uint2 *>(p)[0] = a;
}

template <class S>
__global__ void k_dots_beta4(int nc, const S *__restrict__ s, const double *__restrict__ r,
                             const double *__restrict__ dr, KrylovScalars *sc, DSum *part, unsigned *counter) {
    pdl_trigger();
    pdl_wait();
    const int variant = sc->variant;
    const bool need_sdr = (variant == 1) && (sc->restart == 0);
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 2
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        double sv[4], rv[4];
        lds4<S>(sv, s + 4 * c);
        ld4(rv, r + 4 * c);
#pragma unroll
        for (int k = 0; k < 4; ++k) a0 = fma(sv[k], rv[k], a0);
        if (need_sdr) {
            double dv[4];
            ld4(dv, dr + 4 * c);
#pragma unroll
            for (int k = 0; k < 4; ++k) a1 = fma(sv[k], dv[k], a1);
        }
    }
    double v[2] = {a0, a1};
    double tot[2];
    if (grid_reduce<2>(v, part, counter, tot) && threadIdx.x == 0) {
        const double rho = tot[0];
        double beta = 0.0;
        if (sc->restart == 0 && variant != 2) {
            if (sc->rho_prev == 0.0) {
                sc->status = -4;
            } else {
                beta = (variant == 0) ? rho / sc->rho_prev : tot[1] / sc->rho_prev;
            }
        }
        if (!isfinite(rho) || !isfinite(beta)) sc->status = -6;
        sc->rho = rho;
        sc->sdr = tot[1];
        sc->beta = beta;
    }
}

template <class S>
__global__ void k_update_p4(int nc, const S *__restrict__ s, double *__restrict__ p, const KrylovScalars *sc) {
    pdl_trigger();
    pdl_wait();
    const double beta = sc->beta;
#pragma unroll 2
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        double sv[4], pv[4];
        lds4<S>(sv, s + 4 * c);
        if (beta == 0.0) {
            st4(p + 4 * c, sv);
        } else {
            ld4(pv, p + 4 * c);
#pragma unroll
            for (int k = 0; k < 4; ++k) pv[k] = fma(beta, pv[k], sv[k]);
            st4(p + 4 * c, pv);
        }
    }
}

// q = A p on four consecutive points of an x-row (nx % 4 == 0), the neighbour terms summed in the
// order of stencil7.
__global__ void k_spmv_alpha4(int nx, int ny, int nz, const double *__restrict__ p, double *__restrict__ q,
                              KrylovScalars *sc, DSum *part, unsigned *counter) {
    pdl_trigger();
    pdl_wait();
    const int nq = nx >> 2, npi = nx * ny, nc = (npi >> 2) * nz;
    double a0 = 0.0;
#pragma unroll 2
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int row = c / nq, xq = c - row * nq;
        const int zz = row / ny, yy = row - zz * ny, xx = 4 * xq;
        const int i = 4 * c;
        double pc[4], nb[4] = {0.0, 0.0, 0.0, 0.0};
        ld4(pc, p + i);
        const double pl = (xx > 0) ? p[i - 1] : 0.0, pr = (xx + 4 < nx) ? p[i + 4] : 0.0;
        // x-1, x+1
        if (xx > 0) nb[0] += pl;
        nb[1] += pc[0];
        nb[2] += pc[1];
        nb[3] += pc[2];
        nb[0] += pc[1];
        nb[1] += pc[2];
        nb[2] += pc[3];
        if (xx + 4 < nx) nb[3] += pr;
        double t[4];
        if (yy > 0) {
            ld4(t, p + i - nx);
#pragma unroll
            for (int k = 0; k < 4; ++k) nb[k] += t[k];
        }
        if (yy < ny - 1) {
            ld4(t, p + i + nx);
#pragma unroll
            for (int k = 0; k < 4; ++k) nb[k] += t[k];
        }
        if (zz > 0) {
            ld4(t, p + i - npi);
#pragma unroll
            for (int k = 0; k < 4; ++k) nb[k] += t[k];
        }
        if (zz < nz - 1) {
            ld4(t, p + i + npi);
#pragma unroll
            for (int k = 0; k < 4; ++k) nb[k] += t[k];
        }
        double qv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qv[k] = 6.0 * pc[k] - nb[k];
            a0 = fma(pc[k], qv[k], a0);
        }
        st4(q + i, qv);
    }
    double v[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        sc->pq = pq;
        if (!(pq > 0.0)) {
            sc->status = (pq == pq) ? -4 : -6;
            sc->alpha = 0.0;
        } else {
            sc->alpha = sc->rho / pq;
        }
    }
}

template <class S>
__global__ void k_update_xr4(int nc, double *__restrict__ x, const double *__restrict__ p, double *__restrict__ r,
                             const double *__restrict__ q, double *__restrict__ dr, S *__restrict__ f0,
                             KrylovScalars *sc, DSum *part, unsigned *counter, cudaGraphConditionalHandle cond,
                             int use_cond) {
    pdl_trigger();
    pdl_wait();
    const double alpha = sc->alpha;
    const bool want_dr = (sc->variant == 1);
    double a0 = 0.0;
#pragma unroll 2
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int i = 4 * c;
        double xv[4], pv[4], ro[4], qv[4], rn[4];
        ld4(xv, x + i);
        ld4(pv, p + i);
        ld4(ro, r + i);
        ld4(qv, q + i);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            xv[k] = fma(alpha, pv[k], xv[k]);
            rn[k] = fma(-alpha, qv[k], ro[k]);
            a0 = fma(rn[k], rn[k], a0);
        }
        st4(x + i, xv);
        st4(r + i, rn);
        if (want_dr) {
            double dv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) dv[k] = rn[k] - ro[k];
            st4(dr + i, dv);
        }
        if (f0 != nullptr) sts4<S>(f0 + i, rn);
    }
    double v[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) finish_update(sc, tot[0], cond, use_cond);
}

// ---- the four kernels above as one cooperative kernel ---------------------------------------------
// The iteration tail with three grid-wide barriers in place of three kernel boundaries: dots and
// beta | p update | q = A p and alpha | x, r update.  Same grid, same 4-element chunks per thread
// and the same last-CTA reductions as the separate kernels, so every value (partial sums
// included) is bit-identical to theirs.  Neighbour values of p are written by other CTAs in the
// p phase, so the stencil phase reads p through L2 (ld.global.cg).
__device__ __forceinline__ void ld4cg(double (&v)[4], const double *p) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <class S>
__global__ void __launch_bounds__(256) k_tail_fused(int nx, int ny, int nz, const S *__restrict__ s, double *x,
                                                    double *r, double *p, double *q, double *dr, S *f0,
                                                    KrylovScalars *sc, DSum *part, unsigned *counter, unsigned *bar,
                                                    long long spin_limit, cudaGraphConditionalHandle cond,
                                                    int use_cond) {
    const int nq = nx >> 2, npi = nx * ny, nc = (npi >> 2) * nz;
    const int stride = gridDim.x * blockDim.x, c0 = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned *bcount = bar, *bgen = bar + 1;
    int *berr = reinterpret_cast<int *>(bar + 2);
    const unsigned nblk = gridDim.x;
    // A barrier wait that gave up ends this launch and stops the solve: the first CTA to see it
    // records SMG_ERR_TIMEOUT and ends the graph's loop (no x/r update completes then, so nothing
    // else sets the loop condition in this launch).
    auto give_up = [&]() {
        if (threadIdx.x == 0 && atomicCAS(bar + 3, 0u, 1u) == 0u) {
            sc->status = SMG_ERR_TIMEOUT;
            if (use_cond) cudaGraphSetConditional(cond, 0u);
        }
    };
    if (*reinterpret_cast<volatile int *>(berr) != 0) {  // an earlier launch of this solve gave up
        give_up();
        return;
    }
    // ---- rho = (s, r), sdr = (s, r - r_prev); beta ----
    {
        const int variant = sc->variant;
        const bool need_sdr = (variant == 1) && (sc->restart == 0);
        double a0 = 0.0, a1 = 0.0;
#pragma unroll 2
        for (int c = c0; c < nc; c += stride) {
            double sv[4], rv[4];
            lds4<S>(sv, s + 4 * c);
            ld4(rv, r + 4 * c);
#pragma unroll
            for (int k = 0; k < 4; ++k) a0 = fma(sv[k], rv[k], a0);
            if (need_sdr) {
                double dv[4];
                ld4(dv, dr + 4 * c);
#pragma unroll
                for (int k = 0; k < 4; ++k) a1 = fma(sv[k], dv[k], a1);
            }
        }
        double v[2] = {a0, a1};
        double tot[2];
        if (grid_reduce<2>(v, part, counter, tot) && threadIdx.x == 0) {
            const double rho = tot[0];
            double beta = 0.0;
            if (sc->restart == 0 && variant != 2) {
                if (sc->rho_prev == 0.0) {
                    sc->status = -4;
                } else {
                    beta = (variant == 0) ? rho / sc->rho_prev : tot[1] / sc->rho_prev;
                }
            }
            if (!isfinite(rho) || !isfinite(beta)) sc->status = -6;
            sc->rho = rho;
            sc->sdr = tot[1];
            sc->beta = beta;
        }
    }
    if (!grid_barrier(bcount, bgen, berr, spin_limit, nblk)) {
        give_up();
        return;
    }
    // ---- p = s + beta p ----
    {
        const double beta = __ldcg(&sc->beta);
#pragma unroll 2
        for (int c = c0; c < nc; c += stride) {
            double sv[4], pv[4];
            lds4<S>(sv, s + 4 * c);
            if (beta == 0.0) {
                st4(p + 4 * c, sv);
            } else {
                ld4(pv, p + 4 * c);
#pragma unroll
                for (int k = 0; k < 4; ++k) pv[k] = fma(beta, pv[k], sv[k]);
                st4(p + 4 * c, pv);
            }
        }
    }
    if (!grid_barrier(bcount, bgen, berr, spin_limit, nblk)) {
        give_up();
        return;
    }
    // ---- q = A p, pq = (p, q), alpha ----
    {
        double a0 = 0.0;
#pragma unroll 2
        for (int c = c0; c < nc; c += stride) {
            const int row = c / nq, xq = c - row * nq;
            const int zz = row / ny, yy = row - zz * ny, xx = 4 * xq;
            const int i = 4 * c;
            double pc[4], nb[4] = {0.0, 0.0, 0.0, 0.0};
            ld4cg(pc, p + i);
            const double pl = (xx > 0) ? __ldcg(p + i - 1) : 0.0, pr = (xx + 4 < nx) ? __ldcg(p + i + 4) : 0.0;
            if (xx > 0) nb[0] += pl;
            nb[1] += pc[0];
            nb[2] += pc[1];
            nb[3] += pc[2];
            nb[0] += pc[1];
            nb[1] += pc[2];
            nb[2] += pc[3];
            if (xx + 4 < nx) nb[3] += pr;
            double t[4];
            if (yy > 0) {
                ld4cg(t, p + i - nx);
#pragma unroll
                for (int k = 0; k < 4; ++k) nb[k] += t[k];
            }
            if (yy < ny - 1) {
                ld4cg(t, p + i + nx);
#pragma unroll
                for (int k = 0; k < 4; ++k) nb[k] += t[k];
            }
            if (zz > 0) {
                ld4cg(t, p + i - npi);
#pragma unroll
                for (int k = 0; k < 4; ++k) nb[k] += t[k];
            }
            if (zz < nz - 1) {
                ld4cg(t, p + i + npi);
#pragma unroll
                for (int k = 0; k < 4; ++k) nb[k] += t[k];
            }
            double qv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qv[k] = 6.0 * pc[k] - nb[k];
                a0 = fma(pc[k], qv[k], a0);
            }
            st4(q + i, qv);
        }
        double v[1] = {a0};
        double tot[1];
        if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) {
            const double pq = tot[0];
            sc->pq = pq;
            if (!(pq > 0.0)) {
                sc->status = (pq == pq) ? -4 : -6;
                sc->alpha = 0.0;
            } else {
                sc->alpha = sc->rho / pq;
            }
        }
    }
    if (!grid_barrier(bcount, bgen, berr, spin_limit, nblk)) {
        give_up();
        return;
    }
    // ---- x += alpha p, r_new = r - alpha q, dr, f0 = (S) r_new, rr ----
    {
        const double alpha = __ldcg(&sc->alpha);
        const bool want_dr = (sc->variant == 1);
        double a0 = 0.0;
#pragma unroll 2
        for (int c = c0; c < nc; c += stride) {
            const int i = 4 * c;
            double xv[4], pv[4], ro[4], qv[4], rn[4];
            ld4(xv, x + i);
            ld4(pv, p + i);
            ld4(ro, r + i);
            ld4(qv, q + i);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xv[k] = fma(alpha, pv[k], xv[k]);
                rn[k] = fma(-alpha, qv[k], ro[k]);
                a0 = fma(rn[k], rn[k], a0);
            }
            st4(x + i, xv);
            st4(r + i, rn);
            if (want_dr) {
                double dv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) dv[k] = rn[k] - ro[k];
                st4(dr + i, dv);
            }
            if (f0 != nullptr) sts4<S>(f0 + i, rn);
        }
        double v[1] = {a0};
        double tot[1];
        if (grid_reduce<1>(v, part, counter, tot) && threadIdx.x == 0) finish_update(sc, tot[0], cond, use_cond);
    }
}

// ---- launchers --------------------------------------------------------------------------------
// Grid of the reduction kernels, measured on GB300: while the Krylov vectors (about six of N
// doubles) stay in the 129 MB L2, two 256-thread CTAs per SM (each thread sums tens of
// products; the last CTA's compensated pass over the partials stays short); past that the
// kernels stream from HBM and need every SM full of warps (8 CTAs per SM) to keep enough loads
// in flight.
int reduction_blocks(long long n) {
    long long b = (n + 256LL * 16 - 1) / (256LL * 16);
    const long long cap = (n <= (4LL << 20)) ? kReduceBlocks : kMaxReduceBlocks;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return static_cast<int>(b);
}

// Grid of the 4-element-chunk kernels: four 256-thread CTAs per SM (a thread handles a few chunks
// at 128^3; the partials stay within the reduction buffer).
int reduction_blocks4(long long n) {
    long long b = (n / 4 + 255) / 256;
    const long long cap = (n <= (4LL << 20)) ? 4 * 152 : kMaxReduceBlocks;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return static_cast<int>(b);
}

// Polls of a grid-barrier wait in the fused tail before it gives up (about a second).
constexpr long long kTailSpinLimit = 10000000;

// True when nb CTAs of the fused tail can all be resident on this device (cached per device).
template <class S>
bool fused_tail_fits(int nb) {
    static int per_sm[64] = {0};
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (per_sm[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tail_fused<S>, 256, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        per_sm[dev] = b > 0 ? b : -1;
    }
    return per_sm[dev] > 0 && static_cast<long long>(per_sm[dev]) * sms[dev] >= nb;
}

#define SMG_PREC_SWITCH(storage, ...)                               \
    switch (storage) {                                              \
    case Prec::F64: { using S = double; __VA_ARGS__; break; }       \
    case Prec::F32: { using S = float; __VA_ARGS__; break; }        \
    case Prec::BF16: { using S = __nv_bfloat16; __VA_ARGS__; break; } \
    }

cudaError_t kry_init_residual(Prec st_prec, int nx, int ny, int nz, const double *b, const double *x, double *r,
                              void *f0, KrylovWork &w, cudaStream_t st) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int nb = reduction_blocks(n);
    SMG_PREC_SWITCH(st_prec, k_init_residual<S><<<nb, 256, 0, st>>>(nx, ny, nz, b, x, r, static_cast<S *>(f0),
                                                                      w.sc, w.part, w.counter));
    return cudaGetLastError();
}

cudaError_t kry_true_residual(int nx, int ny, int nz, const double *b, const double *x, KrylovWork &w,
                              cudaStream_t st) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    k_true_residual<<<reduction_blocks(n), 256, 0, st>>>(nx, ny, nz, b, x, w.sc, w.part, w.counter);
    return cudaGetLastError();
}

cudaError_t kry_iteration_tail(Prec st_prec, int nx, int ny, int nz, const void *s, double *x, double *r, double *p,
                               double *q, double *dr, void *f0, KrylovWork &w, cudaStream_t st,
                               cudaGraphConditionalHandle cond, int use_cond) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int nb = reduction_blocks(n);
    cudaError_t e = cudaSuccess;
    auto al16 = [](const void *v) { return v == nullptr || (reinterpret_cast<uintptr_t>(v) & 15u) == 0; };
    if (nx % 4 == 0 && al16(s) && al16(x) && al16(r) && al16(p) && al16(q) && al16(dr) && al16(f0)) {
        const int nc = static_cast<int>(n / 4);
        const int nb4 = reduction_blocks4(n);
        SMG_PREC_SWITCH(st_prec, {
            const S *sp = static_cast<const S *>(s);
            S *f0p = static_cast<S *>(f0);
            if (w.fused && w.bar != nullptr && fused_tail_fits<S>(nb4)) {
                // one cooperative launch: the runtime refuses it unless every CTA is resident
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(nb4);
                cfg.blockDim = dim3(256);
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, k_tail_fused<S>, nx, ny, nz, sp, x, r, p, q, dr, f0p, w.sc, w.part, w.counter,
                                       w.bar, static_cast<long long>(kTailSpinLimit), cond, use_cond);
                return e != cudaSuccess ? e : cudaGetLastError();
            }
            if (e == cudaSuccess) e = launch_pdl(k_dots_beta4<S>, dim3(nb4), dim3(256), 0, st, nc, sp, r, dr, w.sc, w.part, w.counter);
            if (e == cudaSuccess) e = launch_pdl(k_update_p4<S>, dim3(nb4), dim3(256), 0, st, nc, sp, p, w.sc);
            if (e == cudaSuccess)
                e = launch_pdl(k_spmv_alpha4, dim3(nb4), dim3(256), 0, st, nx, ny, nz, p, q, w.sc, w.part, w.counter);
            if (e == cudaSuccess)
                e = launch_pdl(k_update_xr4<S>, dim3(nb4), dim3(256), 0, st, nc, x, p, r, q, dr, f0p, w.sc, w.part, w.counter,
                               cond, use_cond);
        });
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    SMG_PREC_SWITCH(st_prec, {
        const S *sp = static_cast<const S *>(s);
        S *f0p = static_cast<S *>(f0);
        if (e == cudaSuccess) e = launch_pdl(k_dots_beta<S>, dim3(nb), dim3(256), 0, st, n, sp, r, dr, w.sc, w.part, w.counter);
        if (e == cudaSuccess) e = launch_pdl(k_update_p<S>, dim3(nb), dim3(256), 0, st, n, sp, p, w.sc);
        if (e == cudaSuccess)
            e = launch_pdl(k_spmv_alpha, dim3(nb), dim3(256), 0, st, nx, ny, nz, p, q, w.sc, w.part, w.counter);
        if (e == cudaSuccess)
            e = launch_pdl(k_update_xr<S>, dim3(nb), dim3(256), 0, st, n, x, p, r, q, dr, f0p, w.sc, w.part, w.counter, cond,
                           use_cond);
    });
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace smg
