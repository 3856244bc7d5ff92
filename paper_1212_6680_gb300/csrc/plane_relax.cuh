// plane_relax.cuh -- SMG plane relaxation on sm_103a: one CTA per z-plane runs the whole 2D
// plane cycle on chip.
//
// One launch relaxes every plane of one colour of one z-level (section "Preconditioning with
// SMG" of arXiv:1212.6680: plane relaxation as the smoother of the SMG V-cycle), for all
// right-hand sides of a batch (blockIdx.y).  Per CTA:
//   1. plane right-hand side g_0 = f_z - sum_dz A_{z,z+dz} u_{z+dz} (terms known to be zero
//      are skipped: mode 0 = first red sweep, mode 1 = first black sweep);
//   2. one 2D V-cycle v = C_z g_0 with zero initial guess: y-semicoarsening, red/black exact
//      x-line relaxation (even then odd lines going down, odd then even going up), exact
//      solve of the single line at the bottom;
//   3. u_z += v (correction form; mode < 2 writes u_z = v).
// Each x-line system (S(y,y) Lx + T(y,y) I) u_y = rhs is tridiagonal and Toeplitz with
// Dirichlet ends; a warp solves it: every lane eliminates its K consecutive rows down to one
// interface unknown (partition method), the 32 interface unknowns are solved by parallel
// cyclic reduction over warp shuffles, and the lanes back-substitute.
//
// Two identities of exact line relaxation are used (they hold exactly in real arithmetic,
// the results differ from the literal cycle only by rounding):
//   * after the down-sweep (even lines with zero neighbours, then odd lines) the residual
//     is zero on odd lines and equals -B_{e,o} u_o on even lines;
//   * going up, odd lines are relaxed first and each new odd line depends only on its even
//     neighbours, so the coarse correction is interpolated to even lines on the fly and
//     the injection into odd lines is not stored.
#pragma once

#include <cuda_bf16.h>

#include "smg_internal.h"

namespace smg {

// ---- storage <-> compute conversion -------------------------------------------------------
template <class C, class S> __device__ __forceinline__ C ldv(const S *p);
template <> __device__ __forceinline__ float ldv<float, float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ldv<float, __nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ double ldv<double, double>(const double *p) { return *p; }
template <> __device__ __forceinline__ double ldv<double, float>(const float *p) { return static_cast<double>(*p); }
template <> __device__ __forceinline__ double ldv<double, __nv_bfloat16>(const __nv_bfloat16 *p) { return static_cast<double>(__bfloat162float(*p)); }

template <class S, class C> __device__ __forceinline__ void stv(S *p, C v);
template <> __device__ __forceinline__ void stv<float, float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void stv<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ void stv<double, double>(double *p, double v) { *p = v; }
template <> __device__ __forceinline__ void stv<float, double>(float *p, double v) { *p = static_cast<float>(v); }
template <> __device__ __forceinline__ void stv<__nv_bfloat16, double>(__nv_bfloat16 *p, double v) { *p = __float2bfloat16_rn(static_cast<float>(v)); }

// ---- warp tridiagonal solver ---------------------------------------------------------------
// Solves the n x n system  of*x[i-1] + dg*x[i] + of*x[i+1] = d[i]  (Dirichlet ends) held by a
// warp: lane l owns rows lK .. lK+K-1 in d[]; rows >= n are identity rows with d = 0.  On
// return d holds x.  dg > 2|of| (strict diagonal dominance) keeps every pivot away from 0.
template <class C, int K>
__device__ __forceinline__ void warp_tridiag(const C dg, const C of, C (&d)[K], const int n, const int lane) {
    const int i0 = lane * K;
    auto A = [&](int j) -> C { const int i = i0 + j; return (i > 0 && i < n) ? of : C(0); };
    auto B = [&](int j) -> C { const int i = i0 + j; return (i < n) ? dg : C(1); };
    auto Cu = [&](int j) -> C { const int i = i0 + j; return (i < n - 1) ? of : C(0); };
    C RA, RB, RC, RD;  // reduced row of the lane's first unknown F:  RA F_prev + RB F + RC F_next = RD
    C ab[K > 1 ? K : 1], cb[K > 1 ? K : 1];
    if constexpr (K == 1) {
        RA = A(0);
        RB = B(0);
        RC = Cu(0);
        RD = d[0];
    } else {
        // forward: rows j >= 1 as  ab[j] F + x_j + cb[j] x_{j+1} = d[j]
        {
            const C inv = C(1) / B(1);
            ab[1] = A(1) * inv;
            cb[1] = Cu(1) * inv;
            d[1] *= inv;
        }
#pragma unroll
        for (int j = 2; j < K; ++j) {
            const C aj = A(j);
            const C inv = C(1) / (B(j) - aj * cb[j - 1]);
            ab[j] = -aj * ab[j - 1] * inv;
            cb[j] = Cu(j) * inv;
            d[j] = (d[j] - aj * d[j - 1]) * inv;
        }
        // backward: rows j >= 1 as  x_j = d[j] - ab[j] F - cb[j] G   (G = next lane's F)
#pragma unroll
        for (int j = K - 2; j >= 1; --j) {
            const C c = cb[j];
            d[j] -= c * d[j + 1];
            ab[j] -= c * ab[j + 1];
            cb[j] = -c * cb[j + 1];
        }
        // previous lane's last row gives x_{i0-1} = pd - pa F_prev - pc F
        C pd = __shfl_up_sync(0xffffffffu, d[K - 1], 1);
        C pa = __shfl_up_sync(0xffffffffu, ab[K - 1], 1);
        C pc = __shfl_up_sync(0xffffffffu, cb[K - 1], 1);
        if (lane == 0) { pd = C(0); pa = C(0); pc = C(0); }
        const C a0 = A(0), c0 = Cu(0);
        RA = -a0 * pa;
        RB = B(0) - a0 * pc - c0 * ab[1];
        RC = -c0 * cb[1];
        RD = d[0] - a0 * pd - c0 * d[1];
    }
    // parallel cyclic reduction of the 32 interface rows
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const C rb = C(1) / RB;
        C am = __shfl_up_sync(0xffffffffu, RA, s), rbm = __shfl_up_sync(0xffffffffu, rb, s);
        C cm = __shfl_up_sync(0xffffffffu, RC, s), dm = __shfl_up_sync(0xffffffffu, RD, s);
        C ap = __shfl_down_sync(0xffffffffu, RA, s), rbp = __shfl_down_sync(0xffffffffu, rb, s);
        C cp = __shfl_down_sync(0xffffffffu, RC, s), dp = __shfl_down_sync(0xffffffffu, RD, s);
        if (lane < s) { am = C(0); rbm = C(0); cm = C(0); dm = C(0); }
        if (lane + s >= 32) { ap = C(0); rbp = C(0); cp = C(0); dp = C(0); }
        const C k1 = RA * rbm, k2 = RC * rbp;
        RB = RB - k1 * cm - k2 * ap;
        RD = RD - k1 * dm - k2 * dp;
        RA = -k1 * am;
        RC = -k2 * cp;
    }
    const C F = RD / RB;
    d[0] = F;
    if constexpr (K > 1) {
        C G = __shfl_down_sync(0xffffffffu, F, 1);
        if (lane == 31) G = C(0);
#pragma unroll
        for (int j = 1; j < K; ++j) d[j] = d[j] - ab[j] * F - cb[j] * G;
    }
}

// ---- one plane: in-plane 5-point term M*L2D u + K*u of a neighbouring plane -----------------
template <class C, class S>
__device__ __forceinline__ C plane_term(const S *u, int x, int y, int nx, int ny, C Mc, C Kc) {
    const long long i = static_cast<long long>(y) * nx + x;
    const C c = ldv<C>(u + i);
    C s = C(4) * c;
    if (x > 0) s -= ldv<C>(u + i - 1);
    if (x < nx - 1) s -= ldv<C>(u + i + 1);
    if (y > 0) s -= ldv<C>(u + i - nx);
    if (y < ny - 1) s -= ldv<C>(u + i + nx);
    return Mc * s + Kc * c;
}

enum : int { NB_NONE = 0, NB_PLAIN = 1, NB_CORR = 2 };
enum : int { OUT_U = 0, OUT_U_AND_PLANE = 1, OUT_PLANE = 2 };

template <class C>
struct PlaneCtx {
    C *sm;       // shared memory base (coefficient table first)
    C *gw;       // this CTA's global slot
    int nx;
};

template <class C>
__device__ __forceinline__ C *arr_u(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m) {
    return (((a.smem_u_mask >> m) & 1u) ? c.sm : c.gw) + a.off_u[m];
}
template <class C>
__device__ __forceinline__ C *arr_g(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m) {
    return (((a.smem_g_mask >> m) & 1u) ? c.sm : c.gw) + a.off_g[m];
}

// Relax line y of 2D level m exactly (one warp).
template <class S, class C, int K>
__device__ __forceinline__ void relax_line(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m, int y,
                                           int nbmode, int out, S *plane, bool accumulate, int lane) {
    const int nx = c.nx, nym = a.ny_m[m];
    const C *lc = c.sm + (a.line_base[m] + y) * kCoefPerLine;
    const C *g = arr_g(a, c, m) + static_cast<long long>(y) * nx;
    C d[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        d[j] = (x < nx) ? g[x] : C(0);
    }
    if (nbmode != NB_NONE) {
        const C *um = arr_u(a, c, m);
        const C *uc = (nbmode == NB_CORR) ? arr_u(a, c, m + 1) : nullptr;
        const int nyc = (nbmode == NB_CORR) ? a.ny_m[m + 1] : 0;
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const int yy = y + s;
            if (yy < 0 || yy >= nym) continue;
            const C sc = lc[1 + s], tc = lc[4 + s];
            C v[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int x = lane * K + j;
                v[j] = (x < nx) ? um[static_cast<long long>(yy) * nx + x] : C(0);
            }
            if (nbmode == NB_CORR) {  // neighbour yy is an even line: add P e from level m+1
                const C *lcy = c.sm + (a.line_base[m] + yy) * kCoefPerLine;
                const int jl = yy / 2 - 1, jh = yy / 2;
                const C wm = lcy[6], wp = lcy[7];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int x = lane * K + j;
                    if (x < nx) {
                        C e = C(0);
                        if (jl >= 0) e += wm * uc[static_cast<long long>(jl) * nx + x];
                        if (jh < nyc) e += wp * uc[static_cast<long long>(jh) * nx + x];
                        v[j] += e;
                    }
                }
            }
            C vl = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
            C vr = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (lane == 0) vl = C(0);
            if (lane == 31) vr = C(0);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const C left = (j == 0) ? vl : v[j - 1];
                const C right = (j == K - 1) ? vr : v[j + 1];
                d[j] -= sc * (C(2) * v[j] - left - right) + tc * v[j];
            }
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (lane * K + j >= nx) d[j] = C(0);
    }
    warp_tridiag<C, K>(C(2) * lc[1] + lc[4], -lc[1], d, nx, lane);
    if (out != OUT_PLANE) {
        C *u = arr_u(a, c, m) + static_cast<long long>(y) * nx;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int x = lane * K + j;
            if (x < nx) u[x] = d[j];
        }
    }
    if (out != OUT_U) {
        S *p = plane + static_cast<long long>(y) * nx;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int x = lane * K + j;
            if (x < nx) {
                const C v = accumulate ? ldv<C>(p + x) + d[j] : d[j];
                stv<S, C>(p + x, v);
            }
        }
    }
}

// g_{m+1}[j] = wp(2j) r_{2j} + wm(2j+2) r_{2j+2},  r_e = -sum_{dy=+-1} B_{e,e+dy} u_{e+dy}
template <class C, int K>
__device__ __forceinline__ void restrict_line(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m, int jc, int lane) {
    const int nx = c.nx, nym = a.ny_m[m];
    const C *um = arr_u(a, c, m);
    C acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = C(0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = 2 * jc + 2 * k;
        if (e >= nym) continue;
        const C *lc = c.sm + (a.line_base[m] + e) * kCoefPerLine;
        const C w = (k == 0) ? lc[7] : lc[6];
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const int yy = e + s;
            if (yy < 0 || yy >= nym) continue;
            const C sc = lc[1 + s], tc = lc[4 + s];
            C v[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int x = lane * K + j;
                v[j] = (x < nx) ? um[static_cast<long long>(yy) * nx + x] : C(0);
            }
            C vl = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
            C vr = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (lane == 0) vl = C(0);
            if (lane == 31) vr = C(0);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const C left = (j == 0) ? vl : v[j - 1];
                const C right = (j == K - 1) ? vr : v[j + 1];
                acc[j] -= w * (sc * (C(2) * v[j] - left - right) + tc * v[j]);
            }
        }
    }
    C *gc = arr_g(a, c, m + 1) + static_cast<long long>(jc) * nx;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        if (x < nx) gc[x] = acc[j];
    }
}

template <class S, class C, int K>
__global__ void __launch_bounds__(512, 1) plane_relax_kernel(const PlaneRelaxArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PlaneCtx<C> c;
    c.sm = reinterpret_cast<C *>(smem_raw);
    c.nx = a.nx;
    const int nx = a.nx, ny = a.ny;
    const long long np = static_cast<long long>(nx) * ny;
    const int z = a.colour + 2 * static_cast<int>(blockIdx.x);
    const int b = blockIdx.y;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    c.gw = reinterpret_cast<C *>(a.gws) + (static_cast<long long>(b) * gridDim.x + blockIdx.x) * a.ws_per_plane;
    const S *fb = reinterpret_cast<const S *>(a.f) + static_cast<long long>(b) * a.vstride;
    S *ub = reinterpret_cast<S *>(a.u) + static_cast<long long>(b) * a.vstride;
    S *plane = ub + static_cast<long long>(z) * np;
    const double *zc = a.zcoef + static_cast<long long>(z) * kCoefPerPlane;
    {
        const double *pc = a.pcoef + static_cast<long long>(z) * a.sum_ny * kCoefPerLine;
        for (int i = tid; i < a.sum_ny * kCoefPerLine; i += nt) c.sm[i] = static_cast<C>(pc[i]);
    }
    const int P = a.P;
    for (int it = 0; it < a.iters; ++it) {
        const int mode = (it == 0) ? a.mode : 2;
        // 1. plane right-hand side
        {
            C *g0 = arr_g(a, c, 0);
            const C Mm = static_cast<C>(zc[0]), M0 = static_cast<C>(zc[1]), Mp = static_cast<C>(zc[2]);
            const C Km = static_cast<C>(zc[3]), K0 = static_cast<C>(zc[4]), Kp = static_cast<C>(zc[5]);
            for (long long i = tid; i < np; i += nt) {
                const int y = static_cast<int>(i / nx), x = static_cast<int>(i - static_cast<long long>(y) * nx);
                C v = ldv<C>(fb + static_cast<long long>(z) * np + i);
                if (mode >= 1) {
                    if (z > 0) v -= plane_term<C>(ub + static_cast<long long>(z - 1) * np, x, y, nx, ny, Mm, Km);
                    if (z + 1 < a.nz) v -= plane_term<C>(ub + static_cast<long long>(z + 1) * np, x, y, nx, ny, Mp, Kp);
                    if (mode == 2) v -= plane_term<C>(plane, x, y, nx, ny, M0, K0);
                }
                g0[i] = v;
            }
        }
        __syncthreads();
        const bool acc = (mode == 2);
        // 2.-3. the 2D cycle, writing v into the plane on the way up
        if (P == 1) {
            if (warp == 0) relax_line<S, C, K>(a, c, 0, 0, NB_NONE, OUT_PLANE, plane, acc, lane);
            __syncthreads();
            continue;
        }
        for (int m = 0; m < P - 1; ++m) {
            const int nym = a.ny_m[m];
            for (int y = 2 * warp; y < nym; y += 2 * nw) relax_line<S, C, K>(a, c, m, y, NB_NONE, OUT_U, plane, false, lane);
            __syncthreads();
            for (int y = 1 + 2 * warp; y < nym; y += 2 * nw) relax_line<S, C, K>(a, c, m, y, NB_PLAIN, OUT_U, plane, false, lane);
            __syncthreads();
            for (int j = warp; j < a.ny_m[m + 1]; j += nw) restrict_line<C, K>(a, c, m, j, lane);
            __syncthreads();
        }
        if (warp == 0) relax_line<S, C, K>(a, c, P - 1, 0, NB_NONE, OUT_U, plane, false, lane);
        __syncthreads();
        for (int m = P - 2; m >= 0; --m) {
            const int nym = a.ny_m[m];
            const int o1 = (m == 0) ? OUT_U_AND_PLANE : OUT_U;
            for (int y = 1 + 2 * warp; y < nym; y += 2 * nw) relax_line<S, C, K>(a, c, m, y, NB_CORR, o1, plane, acc, lane);
            __syncthreads();
            const int o2 = (m == 0) ? OUT_PLANE : OUT_U;
            for (int y = 2 * warp; y < nym; y += 2 * nw) relax_line<S, C, K>(a, c, m, y, NB_PLAIN, o2, plane, acc, lane);
            __syncthreads();
        }
    }
}

template <class S, class C, int K>
int set_smem_attr(size_t smem) {
    return static_cast<int>(cudaFuncSetAttribute(plane_relax_kernel<S, C, K>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)));
}

template <class S, class C, int K>
cudaError_t launch_pr(int nplanes, int nb, int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    dim3 grid(nplanes, nb);
    plane_relax_kernel<S, C, K><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace smg
