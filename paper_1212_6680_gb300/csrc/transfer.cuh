// transfer.cuh -- the z-level grid transfers of the SMG V-cycle for one point of a plane
// (section "Preconditioning with SMG" of arXiv:1212.6680; coarse planes at the odd fine
// indices, coarse j <-> fine 2j+1, interpolation weights wm, wp of the even fine planes):
//   restriction of the residual  f_c[j] = r[2j+1] + wp(2j) r[2j] + wm(2j+2) r[2j+2],  r = f - A_l u
//   prolongation + correction    u[2j+1] += e[j],  u[2j] += wm(2j) e[j-1] + wp(2j) e[j]
// Shared by the per-level kernels and the persistent multi-system kernel.
#pragma once

#include "plane_relax.cuh"

namespace smg {

// f_c at point ip of coarse plane j (f, u, fc: one batch entry; zcoef: this level's table).
template <class S, class C>
__device__ __forceinline__ void restrict_point(int nx, int ny, int nzf, const S *__restrict__ f,
                                               const S *__restrict__ u, S *__restrict__ fc,
                                               const C *__restrict__ zcoef, int j, int ip) {
    const long long np = static_cast<long long>(nx) * ny;
    const int y = ip / nx, x = ip - y * nx;
    C acc = C(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int zf = 2 * j + k;
        if (zf >= nzf) break;
        const C *zc = zcoef + static_cast<long long>(zf) * kCoefPerPlane;
        const C w = (k == 1) ? C(1) : (k == 0 ? zc[7] : zc[6]);
        C r = ldv<C>(f + zf * np + ip);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = zf + dz;
            if (zz < 0 || zz >= nzf) continue;
            r -= plane_term<C>(u + zz * np, x, y, nx, ny, zc[1 + dz], zc[4 + dz]);
        }
        acc = fma(w, r, acc);
    }
    stv<S, C>(fc + j * np + ip, acc);
}

// f_c at point ip of the coarse planes j0 .. j1-1: one walk up the fine planes 2 j0 .. 2 j1 that
// computes each fine residual once (the even plane 2j+2 serves coarse planes j and j+1) and each
// plane's (L2D u, u) once (it enters the residuals of three fine planes).  The arithmetic of
// every f_c value is restrict_point's, term by term in the same order and with the same explicit
// roundings.
template <class S, class C>
__device__ __forceinline__ void restrict_column(int nx, int ny, int nzf, const S *__restrict__ f,
                                                const S *__restrict__ u, S *__restrict__ fc,
                                                const C *__restrict__ zcoef, int j0, int j1, int ip) {
    const long long np = static_cast<long long>(nx) * ny;
    const int y = ip / nx, x = ip - y * nx;
    const int zb = 2 * j0, ze = min(2 * j1, nzf - 1);  // fine planes walked
    PlanePoint<C> wm{C(0), C(0)}, w0, wp{C(0), C(0)};  // planes zf - 1, zf, zf + 1
    if (zb > 0) wm = plane_point<C, S>(u + (zb - 1) * np, x, y, nx, ny);
    w0 = plane_point<C, S>(u + zb * np, x, y, nx, ny);
    if (zb + 1 < nzf) wp = plane_point<C, S>(u + (zb + 1) * np, x, y, nx, ny);
    C acc = C(0);  // f_c of the coarse plane being summed
    for (int zf = zb; zf <= ze; ++zf) {
        const C *zc = zcoef + static_cast<long long>(zf) * kCoefPerPlane;
        C r = ldv<C>(f + zf * np + ip);
        if (zf > 0) r -= plane_term_of<C>(wm, zc[0], zc[3]);
        r -= plane_term_of<C>(w0, zc[1], zc[4]);
        if (zf + 1 < nzf) r -= plane_term_of<C>(wp, zc[2], zc[5]);
        const int j = zf >> 1;
        if (zf & 1) {
            acc = fma(C(1), r, acc);          // coarse j, its own fine plane
        } else {
            if (j > j0) {                     // coarse j - 1, its upper even plane: done
                acc = fma(zc[6], r, acc);
                stv<S, C>(fc + (j - 1) * np + ip, acc);
            }
            if (j < j1) acc = fma(zc[7], r, C(0));  // coarse j, its lower even plane
        }
        wm = w0;
        w0 = wp;
        if (zf < ze && zf + 2 < nzf) wp = plane_point<C, S>(u + (zf + 2) * np, x, y, nx, ny);
    }
    if (2 * j1 >= nzf) stv<S, C>(fc + (j1 - 1) * np + ip, acc);  // the last coarse plane has no upper even plane
}

// u at point ip of fine plane z += (P e)
template <class S, class C>
__device__ __forceinline__ void prolong_point(int nx, int ny, int nzf, S *__restrict__ u, const S *__restrict__ uc,
                                              const C *__restrict__ zcoef, int z, int ip) {
    const long long np = static_cast<long long>(nx) * ny;
    const int nzc = nzf / 2;
    C e;
    if (z & 1) {
        e = ldv<C>(uc + static_cast<long long>((z - 1) / 2) * np + ip);
    } else {
        const C *zc = zcoef + static_cast<long long>(z) * kCoefPerPlane;
        e = C(0);
        const int jl = z / 2 - 1, jh = z / 2;
        if (jl >= 0) e += zc[6] * ldv<C>(uc + static_cast<long long>(jl) * np + ip);
        if (jh < nzc) e += zc[7] * ldv<C>(uc + static_cast<long long>(jh) * np + ip);
    }
    S *p = u + static_cast<long long>(z) * np + ip;
    stv<S, C>(p, ldv<C>(p) + e);
}

}  // namespace smg
