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
        acc += w * r;
    }
    stv<S, C>(fc + j * np + ip, acc);
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
