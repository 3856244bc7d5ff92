// cycle.cu -- z-level transfer kernels of the SMG V-cycle, precision conversion, the 7-point
// operator, and the dispatch of the plane-relaxation instantiations.
//
// Residual + restriction (one launch per z-level going down) and prolongation + correction
// (one launch per z-level going up) are the grid-transfer steps of the SMG V-cycle
// (section "Preconditioning with SMG" of arXiv:1212.6680).  With the coarse planes at the odd
// fine indices (coarse j <-> fine 2j+1) and the interpolation weights wm, wp of the even fine
// planes:
//   f_c[j] = r[2j+1] + wp(2j) r[2j] + wm(2j+2) r[2j+2],   r = f - A_l u      (R = P^T)
//   u[2j+1] += e[j],  u[2j] += wm(2j) e[j-1] + wp(2j) e[j]                   (P)
// Both are bandwidth-bound stencils; one thread per output point, x fastest (coalesced), the
// 15-point residual reads its five planes through L1/L2.
#include "plane_relax.cuh"

namespace smg {

size_t storage_bytes(Prec p) { return p == Prec::F64 ? 8 : (p == Prec::F32 ? 4 : 2); }

// ---- plane-relaxation dispatch over K ---------------------------------------------------------
#define SMG_DECL_K(k)                                                                                 \
    cudaError_t launch_plane_relax_k##k(Prec, bool, int, int, int, const PlaneRelaxArgs &, size_t,    \
                                        cudaStream_t);                                                \
    int set_plane_relax_smem_k##k(Prec, bool, size_t);
SMG_DECL_K(1)
SMG_DECL_K(2)
SMG_DECL_K(3)
SMG_DECL_K(4)
SMG_DECL_K(6)
SMG_DECL_K(8)
SMG_DECL_K(16)

cudaError_t launch_plane_relax(Prec storage, bool f64, int K, int nplanes, int nb, int threads,
                               const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    switch (K) {
    case 1: return launch_plane_relax_k1(storage, f64, nplanes, nb, threads, a, smem, st);
    case 2: return launch_plane_relax_k2(storage, f64, nplanes, nb, threads, a, smem, st);
    case 3: return launch_plane_relax_k3(storage, f64, nplanes, nb, threads, a, smem, st);
    case 4: return launch_plane_relax_k4(storage, f64, nplanes, nb, threads, a, smem, st);
    case 6: return launch_plane_relax_k6(storage, f64, nplanes, nb, threads, a, smem, st);
    case 8: return launch_plane_relax_k8(storage, f64, nplanes, nb, threads, a, smem, st);
    case 16: return launch_plane_relax_k16(storage, f64, nplanes, nb, threads, a, smem, st);
    }
    return cudaErrorInvalidValue;
}

int set_plane_relax_smem(Prec storage, bool f64, int K, int, size_t smem) {
    switch (K) {
    case 1: return set_plane_relax_smem_k1(storage, f64, smem);
    case 2: return set_plane_relax_smem_k2(storage, f64, smem);
    case 3: return set_plane_relax_smem_k3(storage, f64, smem);
    case 4: return set_plane_relax_smem_k4(storage, f64, smem);
    case 6: return set_plane_relax_smem_k6(storage, f64, smem);
    case 8: return set_plane_relax_smem_k8(storage, f64, smem);
    case 16: return set_plane_relax_smem_k16(storage, f64, smem);
    }
    return static_cast<int>(cudaErrorInvalidValue);
}

// ---- residual + restriction -------------------------------------------------------------------
template <class S, class C>
__global__ void restrict_kernel(int nx, int ny, int nzf, int nzc, long long total, const S *__restrict__ f,
                                const S *__restrict__ u, S *__restrict__ fc, const double *__restrict__ zcoef,
                                long long vsf, long long vsc) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long np = static_cast<long long>(nx) * ny;
    const int x = static_cast<int>(idx % nx);
    long long t = idx / nx;
    const int y = static_cast<int>(t % ny);
    t /= ny;
    const int j = static_cast<int>(t % nzc);
    const int b = static_cast<int>(t / nzc);
    const S *fb = f + b * vsf;
    const S *ub = u + b * vsf;
    const long long ip = static_cast<long long>(y) * nx + x;
    C acc = C(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int zf = 2 * j + k;
        if (zf >= nzf) break;
        const double *zc = zcoef + static_cast<long long>(zf) * kCoefPerPlane;
        const C w = (k == 1) ? C(1) : static_cast<C>(k == 0 ? zc[7] : zc[6]);
        C r = ldv<C>(fb + zf * np + ip);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = zf + dz;
            if (zz < 0 || zz >= nzf) continue;
            r -= plane_term<C>(ub + zz * np, x, y, nx, ny, static_cast<C>(zc[1 + dz]), static_cast<C>(zc[4 + dz]));
        }
        acc += w * r;
    }
    stv<S, C>(fc + b * vsc + j * np + ip, acc);
}

// ---- prolongation + correction ----------------------------------------------------------------
template <class S, class C>
__global__ void prolong_kernel(int nx, int ny, int nzf, int nzc, long long total, S *__restrict__ u,
                               const S *__restrict__ uc, const double *__restrict__ zcoef, long long vsf,
                               long long vsc) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long np = static_cast<long long>(nx) * ny;
    const long long ip = idx % np;
    long long t = idx / np;
    const int z = static_cast<int>(t % nzf);
    const int b = static_cast<int>(t / nzf);
    const S *cb = uc + b * vsc;
    C e;
    if (z & 1) {
        e = ldv<C>(cb + static_cast<long long>((z - 1) / 2) * np + ip);
    } else {
        const double *zc = zcoef + static_cast<long long>(z) * kCoefPerPlane;
        e = C(0);
        const int jl = z / 2 - 1, jh = z / 2;
        if (jl >= 0) e += static_cast<C>(zc[6]) * ldv<C>(cb + static_cast<long long>(jl) * np + ip);
        if (jh < nzc) e += static_cast<C>(zc[7]) * ldv<C>(cb + static_cast<long long>(jh) * np + ip);
    }
    S *p = u + b * vsf + static_cast<long long>(z) * np + ip;
    stv<S, C>(p, ldv<C>(p) + e);
}

static inline unsigned nblocks(long long total, int threads) {
    return static_cast<unsigned>((total + threads - 1) / threads);
}

cudaError_t launch_restrict(Prec storage, int nx, int ny, int nzf, int nb, const void *f, const void *u, void *fc,
                            const double *zcoef, long long vsf, long long vsc, cudaStream_t st) {
    const int nzc = nzf / 2;
    const long long total = static_cast<long long>(nx) * ny * nzc * nb;
    if (total == 0) return cudaSuccess;
    const int T = 256;
    switch (storage) {
    case Prec::F64:
        restrict_kernel<double, double><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<const double *>(f), static_cast<const double *>(u),
            static_cast<double *>(fc), zcoef, vsf, vsc);
        break;
    case Prec::F32:
        restrict_kernel<float, float><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<const float *>(f), static_cast<const float *>(u),
            static_cast<float *>(fc), zcoef, vsf, vsc);
        break;
    case Prec::BF16:
        restrict_kernel<__nv_bfloat16, float><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<const __nv_bfloat16 *>(f), static_cast<const __nv_bfloat16 *>(u),
            static_cast<__nv_bfloat16 *>(fc), zcoef, vsf, vsc);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_prolong(Prec storage, int nx, int ny, int nzf, int nb, void *u, const void *uc,
                           const double *zcoef, long long vsf, long long vsc, cudaStream_t st) {
    const int nzc = nzf / 2;
    const long long total = static_cast<long long>(nx) * ny * nzf * nb;
    const int T = 256;
    switch (storage) {
    case Prec::F64:
        prolong_kernel<double, double><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<double *>(u), static_cast<const double *>(uc), zcoef, vsf, vsc);
        break;
    case Prec::F32:
        prolong_kernel<float, float><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<float *>(u), static_cast<const float *>(uc), zcoef, vsf, vsc);
        break;
    case Prec::BF16:
        prolong_kernel<__nv_bfloat16, float><<<nblocks(total, T), T, 0, st>>>(
            nx, ny, nzf, nzc, total, static_cast<__nv_bfloat16 *>(u), static_cast<const __nv_bfloat16 *>(uc), zcoef,
            vsf, vsc);
        break;
    }
    return cudaGetLastError();
}

// ---- conversions ------------------------------------------------------------------------------
template <class S>
__global__ void to_storage_kernel(long long n, const double *__restrict__ src, S *__restrict__ dst) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) stv<S, double>(dst + i, src[i]);
}
template <class S>
__global__ void from_storage_kernel(long long n, const S *__restrict__ src, double *__restrict__ dst) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = ldv<double>(src + i);
}

cudaError_t launch_convert_to(Prec storage, long long n, const double *src, void *dst, cudaStream_t st) {
    const int T = 256;
    if (n == 0) return cudaSuccess;
    switch (storage) {
    case Prec::F64: return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    case Prec::F32: to_storage_kernel<float><<<nblocks(n, T), T, 0, st>>>(n, src, static_cast<float *>(dst)); break;
    case Prec::BF16:
        to_storage_kernel<__nv_bfloat16><<<nblocks(n, T), T, 0, st>>>(n, src, static_cast<__nv_bfloat16 *>(dst));
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_convert_from(Prec storage, long long n, const void *src, double *dst, cudaStream_t st) {
    const int T = 256;
    if (n == 0) return cudaSuccess;
    switch (storage) {
    case Prec::F64: return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    case Prec::F32:
        from_storage_kernel<float><<<nblocks(n, T), T, 0, st>>>(n, static_cast<const float *>(src), dst);
        break;
    case Prec::BF16:
        from_storage_kernel<__nv_bfloat16><<<nblocks(n, T), T, 0, st>>>(n, static_cast<const __nv_bfloat16 *>(src), dst);
        break;
    }
    return cudaGetLastError();
}

// ---- the 7-point operator in FP64 -------------------------------------------------------------
__global__ void apply_A_kernel(int nx, int ny, int nz, long long total, const double *__restrict__ u,
                               double *__restrict__ out) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long np = static_cast<long long>(nx) * ny, nn = np * nz;
    const long long iv = i % nn;
    const int x = static_cast<int>(iv % nx);
    const int y = static_cast<int>((iv / nx) % ny);
    const int z = static_cast<int>(iv / np);
    double s = u[i - 0] * 6.0;
    double nb = 0.0;
    if (x > 0) nb += u[i - 1];
    if (x < nx - 1) nb += u[i + 1];
    if (y > 0) nb += u[i - nx];
    if (y < ny - 1) nb += u[i + nx];
    if (z > 0) nb += u[i - np];
    if (z < nz - 1) nb += u[i + np];
    out[i] = s - nb;
}

cudaError_t launch_apply_A(int nx, int ny, int nz, int nb, const double *u, double *out, cudaStream_t st) {
    const long long total = static_cast<long long>(nx) * ny * nz * nb;
    const int T = 256;
    if (total == 0) return cudaSuccess;
    apply_A_kernel<<<nblocks(total, T), T, 0, st>>>(nx, ny, nz, total, u, out);
    return cudaGetLastError();
}

}  // namespace smg
