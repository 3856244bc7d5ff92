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
// Both are bandwidth-bound stencils, x fastest (coalesced).  The restriction walks a column of
// kRestrictJ coarse planes per thread, computing each fine residual once; the prolongation has one
// thread per fine point.
#include <cstdlib>
#include "plane_relax.cuh"
#include "transfer.cuh"

namespace smg {

size_t storage_bytes(Prec p) { return p == Prec::F64 ? 8 : (p == Prec::F32 ? 4 : 2); }

// ---- plane-relaxation dispatch over (K, storage precision) -------------------------------------
#define SMG_DECL_KP(k, p)                                                                             \
    cudaError_t launch_plane_relax_k##k##_p##p(bool, int, int, int, const PlaneRelaxArgs &, size_t,   \
                                               cudaStream_t);                                         \
    int set_plane_relax_smem_k##k##_p##p(bool, bool, size_t);                                         \
    bool cluster_resident_k##k##_p##p(bool, int, int, size_t);
#define SMG_DECL_K(k) SMG_DECL_KP(k, 0) SMG_DECL_KP(k, 1) SMG_DECL_KP(k, 2)
SMG_DECL_K(1)
SMG_DECL_K(2)
SMG_DECL_K(3)
SMG_DECL_K(4)
SMG_DECL_K(6)
SMG_DECL_K(8)
SMG_DECL_K(16)

#define SMG_SWITCH_KP(K, storage, CALL)                                                               \
    switch (K) {                                                                                      \
    case 1: SMG_SWITCH_P(1, storage, CALL)                                                            \
    case 2: SMG_SWITCH_P(2, storage, CALL)                                                            \
    case 3: SMG_SWITCH_P(3, storage, CALL)                                                            \
    case 4: SMG_SWITCH_P(4, storage, CALL)                                                            \
    case 6: SMG_SWITCH_P(6, storage, CALL)                                                            \
    case 8: SMG_SWITCH_P(8, storage, CALL)                                                            \
    case 16: SMG_SWITCH_P(16, storage, CALL)                                                          \
    }
#define SMG_SWITCH_P(k, storage, CALL)                                                                \
    switch (storage) {                                                                                \
    case Prec::F64: return CALL(k, 0);                                                                \
    case Prec::F32: return CALL(k, 1);                                                                \
    case Prec::BF16: return CALL(k, 2);                                                               \
    }                                                                                                 \
    break;

// ---- the wide-line kernel's two instantiations (plane_wide.cu with SMG_WK = 8 and 16) -----------
#define SMG_DECL_W(w)                                                                                 \
    long long wide_factor_values_w##w(int, int);                                                      \
    cudaError_t launch_wide_factor_table_w##w(int, int, int, int, const int *, const int *, int,       \
                                              const int *, const double *, const float *, bool, void *, \
                                              cudaStream_t);                                            \
    cudaError_t launch_plane_wide_w##w(Prec, bool, int, int, int, const PlaneRelaxArgs &, size_t,      \
                                       cudaStream_t);                                                 \
    int set_plane_wide_smem_w##w(Prec, bool, bool, size_t);                                           \
    bool wide_cluster_resident_w##w(Prec, bool, int, int, size_t);
SMG_DECL_W(8)
SMG_DECL_W(16)

long long wide_factor_values(int wk, int P, int W) {
    return wk == 8 ? wide_factor_values_w8(P, W) : wide_factor_values_w16(P, W);
}
cudaError_t launch_wide_factor_table(int wk, int nx, int W, int P, int sum_ny, const int *ny_m, const int *line_base,
                                     int nslots, const int *planes, const double *pcoef, const float *pcoef32,
                                     bool f64, void *tab, cudaStream_t st) {
    return wk == 8 ? launch_wide_factor_table_w8(nx, W, P, sum_ny, ny_m, line_base, nslots, planes, pcoef, pcoef32, f64,
                                                 tab, st)
                   : launch_wide_factor_table_w16(nx, W, P, sum_ny, ny_m, line_base, nslots, planes, pcoef, pcoef32,
                                                  f64, tab, st);
}
cudaError_t launch_plane_wide(int wk, Prec storage, bool f64, int nplanes, int nb, int threads, const PlaneRelaxArgs &a,
                              size_t smem, cudaStream_t st) {
    return wk == 8 ? launch_plane_wide_w8(storage, f64, nplanes, nb, threads, a, smem, st)
                   : launch_plane_wide_w16(storage, f64, nplanes, nb, threads, a, smem, st);
}
int set_plane_wide_smem(int wk, Prec storage, bool f64, bool cl, size_t smem) {
    return wk == 8 ? set_plane_wide_smem_w8(storage, f64, cl, smem) : set_plane_wide_smem_w16(storage, f64, cl, smem);
}
bool wide_cluster_resident(int wk, Prec storage, bool f64, int R, int threads, size_t smem) {
    return wk == 8 ? wide_cluster_resident_w8(storage, f64, R, threads, smem)
                   : wide_cluster_resident_w16(storage, f64, R, threads, smem);
}

cudaError_t launch_plane_relax(Prec storage, bool f64, int K, int nplanes, int nb, int threads,
                               const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
#define SMG_CALL_LAUNCH(k, p) launch_plane_relax_k##k##_p##p(f64, nplanes, nb, threads, a, smem, st)
    SMG_SWITCH_KP(K, storage, SMG_CALL_LAUNCH)
    return cudaErrorInvalidValue;
}

int set_plane_relax_smem(Prec storage, bool f64, bool cl, int K, size_t smem) {
#define SMG_CALL_SMEM(k, p) set_plane_relax_smem_k##k##_p##p(f64, cl, smem)
    SMG_SWITCH_KP(K, storage, SMG_CALL_SMEM)
    return static_cast<int>(cudaErrorInvalidValue);
}

bool cluster_resident(Prec storage, bool f64, int K, int R, int threads, size_t smem) {
#define SMG_CALL_RES(k, p) cluster_resident_k##k##_p##p(f64, R, threads, smem)
    SMG_SWITCH_KP(K, storage, SMG_CALL_RES)
    return false;
}

// ---- the shortened-step plane cycle (K <= 4) --------------------------------------------------
#define SMG_DECL_LEAN(k, p)                                                                           \
    cudaError_t launch_plane_lean_k##k##_p##p(bool, int, int, int, const PlaneRelaxArgs &, size_t, cudaStream_t); \
    int set_plane_lean_smem_k##k##_p##p(bool, bool, size_t);                                          \
    bool lean_cluster_resident_k##k##_p##p(bool, int, int, size_t);
#define SMG_DECL_LEAN_K(k) SMG_DECL_LEAN(k, 0) SMG_DECL_LEAN(k, 1) SMG_DECL_LEAN(k, 2)
SMG_DECL_LEAN_K(1)
SMG_DECL_LEAN_K(2)
SMG_DECL_LEAN_K(3)
SMG_DECL_LEAN_K(4)
SMG_DECL_LEAN_K(6)
SMG_DECL_LEAN_K(8)

#define SMG_LEAN_SWITCH(K, storage, CALL)                                                             \
    switch (K) {                                                                                      \
    case 1: SMG_SWITCH_P(1, storage, CALL)                                                            \
    case 2: SMG_SWITCH_P(2, storage, CALL)                                                            \
    case 3: SMG_SWITCH_P(3, storage, CALL)                                                            \
    case 4: SMG_SWITCH_P(4, storage, CALL)                                                            \
    case 6: SMG_SWITCH_P(6, storage, CALL)                                                            \
    case 8: SMG_SWITCH_P(8, storage, CALL)                                                            \
    }

bool lean_supported(int K) { return K >= 1 && K <= 8; }

cudaError_t launch_plane_lean(Prec storage, bool f64, int K, int nplanes, int nb, int threads, const PlaneRelaxArgs &a,
                              size_t smem, cudaStream_t st) {
#define SMG_CALL_LEAN(k, p) launch_plane_lean_k##k##_p##p(f64, nplanes, nb, threads, a, smem, st)
    SMG_LEAN_SWITCH(K, storage, SMG_CALL_LEAN)
    return cudaErrorInvalidValue;
}

int set_plane_lean_smem(Prec storage, bool f64, bool cl, int K, size_t smem) {
#define SMG_CALL_LEAN_SMEM(k, p) set_plane_lean_smem_k##k##_p##p(f64, cl, smem)
    SMG_LEAN_SWITCH(K, storage, SMG_CALL_LEAN_SMEM)
    return static_cast<int>(cudaErrorInvalidValue);
}

bool lean_cluster_resident(Prec storage, bool f64, int K, int R, int threads, size_t smem) {
#define SMG_CALL_LEAN_RES(k, p) lean_cluster_resident_k##k##_p##p(f64, R, threads, smem)
    SMG_LEAN_SWITCH(K, storage, SMG_CALL_LEAN_RES)
    return false;
}

// ---- residual + restriction -------------------------------------------------------------------
constexpr int kRestrictJ = 4;  // coarse planes per thread (restrict_column)
template <class S, class C>
__global__ void restrict_kernel(int nx, int ny, int nzf, int nzc, long long total, const S *__restrict__ f,
                                const S *__restrict__ u, S *__restrict__ fc, const double *__restrict__ zcoef64,
                                const float *__restrict__ zcoef32, long long vsf, long long vsc, int jper) {
    // blockIdx.y: jper consecutive coarse planes, blockIdx.z: one batch entry; x covers the plane
    pdl_trigger();
    pdl_wait();
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= nx * ny) return;
    const int b = blockIdx.z;
    if (jper == 1) {  // one coarse plane per thread
        restrict_point<S, C>(nx, ny, nzf, f + b * vsf, u + b * vsf, fc + b * vsc, coef_table<C>(zcoef64, zcoef32),
                             blockIdx.y, ip);
        return;
    }
    const int j0 = blockIdx.y * jper, j1 = min(j0 + jper, nzc);
    restrict_column<S, C>(nx, ny, nzf, f + b * vsf, u + b * vsf, fc + b * vsc, coef_table<C>(zcoef64, zcoef32), j0,
                          j1, ip);
}

// ---- prolongation + correction ----------------------------------------------------------------
template <class S, class C>
__global__ void prolong_kernel(int nx, int ny, int nzf, int nzc, long long total, S *__restrict__ u,
                               const S *__restrict__ uc, const double *__restrict__ zcoef64,
                               const float *__restrict__ zcoef32, long long vsf, long long vsc) {
    pdl_trigger();
    pdl_wait();
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= nx * ny) return;
    const int b = blockIdx.z;
    prolong_point<S, C>(nx, ny, nzf, u + b * vsf, uc + b * vsc, coef_table<C>(zcoef64, zcoef32), blockIdx.y, ip);
}

static inline unsigned nblocks(long long total, int threads) {
    return static_cast<unsigned>((total + threads - 1) / threads);
}

// Programmatic dependent launch for the kernel chain of one cycle: on unless the environment
// sets SMG_PDL=0 (read once per process).
bool &pdl_enabled() {
    static bool on = [] {
        const char *v = std::getenv("SMG_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

cudaError_t launch_restrict(Prec storage, int nx, int ny, int nzf, int nb, const void *f, const void *u, void *fc,
                            const double *zcoef, const float *zcoef32, long long vsf, long long vsc, cudaStream_t st,
                            bool column) {
    const int nzc = nzf / 2;
    const long long total = static_cast<long long>(nx) * ny * nzc * nb;
    if (total == 0) return cudaSuccess;
    const int T = 256;
    // column walks of kRestrictJ coarse planes per thread where they pay (measured on GB300): with
    // FP64 storage, whose residual arithmetic runs on the slow FP64 pipe, and for launches of at
    // least 4M coarse points; smaller FP32 / BF16 launches are latency-bound and keep one coarse
    // plane per thread (one round of independent loads instead of a walk up nine planes)
    const bool walk = column && (storage == Prec::F64 || total >= (1ll << 22));
    const int jper = walk ? kRestrictJ : 1;
    const int gy = (nzc + jper - 1) / jper;
    const dim3 grid(nblocks(static_cast<long long>(nx) * ny, T), gy, nb);
    cudaError_t e = cudaSuccess;
    switch (storage) {
    case Prec::F64:
        e = launch_pdl(restrict_kernel<double, double>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<const double *>(f), static_cast<const double *>(u),
            static_cast<double *>(fc), zcoef, zcoef32, vsf, vsc, jper);
        break;
    case Prec::F32:
        e = launch_pdl(restrict_kernel<float, float>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<const float *>(f), static_cast<const float *>(u),
            static_cast<float *>(fc), zcoef, zcoef32, vsf, vsc, jper);
        break;
    case Prec::BF16:
        e = launch_pdl(restrict_kernel<__nv_bfloat16, float>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<const __nv_bfloat16 *>(f), static_cast<const __nv_bfloat16 *>(u),
            static_cast<__nv_bfloat16 *>(fc), zcoef, zcoef32, vsf, vsc, jper);
        break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_prolong(Prec storage, int nx, int ny, int nzf, int nb, void *u, const void *uc,
                           const double *zcoef, const float *zcoef32, long long vsf, long long vsc, cudaStream_t st) {
    const int nzc = nzf / 2;
    const long long total = static_cast<long long>(nx) * ny * nzf * nb;
    const int T = 256;
    const dim3 grid(nblocks(static_cast<long long>(nx) * ny, T), nzf, nb);
    cudaError_t e = cudaSuccess;
    switch (storage) {
    case Prec::F64:
        e = launch_pdl(prolong_kernel<double, double>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<double *>(u), static_cast<const double *>(uc), zcoef, zcoef32, vsf, vsc);
        break;
    case Prec::F32:
        e = launch_pdl(prolong_kernel<float, float>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<float *>(u), static_cast<const float *>(uc), zcoef, zcoef32, vsf, vsc);
        break;
    case Prec::BF16:
        e = launch_pdl(prolong_kernel<__nv_bfloat16, float>, grid, dim3(T), 0, st,
            nx, ny, nzf, nzc, total, static_cast<__nv_bfloat16 *>(u), static_cast<const __nv_bfloat16 *>(uc), zcoef,
            zcoef32, vsf, vsc);
        break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
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

// ---- conversion self-check -------------------------------------------------------------------
__global__ void check_conversions_kernel(long long n, const double *__restrict__ src, int *mism) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = src[i];
    const float hw = __double2float_rn(d), sw = narrow_f64(d);
    if (__float_as_uint(hw) != __float_as_uint(sw)) atomicAdd(&mism[0], 1);
    const double wh = static_cast<double>(hw), ws = widen_f32(hw);
    if (__double_as_longlong(wh) != __double_as_longlong(ws)) atomicAdd(&mism[1], 1);
}

cudaError_t launch_check_conversions(long long n, const double *src, int *mism, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    check_conversions_kernel<<<nblocks(n, 256), 256, 0, st>>>(n, src, mism);
    return cudaGetLastError();
}

// ---- the 7-point operator in FP64 -------------------------------------------------------------
__global__ void apply_A_kernel(int nx, int ny, int nz, long long total, const double *__restrict__ u,
                               double *__restrict__ out) {
    // blockIdx.y: plane z, blockIdx.z: batch entry
    const int ip32 = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip32 >= nx * ny) return;
    const long long np = static_cast<long long>(nx) * ny;
    const int y = ip32 / nx, x = ip32 - y * nx;
    const int z = blockIdx.y;
    const long long i = (static_cast<long long>(blockIdx.z) * nz + z) * np + ip32;
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
    apply_A_kernel<<<dim3(nblocks(static_cast<long long>(nx) * ny, T), nz, nb), T, 0, st>>>(nx, ny, nz, total, u, out);
    return cudaGetLastError();
}

}  // namespace smg
