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

#include <cooperative_groups.h>

#include <type_traits>

#include "smg_internal.h"

namespace smg {

namespace cg = cooperative_groups;

// Step-trace hook for latency studies: compiled out unless SMG_STEP_TRACE names a device
// function `void f(const PlaneRelaxArgs &, int step)`.
#ifdef SMG_STEP_TRACE
#define SMG_TRACE(k) SMG_STEP_TRACE(a, (k))
#else
#define SMG_TRACE(k) ((void)0)
#endif

// ---- storage <-> compute conversion -------------------------------------------------------
// FP32 <-> FP64 conversions written out on the integer pipe from the IEEE-754 binary32 and
// binary64 formats (GB300's conversion instruction runs at a small fraction of even its FP64
// rate).  Widening a normal or zero float is exact: rebias the exponent (1023 - 127 = 896) and
// shift the 23-bit fraction into the top of the 52-bit one.  Narrowing a double whose result
// is a normal float rounds the 52-bit fraction to 23 bits to nearest, ties to even; a carry out
// of the fraction increments the exponent (and gives infinity past the largest float).
// Denormals, infinities and NaNs go through the hardware instruction.
__device__ __forceinline__ double widen_f32(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double(static_cast<long long>(static_cast<unsigned long long>(u) << 32));
    if (e == 0u || e == 0xffu) return static_cast<double>(f);
    const unsigned long long bits = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                                    (static_cast<unsigned long long>(e + 896u) << 52) |
                                    (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ float narrow_f64(double d) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    const unsigned hi = static_cast<unsigned>(b >> 32);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e < 897u || e > 1150u) return __double2float_rn(d);  // not a normal float (or zero)
    const unsigned long long m = b & 0xfffffffffffffull;
    unsigned mant = static_cast<unsigned>(m >> 29);
    const unsigned rem = static_cast<unsigned>(m & 0x1fffffffull);
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) mant += 1u;
    return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + mant));
}

// Programmatic dependent launch (see launch_pdl): both are no-ops for a kernel launched without it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class C, class S> __device__ __forceinline__ C ldv(const S *p);
template <> __device__ __forceinline__ float ldv<float, float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ldv<float, __nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ double ldv<double, double>(const double *p) { return *p; }
template <> __device__ __forceinline__ double ldv<double, float>(const float *p) { return widen_f32(*p); }
template <> __device__ __forceinline__ double ldv<double, __nv_bfloat16>(const __nv_bfloat16 *p) { return widen_f32(__bfloat162float(*p)); }

template <class S, class C> __device__ __forceinline__ void stv(S *p, C v);
template <> __device__ __forceinline__ void stv<float, float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void stv<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ void stv<double, double>(double *p, double v) { *p = v; }
template <> __device__ __forceinline__ void stv<float, double>(float *p, double v) { *p = narrow_f64(v); }
template <> __device__ __forceinline__ void stv<__nv_bfloat16, double>(__nv_bfloat16 *p, double v) { *p = __float2bfloat16_rn(narrow_f64(v)); }

// Coefficient tables are stored in both precisions; each kernel reads the one it computes in.
template <class C> __device__ __forceinline__ const C *coef_table(const double *d64, const float *d32);
template <> __device__ __forceinline__ const double *coef_table<double>(const double *d64, const float *) { return d64; }
template <> __device__ __forceinline__ const float *coef_table<float>(const double *, const float *d32) { return d32; }

// ---- warp tridiagonal solver ---------------------------------------------------------------
// Solves the n x n system  of*x[i-1] + dg*x[i] + of*x[i+1] = d[i]  (Dirichlet ends) held by a
// warp: lane l owns rows lK .. lK+K-1; rows >= n are identity rows with d = 0.  dg > 2|of|
// (strict diagonal dominance) keeps every pivot away from 0.
// Partition method + parallel cyclic reduction, split in two parts:
//   tri_factor : everything that depends only on (dg, of, n) -- all divisions and the
//                coefficient shuffles -- computed once and reused for every line of a level
//                that has the same matrix (all interior lines do);
//   tri_apply  : the right-hand-side sweeps (FMAs and two shuffles per reduction step), for NL
//                lines at once so that their dependency chains interleave.
template <class C, int K>
struct TriFac {
    C dg, of;                  // the matrix these factors belong to
    C inv[K], cbf[K];          // forward pivots (reciprocal) and forward upper coefficients
    C ab[K], cb[K];            // x_j = d_j - ab_j F - cb_j G after the backward sweep
    C a0, c0, rbf;             // the lane's first row and the final pivot (reciprocal)
    C k1[5], k2[5];            // cyclic-reduction multipliers
};

// 1/x: the correctly rounded single-precision reciprocal, or the double division.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <class C, int K>
__device__ __forceinline__ void tri_factor_body(TriFac<C, K> &f, const C dg, const C of, const int n, const int lane) {
    const int i0 = lane * K;
    auto A = [&](int j) -> C { const int i = i0 + j; return (i > 0 && i < n) ? of : C(0); };
    auto B = [&](int j) -> C { const int i = i0 + j; return (i < n) ? dg : C(1); };
    auto Cu = [&](int j) -> C { const int i = i0 + j; return (i < n - 1) ? of : C(0); };
    f.dg = dg;
    f.of = of;
    C RA, RB, RC;
    f.a0 = A(0);
    f.c0 = Cu(0);
    if constexpr (K == 1) {
        RA = f.a0;
        RB = B(0);
        RC = f.c0;
    } else {
        f.inv[1] = recip(B(1));
        f.ab[1] = A(1) * f.inv[1];
        f.cb[1] = Cu(1) * f.inv[1];
#pragma unroll
        for (int j = 2; j < K; ++j) {
            const C aj = A(j);
            f.inv[j] = recip(B(j) - aj * f.cb[j - 1]);
            f.ab[j] = -aj * f.ab[j - 1] * f.inv[j];
            f.cb[j] = Cu(j) * f.inv[j];
        }
#pragma unroll
        for (int j = 1; j < K; ++j) f.cbf[j] = f.cb[j];
#pragma unroll
        for (int j = K - 2; j >= 1; --j) {
            const C c = f.cb[j];
            f.ab[j] -= c * f.ab[j + 1];
            f.cb[j] = -c * f.cb[j + 1];
        }
        C pa = __shfl_up_sync(0xffffffffu, f.ab[K - 1], 1);
        C pc = __shfl_up_sync(0xffffffffu, f.cb[K - 1], 1);
        if (lane == 0) { pa = C(0); pc = C(0); }
        RA = -f.a0 * pa;
        RB = B(0) - f.a0 * pc - f.c0 * f.ab[1];
        RC = -f.c0 * f.cb[1];
    }
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int s = 1 << t;
        const C rb = recip(RB);
        C am = __shfl_up_sync(0xffffffffu, RA, s), rbm = __shfl_up_sync(0xffffffffu, rb, s);
        C cm = __shfl_up_sync(0xffffffffu, RC, s);
        C ap = __shfl_down_sync(0xffffffffu, RA, s), rbp = __shfl_down_sync(0xffffffffu, rb, s);
        C cp = __shfl_down_sync(0xffffffffu, RC, s);
        if (lane < s) { am = C(0); rbm = C(0); cm = C(0); }
        if (lane + s >= 32) { ap = C(0); rbp = C(0); cp = C(0); }
        const C k1 = RA * rbm, k2 = RC * rbp;
        RB = RB - k1 * cm - k2 * ap;
        RA = -k1 * am;
        RC = -k2 * cp;
        f.k1[t] = k1;
        f.k2[t] = k2;
    }
    f.rbf = recip(RB);
}

template <class C, int K>
__device__ __noinline__ void tri_factor_call(TriFac<C, K> &f, const C dg, const C of, const int n, const int lane) {
    tri_factor_body<C, K>(f, dg, of, n, lane);
}

// Inlined, the factors of the current line matrix stay in registers for the whole 2D cycle; an
// out-of-line call puts them in local memory instead (every tri_apply then reloads them), which
// is only worth it when the registers would otherwise spill: the factors take 4K + 15
// values per lane, so they are kept in registers while K * sizeof(C) <= SMG_FAC_REG_BYTES.
#ifndef SMG_FAC_REG_BYTES
#define SMG_FAC_REG_BYTES 32
#endif
template <class C, int K>
__device__ __forceinline__ void tri_factor(TriFac<C, K> &f, const C dg, const C of, const int n, const int lane) {
    if constexpr (K * sizeof(C) <= SMG_FAC_REG_BYTES) tri_factor_body<C, K>(f, dg, of, n, lane);
    else tri_factor_call<C, K>(f, dg, of, n, lane);
}

// A factor set in shared memory: field k of lane l at fs[k * 32 + l].  Only the fields the
// right-hand-side sweeps read are kept: inv[1..K-1], cbf[1..K-2], ab[1..K-1], cb[1..K-1].
template <class C, int K>
constexpr int trifac_fields() { return 2 + (K > 1 ? 4 * K - 5 : 0) + 13; }

template <class C, int K>
__device__ __forceinline__ void trifac_store(C *fs, const TriFac<C, K> &f, int lane) {
    int k = 0;
    fs[(k++) * 32 + lane] = f.dg;
    fs[(k++) * 32 + lane] = f.of;
#pragma unroll
    for (int j = 1; j < K; ++j) fs[(k++) * 32 + lane] = f.inv[j];
#pragma unroll
    for (int j = 1; j < K - 1; ++j) fs[(k++) * 32 + lane] = f.cbf[j];
#pragma unroll
    for (int j = 1; j < K; ++j) fs[(k++) * 32 + lane] = f.ab[j];
#pragma unroll
    for (int j = 1; j < K; ++j) fs[(k++) * 32 + lane] = f.cb[j];
    fs[(k++) * 32 + lane] = f.a0;
    fs[(k++) * 32 + lane] = f.c0;
    fs[(k++) * 32 + lane] = f.rbf;
#pragma unroll
    for (int t = 0; t < 5; ++t) fs[(k++) * 32 + lane] = f.k1[t];
#pragma unroll
    for (int t = 0; t < 5; ++t) fs[(k++) * 32 + lane] = f.k2[t];
}

template <class C, int K>
__device__ __forceinline__ void trifac_load(TriFac<C, K> &f, const C *fs, int lane) {
    int k = 0;
    f.dg = fs[(k++) * 32 + lane];
    f.of = fs[(k++) * 32 + lane];
#pragma unroll
    for (int j = 1; j < K; ++j) f.inv[j] = fs[(k++) * 32 + lane];
#pragma unroll
    for (int j = 1; j < K - 1; ++j) f.cbf[j] = fs[(k++) * 32 + lane];
#pragma unroll
    for (int j = 1; j < K; ++j) f.ab[j] = fs[(k++) * 32 + lane];
#pragma unroll
    for (int j = 1; j < K; ++j) f.cb[j] = fs[(k++) * 32 + lane];
    f.a0 = fs[(k++) * 32 + lane];
    f.c0 = fs[(k++) * 32 + lane];
    f.rbf = fs[(k++) * 32 + lane];
#pragma unroll
    for (int t = 0; t < 5; ++t) f.k1[t] = fs[(k++) * 32 + lane];
#pragma unroll
    for (int t = 0; t < 5; ++t) f.k2[t] = fs[(k++) * 32 + lane];
}

template <class C, int K, int NL>
__device__ __forceinline__ void tri_apply(const TriFac<C, K> &f, C (&d)[NL][K], const int n, const int lane) {
    const int i0 = lane * K;
    C RD[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if constexpr (K == 1) {
            RD[l] = d[l][0];
        } else {
            d[l][1] *= f.inv[1];
#pragma unroll
            for (int j = 2; j < K; ++j) {
                const C aj = (i0 + j < n) ? f.of : C(0);
                d[l][j] = (d[l][j] - aj * d[l][j - 1]) * f.inv[j];
            }
#pragma unroll
            for (int j = K - 2; j >= 1; --j) d[l][j] -= f.cbf[j] * d[l][j + 1];
        }
    }
    if constexpr (K > 1) {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            C pd = __shfl_up_sync(0xffffffffu, d[l][K - 1], 1);
            if (lane == 0) pd = C(0);
            RD[l] = d[l][0] - f.a0 * pd - f.c0 * d[l][1];
        }
    }
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int s = 1 << t;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const C dm = __shfl_up_sync(0xffffffffu, RD[l], s);
            const C dp = __shfl_down_sync(0xffffffffu, RD[l], s);
            RD[l] = RD[l] - f.k1[t] * dm - f.k2[t] * dp;   // k1 = 0 / k2 = 0 where the partner is absent
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const C F = RD[l] * f.rbf;
        if constexpr (K > 1) {
            C G = __shfl_down_sync(0xffffffffu, F, 1);
            if (lane == 31) G = C(0);
#pragma unroll
            for (int j = 1; j < K; ++j) d[l][j] = d[l][j] - f.ab[j] * F - f.cb[j] * G;
        }
        d[l][0] = F;
    }
}

// ---- one plane: in-plane 5-point term M*L2D u + K*u of a neighbouring plane -----------------
// (L2D u, u) at (x, y) of one plane, and the term M*L2D u + K*u from them.
template <class C>
struct PlanePoint {
    C s, c;
};
template <class C, class S>
__device__ __forceinline__ PlanePoint<C> plane_point(const S *u, int x, int y, int nx, int ny) {
    const long long i = static_cast<long long>(y) * nx + x;
    const C c = ldv<C>(u + i);
    C s = C(4) * c;
    if (x > 0) s -= ldv<C>(u + i - 1);
    if (x < nx - 1) s -= ldv<C>(u + i + 1);
    if (y > 0) s -= ldv<C>(u + i - nx);
    if (y < ny - 1) s -= ldv<C>(u + i + nx);
    return PlanePoint<C>{s, c};
}
// the rounding is spelled out (one product, then one fused multiply-add) so that every caller
// gets the same bits whatever the compiler would contract
template <class C>
__device__ __forceinline__ C plane_term_of(const PlanePoint<C> &v, C Mc, C Kc) {
    return fma(Mc, v.s, Kc * v.c);
}
template <class C, class S>
__device__ __forceinline__ C plane_term(const S *u, int x, int y, int nx, int ny, C Mc, C Kc) {
    return plane_term_of<C>(plane_point<C, S>(u, x, y, nx, ny), Mc, Kc);
}

enum : int { NB_NONE = 0, NB_PLAIN = 1, NB_CORR = 2 };
enum : int { OUT_U = 0, OUT_U_AND_PLANE = 1, OUT_PLANE = 2 };

// Where the 2D-cycle arrays live.  CL = false: one CTA owns the plane; every array is either
// in its shared memory or in its global slot.  CL = true: a thread-block cluster of R CTAs
// shares the plane; line y of a 2D level kept on chip belongs to CTA ((y/2) mod R), which
// keeps it in its shared memory at local line ((y/2) div R)*2 + (y mod 2); other CTAs read it
// through distributed shared memory.  Lines are owned in pairs so both colours are spread over
// all CTAs.  An array that does not fit on chip lives whole in the plane's global slot, shared
// by the cluster.
template <class C>
struct PlaneCtx {
    C *sm;       // shared memory base (coefficient table first)
    C *gw;       // the global slot: this CTA's (CL = false) or the cluster's (CL = true)
    C *g0;       // when set: the level-0 right-hand side lives here (the plane of f itself)
    int nx;
    int R, rank; // cluster size and this CTA's rank in it (1, 0 without a cluster)
    C *fs;       // shared-memory factor sets of the interior line matrix of 2D levels 0..MF-1
    int MF;
    bool vec;    // nx == 32 K and every array 16-byte aligned: lanes move their K values as vectors
    unsigned umask, gmask;  // bit m set: u_m / g_m is on chip
    // Per-2D-level table in shared memory, filled once per CTA (indexing the kernel parameters by
    // the run-time level m instead would put a slow dependent load at the head of every step):
    const int *ny;    // lines of level m
    const int *lb;    // first row of level m in the coefficient table
    C *const *ub;     // u_m: base in shared memory (local lines when clustered) or in the global slot
    C *const *gb;     // g_m: the same
};

template <class C, bool CL>
__device__ __forceinline__ C *line_at(const PlaneCtx<C> &c, bool on_chip, C *base, int y) {
    if constexpr (!CL) {
        return base + y * c.nx;
    } else {
        if (!on_chip) return base + y * c.nx;
        const int k = y >> 1;
        const int owner = k % c.R;
        const int local = (k / c.R) * 2 + (y & 1);
        return cg::this_cluster().map_shared_rank(base + local * c.nx, owner);
    }
}
template <class C, bool CL>
__device__ __forceinline__ C *line_u(const PlaneRelaxArgs &, const PlaneCtx<C> &c, int m, int y) {
    return line_at<C, CL>(c, (c.umask >> m) & 1u, c.ub[m], y);
}
template <class C, bool CL>
__device__ __forceinline__ C *line_g(const PlaneRelaxArgs &, const PlaneCtx<C> &c, int m, int y) {
    if (m == 0 && c.g0 != nullptr) return c.g0 + y * c.nx;  // f itself, in global memory
    return line_at<C, CL>(c, (c.gmask >> m) & 1u, c.gb[m], y);
}

template <bool CL>
__device__ __forceinline__ void plane_sync() {
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
}

// The t-th line of a level that this CTA owns, counting lines in owned pairs (all lines).
template <class C, bool CL>
__device__ __forceinline__ int owned_line(const PlaneCtx<C> &c, int t) {
    if constexpr (!CL) return t;
    else return 2 * (c.rank + c.R * (t >> 1)) + (t & 1);
}

// Vector access to a lane's K consecutive values: 16-byte chunks when K*sizeof(T) allows,
// else 8-byte chunks, else none (scalar).
template <class T, int K>
constexpr int vec_chunk() {
    return ((K * sizeof(T)) % 16 == 0) ? 16 : (((K * sizeof(T)) % 8 == 0) ? 8 : 0);
}
template <int B> struct ChunkT;
template <> struct ChunkT<16> { using type = uint4; };
template <> struct ChunkT<8> { using type = uint2; };

template <class T, int K>
__device__ __forceinline__ void vload(T (&v)[K], const T *p) {
    constexpr int CB = vec_chunk<T, K>();
    using CT = typename ChunkT<CB>::type;
    constexpr int PER = CB / sizeof(T);
    union U { CT c; T t[PER]; };
#pragma unroll
    for (int q = 0; q < K / PER; ++q) {
        U u;
        u.c = reinterpret_cast<const CT *>(p)[q];
#pragma unroll
        for (int j = 0; j < PER; ++j) v[q * PER + j] = u.t[j];
    }
}
template <class T, int K>
__device__ __forceinline__ void vstore(T *p, const T (&v)[K]) {
    constexpr int CB = vec_chunk<T, K>();
    using CT = typename ChunkT<CB>::type;
    constexpr int PER = CB / sizeof(T);
    union U { CT c; T t[PER]; };
#pragma unroll
    for (int q = 0; q < K / PER; ++q) {
        U u;
#pragma unroll
        for (int j = 0; j < PER; ++j) u.t[j] = v[q * PER + j];
        reinterpret_cast<CT *>(p)[q] = u.c;
    }
}

// Load a line (K registers per lane, 0 beyond nx).
template <class C, int K>
__device__ __forceinline__ void load_line(C (&v)[K], const C *line, int nx, bool vec, int lane) {
    if constexpr (vec_chunk<C, K>() != 0) {
        if (vec) {
            vload<C, K>(v, line + lane * K);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        v[j] = (x < nx) ? line[x] : C(0);
    }
}
template <class C, int K>
__device__ __forceinline__ void store_line(C *line, const C (&v)[K], int nx, bool vec, int lane) {
    if constexpr (vec_chunk<C, K>() != 0) {
        if (vec) {
            vstore<C, K>(line + lane * K, v);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        if (x < nx) line[x] = v[j];
    }
}

// One row of the plane's coefficient table: couplings to lines y-1, y, y+1 and the weights.
template <class C>
struct CoefRow {
    C s[3], t[3], wm, wp;
};
template <class C>
__device__ __forceinline__ CoefRow<C> coef_row(const C *row) {
    CoefRow<C> r;
    C v[8];
    vload<C, 8>(v, row);
    r.s[0] = v[0]; r.s[1] = v[1]; r.s[2] = v[2];
    r.t[0] = v[3]; r.t[1] = v[4]; r.t[2] = v[5];
    r.wm = v[6]; r.wp = v[7];
    return r;
}

// d -= sc * Lx v + tc * v  for one neighbouring line v (x-halo through shuffles), written as
// d += sc (v_{x-1} + v_{x+1}) - (2 sc + tc) v.
template <class C, int K>
__device__ __forceinline__ void sub_coupling(C (&d)[K], const C (&v)[K], C sc, C tc, int lane) {
    C vl = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
    C vr = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 0) vl = C(0);
    if (lane == 31) vr = C(0);
    const C ac = C(2) * sc + tc;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const C left = (j == 0) ? vl : v[j - 1];
        const C right = (j == K - 1) ? vr : v[j + 1];
        d[j] = fma(sc, left + right, fma(-ac, v[j], d[j]));
    }
}

// Make `fac` hold the factors of the line matrix (dg, of) of 2D level m: keep it when it
// already does, else copy the level's shared factor set when the matrix is that level's
// interior one, else factor (rare: lines next to the last boundary of a level).
template <class C, int K>
__device__ __forceinline__ void ensure_fac(const PlaneCtx<C> &c, TriFac<C, K> &fac, int m, C dg, C of, int lane) {
    if (fac.dg == dg && fac.of == of) return;
    if (m < c.MF) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {  // the level's interior matrix and its last line's
            const C *fs = c.fs + (2 * m + t) * trifac_fields<C, K>() * 32;
            if (fs[lane] == dg && fs[32 + lane] == of) {
                trifac_load<C, K>(fac, fs, lane);
                return;
            }
        }
    }
    tri_factor<C, K>(fac, dg, of, c.nx, lane);
}

// Exact relaxation of NL lines ys[0 .. nvalid) of 2D level m by one warp (lines of one colour,
// so they do not couple to each other); entries past nvalid, if any, repeat a valid line and are
// solved but not stored.  nbmode: the neighbouring lines are
// zero (NB_NONE), read as they are (NB_PLAIN), or read with the coarse correction P u_{m+1}
// added (NB_CORR, the neighbours are even lines).  out: store into u_m, into the plane, or both.
// The modes are warp-uniform runtime values: one compiled body for every step of the 2D cycle
// keeps the kernel's code small enough for the instruction cache.
template <class S, class C, int K, int NL, bool CL>
__device__ __forceinline__ void relax_group(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, TriFac<C, K> &fac,
                                            int m, const int (&ys)[NL], int nvalid, S *plane, bool accumulate,
                                            int nbmode, int out, int lane) {
    const int nx = c.nx, nym = c.ny[m], lbm = c.lb[m];
    C d[NL][K];
    CoefRow<C> cr[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        cr[l] = coef_row<C>(c.sm + (lbm + ys[l]) * kCoefPerLine);
        load_line<C, K>(d[l], line_g<C, CL>(a, c, m, ys[l]), nx, c.vec, lane);
    }
    if (nbmode != NB_NONE) {
        const int nyc = (nbmode == NB_CORR) ? c.ny[m + 1] : 0;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int y = ys[l];
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                const int yy = y + s;
                if (yy < 0 || yy >= nym) continue;
                C v[K];
                load_line<C, K>(v, line_u<C, CL>(a, c, m, yy), nx, c.vec, lane);
                if (nbmode == NB_CORR) {  // neighbour yy is an even line: add P e from level m+1
                    const CoefRow<C> cy = coef_row<C>(c.sm + (lbm + yy) * kCoefPerLine);
                    const int jl = yy / 2 - 1, jh = yy / 2;
                    if (jl >= 0) {
                        C e[K];
                        load_line<C, K>(e, line_u<C, CL>(a, c, m + 1, jl), nx, c.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fma(cy.wm, e[j], v[j]);
                    }
                    if (jh < nyc) {
                        C e[K];
                        load_line<C, K>(e, line_u<C, CL>(a, c, m + 1, jh), nx, c.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fma(cy.wp, e[j], v[j]);
                    }
                }
                sub_coupling<C, K>(d[l], v, cr[l].s[1 + s], cr[l].t[1 + s], lane);
            }
            if (!c.vec) {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (lane * K + j >= nx) d[l][j] = C(0);
            }
        }
    }
    // the line matrices: S(y,y) Lx + T(y,y) I  ->  diagonal 2S + T, off-diagonal -S
    C dg[NL], of[NL];
    bool same = true;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        dg[l] = C(2) * cr[l].s[1] + cr[l].t[1];
        of[l] = -cr[l].s[1];
        same = same && dg[l] == dg[0] && of[l] == of[0];
    }
    if (same) {
        ensure_fac<C, K>(c, fac, m, dg[0], of[0], lane);
        tri_apply<C, K, NL>(fac, d, nx, lane);
    } else {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            ensure_fac<C, K>(c, fac, m, dg[l], of[l], lane);
            C dl[1][K];
#pragma unroll
            for (int j = 0; j < K; ++j) dl[0][j] = d[l][j];
            tri_apply<C, K, 1>(fac, dl, nx, lane);
#pragma unroll
            for (int j = 0; j < K; ++j) d[l][j] = dl[0][j];
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (l >= nvalid) break;
        const int y = ys[l];
        if (out != OUT_PLANE) store_line<C, K>(line_u<C, CL>(a, c, m, y), d[l], nx, c.vec, lane);
        if (out != OUT_U) {
            S *p = plane + y * nx;
            bool done = false;
            if constexpr (vec_chunk<S, K>() != 0) {
                if (c.vec) {
                    S sv[K];
                    if (accumulate) {
                        vload<S, K>(sv, p + lane * K);
#pragma unroll
                        for (int j = 0; j < K; ++j) stv<S, C>(&sv[j], ldv<C>(&sv[j]) + d[l][j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < K; ++j) stv<S, C>(&sv[j], d[l][j]);
                    }
                    vstore<S, K>(p + lane * K, sv);
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int x = lane * K + j;
                    if (x < nx) {
                        const C v = accumulate ? ldv<C>(p + x) + d[l][j] : d[l][j];
                        stv<S, C>(p + x, v);
                    }
                }
            }
        }
    }
}

// Lines a warp processes together: two interleaved dependency chains when a lane's share of a
// line is at most 16 bytes, else one (measured on GB300: four-line groups lose to the larger
// code's instruction-fetch stalls, and wide lines gain nothing from pairing).
template <class C, int K>
constexpr int max_lines_per_group() {
    return (sizeof(C) * K <= 16) ? 2 : 1;
}

// Relax every line of one colour of 2D level m that this CTA owns: lines colour + 2k with
// k = rank + R i; warp w takes i = w, w + nw, ..., NLM at a time while it has NLM left, then
// single lines (two compiled bodies: each extra body costs more in instruction fetch than its
// interleaving gains).
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void relax_colour(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, TriFac<C, K> &fac,
                                             int m, int colour, S *plane, bool accumulate, int nbmode, int out,
                                             int warp, int nw, int lane) {
    const int nl = (c.ny[m] - colour + 1) / 2;
    int nown = nl;
    if constexpr (CL) nown = (nl > c.rank) ? (nl - c.rank + c.R - 1) / c.R : 0;
    auto Y = [&](int i) { return CL ? colour + 2 * (c.rank + c.R * i) : colour + 2 * i; };
    constexpr int NLM = max_lines_per_group<C, K>();
    int i = warp;
    if constexpr (NLM > 1) {
        for (; i + (NLM - 1) * nw < nown; i += NLM * nw) {
            int ys[NLM];
#pragma unroll
            for (int l = 0; l < NLM; ++l) ys[l] = Y(i + l * nw);
            relax_group<S, C, K, NLM, CL>(a, c, fac, m, ys, NLM, plane, accumulate, nbmode, out, lane);
        }
    }
    // the rest one line at a time (on the coarse levels the critical path is one line per warp)
    for (; i < nown; i += nw) {
        const int ys[1] = {Y(i)};
        relax_group<S, C, K, 1, CL>(a, c, fac, m, ys, 1, plane, accumulate, nbmode, out, lane);
    }
}

// Number of lines of an n-line level owned by this CTA (owned in pairs).
template <class C, bool CL>
__device__ __forceinline__ int owned_count(const PlaneCtx<C> &c, int n) {
    if constexpr (!CL) return n;
    const int pairs = (n + 1) / 2;
    const int own_pairs = (pairs > c.rank) ? (pairs - c.rank + c.R - 1) / c.R : 0;
    int cnt = 2 * own_pairs;
    // the last pair may be a single line
    if (own_pairs > 0 && (n & 1) && ((pairs - 1) % c.R) == c.rank) cnt -= 1;
    return cnt;
}

// g_{m+1}[j] = wp(2j) r_{2j} + wm(2j+2) r_{2j+2},  r_e = -sum_{dy=+-1} B_{e,e+dy} u_{e+dy}: the
// residual of level m after its down-sweep is zero on odd lines, and on the even lines 2j, 2j+2
// it comes from the odd lines a = 2j-1, b = 2j+1, c = 2j+3.  Line b couples to both even lines,
// so its two couplings are summed first (one pass over b instead of two):
//   g = -wp(2j) B_{2j,2j-1} a - (wp(2j) B_{2j,2j+1} + wm(2j+2) B_{2j+2,2j+1}) b - wm(2j+2) B_{2j+2,2j+3} c.
// ha: line a exists (j >= 1); h1: even line 2j+2 exists; hc: line c exists.
template <class C, int K>
__device__ __forceinline__ void restrict_combine(C (&acc)[K], const C (&va)[K], const C (&vb)[K], const C (&vc)[K],
                                                 const CoefRow<C> &c0, const CoefRow<C> &c1, bool ha, bool h1,
                                                 bool hc, int lane) {
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = C(0);
    const C w0 = c0.wp;
    if (ha) sub_coupling<C, K>(acc, va, w0 * c0.s[0], w0 * c0.t[0], lane);
    C sb = w0 * c0.s[2], tb = w0 * c0.t[2], w1 = C(0);
    if (h1) {
        w1 = c1.wm;
        sb = fma(w1, c1.s[0], sb);
        tb = fma(w1, c1.t[0], tb);
    }
    sub_coupling<C, K>(acc, vb, sb, tb, lane);
    if (h1 && hc) sub_coupling<C, K>(acc, vc, w1 * c1.s[2], w1 * c1.t[2], lane);
}

template <class C, int K, int NL, bool CL>
__device__ __forceinline__ void restrict_group(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m,
                                               const int (&js)[NL], int lane) {
    const int nx = c.nx, nym = c.ny[m], lbm = c.lb[m];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const int e0 = 2 * js[l];
        const bool ha = e0 >= 1, h1 = e0 + 2 < nym, hc = e0 + 3 < nym;
        C va[K], vb[K], vc[K], acc[K];
#pragma unroll
        for (int q = 0; q < K; ++q) { va[q] = C(0); vc[q] = C(0); }
        if (ha) load_line<C, K>(va, line_u<C, CL>(a, c, m, e0 - 1), nx, c.vec, lane);
        load_line<C, K>(vb, line_u<C, CL>(a, c, m, e0 + 1), nx, c.vec, lane);
        if (hc) load_line<C, K>(vc, line_u<C, CL>(a, c, m, e0 + 3), nx, c.vec, lane);
        const CoefRow<C> c0 = coef_row<C>(c.sm + (lbm + e0) * kCoefPerLine);
        const CoefRow<C> c1 = coef_row<C>(c.sm + (lbm + (h1 ? e0 + 2 : e0)) * kCoefPerLine);
        restrict_combine<C, K>(acc, va, vb, vc, c0, c1, ha, h1, hc, lane);
        store_line<C, K>(line_g<C, CL>(a, c, m + 1, js[l]), acc, nx, c.vec, lane);
    }
}

// The restriction of one level, one coarse line per warp at a time (a single compiled body keeps
// the kernel's code small; the step is short next to the relaxations around it).
template <class C, int K, bool CL>
__device__ __forceinline__ void restrict_level(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int m, int warp,
                                               int nw, int lane) {
    const int nown = owned_count<C, CL>(c, c.ny[m + 1]);
    for (int t = warp; t < nown; t += nw) {
        const int js[1] = {owned_line<C, CL>(c, t)};
        restrict_group<C, K, 1, CL>(a, c, m, js, lane);
    }
}

// Load line y of a plane in storage precision into the lane's K registers (0 beyond nx).
template <class C, class S, int K>
__device__ __forceinline__ void load_plane_line(C (&v)[K], const S *plane, int y, int nx, bool vec, int lane) {
    if constexpr (vec_chunk<S, K>() != 0) {
        if (vec) {
            S sv[K];
            vload<S, K>(sv, plane + y * nx + lane * K);
#pragma unroll
            for (int j = 0; j < K; ++j) v[j] = ldv<C>(&sv[j]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        v[j] = (x < nx) ? ldv<C>(plane + y * nx + x) : C(0);
    }
}

// d -= M (4c - c_{x-1} - c_{x+1} - c_{y-1} - c_{y+1}) + Kc c  for plane pl at line y.
template <class C, class S, int K>
__device__ __forceinline__ void sub_plane_term(C (&d)[K], const S *pl, int y, int nx, int ny, C Mc, C Kc, bool vec,
                                               int lane) {
    C cv[K], up[K], dn[K];
    load_plane_line<C, S, K>(cv, pl, y, nx, vec, lane);
#pragma unroll
    for (int j = 0; j < K; ++j) { up[j] = C(0); dn[j] = C(0); }
    if (y > 0) load_plane_line<C, S, K>(up, pl, y - 1, nx, vec, lane);
    if (y + 1 < ny) load_plane_line<C, S, K>(dn, pl, y + 1, nx, vec, lane);
    C vl = __shfl_up_sync(0xffffffffu, cv[K - 1], 1);
    C vr = __shfl_down_sync(0xffffffffu, cv[0], 1);
    if (lane == 0) vl = C(0);
    if (lane == 31) vr = C(0);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const C left = (j == 0) ? vl : cv[j - 1];
        const C right = (j == K - 1) ? vr : cv[j + 1];
        d[j] -= Mc * (C(4) * cv[j] - left - right - up[j] - dn[j]) + Kc * cv[j];
    }
}

// g_0 = f_z - sum_dz A_{z,z+dz} u_{z+dz} for NL lines (mode 1: own plane zero; mode 2: all).
template <class S, class C, int K, int NL, bool CL>
__device__ __forceinline__ void rhs_group(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, const int (&ys)[NL],
                                          int mode, const S *fpl, const S *ub, int z, const C *zc, int lane) {
    const int nx = a.nx, ny = a.ny, np = nx * ny;
    C d[NL][K];
#pragma unroll
    for (int l = 0; l < NL; ++l) load_plane_line<C, S, K>(d[l], fpl, ys[l], nx, c.vec, lane);
    if (mode >= 1 && z > 0) {
        const C Mc = zc[0], Kc = zc[3];
#pragma unroll
        for (int l = 0; l < NL; ++l) sub_plane_term<C, S, K>(d[l], ub + (z - 1) * np, ys[l], nx, ny, Mc, Kc, c.vec, lane);
    }
    if (mode >= 1 && z + 1 < a.nz) {
        const C Mc = zc[2], Kc = zc[5];
#pragma unroll
        for (int l = 0; l < NL; ++l) sub_plane_term<C, S, K>(d[l], ub + (z + 1) * np, ys[l], nx, ny, Mc, Kc, c.vec, lane);
    }
    if (mode == 2) {
        const C Mc = zc[1], Kc = zc[4];
#pragma unroll
        for (int l = 0; l < NL; ++l) sub_plane_term<C, S, K>(d[l], ub + z * np, ys[l], nx, ny, Mc, Kc, c.vec, lane);
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) store_line<C, K>(line_g<C, CL>(a, c, 0, ys[l]), d[l], nx, c.vec, lane);
}

// The plane right-hand side, one line per warp at a time (single compiled body, as above).
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void compute_rhs(const PlaneRelaxArgs &a, const PlaneCtx<C> &c, int mode, const S *fpl,
                                            const S *ub, int z, const C *zc, int warp, int nw, int lane) {
    const int nown = owned_count<C, CL>(c, a.ny);
    for (int t = warp; t < nown; t += nw) {
        const int ys[1] = {owned_line<C, CL>(c, t)};
        rhs_group<S, C, K, 1, CL>(a, c, ys, mode, fpl, ub, z, zc, lane);
    }
}

// The relaxation of one plane (the pidx-th plane of the colour, batch entry b) by one CTA
// (CL = false) or by this CTA's share of a cluster (CL = true).  `slot` selects the CTA's part
// of the global workspace.  Used by the per-launch kernel below and by the persistent
// multi-system kernel.
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void plane_task(const PlaneRelaxArgs &a, int pidx, int b, long long slot, int rank,
                                           unsigned char *smem_raw) {
    PlaneCtx<C> c;
    c.sm = reinterpret_cast<C *>(smem_raw);
    c.g0 = nullptr;
    c.nx = a.nx;
    c.vec = a.vec != 0;
    c.R = CL ? a.R : 1;
    c.rank = rank;
    const int nx = a.nx, ny = a.ny;
    const long long np = static_cast<long long>(nx) * ny;
    const int z = a.colour + 2 * pidx;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    c.gw = reinterpret_cast<C *>(a.gws) + slot * a.ws_per_plane;
    c.umask = a.smem_u_mask;
    c.gmask = a.smem_g_mask;
    {
        __shared__ int s_ny[kMaxPlaneLevels], s_lb[kMaxPlaneLevels];
        __shared__ C *s_ub[kMaxPlaneLevels], *s_gb[kMaxPlaneLevels];
        if (tid < a.P) {
            s_ny[tid] = a.ny_m[tid];
            s_lb[tid] = a.line_base[tid];
            s_ub[tid] = (((c.umask >> tid) & 1u) ? c.sm : c.gw) + a.off_u[tid];
            s_gb[tid] = (((c.gmask >> tid) & 1u) ? c.sm : c.gw) + a.off_g[tid];
        }
        c.ny = s_ny;
        c.lb = s_lb;
        c.ub = s_ub;
        c.gb = s_gb;
    }
    const S *fb = reinterpret_cast<const S *>(a.f) + static_cast<long long>(b) * a.vstride;
    S *ub = reinterpret_cast<S *>(a.u) + static_cast<long long>(b) * a.vstride;
    S *plane = ub + static_cast<long long>(z) * np;
    const C *zc = coef_table<C>(a.zcoef, a.zcoef32) + static_cast<long long>(z) * kCoefPerPlane;
    {
        const C *pc = coef_table<C>(a.pcoef, a.pcoef32) + static_cast<long long>(z) * a.sum_ny * kCoefPerLine;
        for (int i = tid; i < a.sum_ny * kCoefPerLine; i += nt) c.sm[i] = pc[i];
    }
    // the interior line matrix of each of the first MF 2D levels is factored once, by warp m
    c.fs = c.sm + a.off_fs;
    c.MF = a.MF;
    TriFac<C, K> fac;
    __syncthreads();
    SMG_TRACE(0);
    // factor sets: per 2D level, the interior line matrix (line 0) and the last line's (the only
    // other one when ny is a power of two); set 2m + t, computed by warps in parallel
    for (int sidx = warp; sidx < 2 * a.MF; sidx += nw) {
        const int mm = sidx >> 1;
        const int y = (sidx & 1) ? c.ny[mm] - 1 : 0;
        const C *lc = c.sm + (c.lb[mm] + y) * kCoefPerLine;
        tri_factor<C, K>(fac, C(2) * lc[1] + lc[4], -lc[1], nx, lane);
        trifac_store<C, K>(c.fs + sidx * trifac_fields<C, K>() * 32, fac, lane);
    }
    // everything above reads only the hierarchy's coefficient tables: with programmatic dependent
    // launch it overlaps the previous kernel; from here on the planes are read and written
    pdl_wait();
    fac.dg = C(0);  // no real line matrix has a zero diagonal: the first line always refreshes
    fac.of = C(0);
    const int P = a.P;
    for (int it = 0; it < a.iters; ++it) {
        const int mode = (it == 0) ? a.mode : 2;
        // 1. plane right-hand side (the first red sweep reads f_z itself when it is in the
        //    compute precision)
        const S *fpl = fb + static_cast<long long>(z) * np;
        c.g0 = nullptr;
        if constexpr (std::is_same<S, C>::value) {
            if (mode == 0) c.g0 = const_cast<C *>(reinterpret_cast<const C *>(fpl));
        }
        if (c.g0 == nullptr) compute_rhs<S, C, K, CL>(a, c, mode, fpl, ub, z, zc, warp, nw, lane);
        plane_sync<CL>();
        SMG_TRACE(1);
        const bool acc = (mode == 2);
        // 2.-3. the 2D cycle, writing v into the plane on the way up, as one loop over its steps
        //   down,   m = 0 .. P-2:  even lines (no neighbours), odd lines, restriction
        //   bottom: the single line of level P-1
        //   up,     m = P-2 .. 0:  odd lines (neighbours + coarse correction), even lines;
        //                          level 0 writes the plane (accumulating in correction form)
        // so that every relaxation goes through the same inlined code.
        const int nsteps = (P == 1) ? 1 : 5 * P - 4;
        for (int st = 0; st < nsteps; ++st) {
            int m, colour, nbmode, out;
            bool accu = false, is_restrict = false;
            if (P == 1) {
                m = 0, colour = 0, nbmode = NB_NONE, out = OUT_PLANE, accu = acc;
            } else if (st < 3 * (P - 1)) {
                m = st / 3;
                const int k = st - 3 * m;
                is_restrict = (k == 2);
                colour = k;
                nbmode = (k == 0) ? NB_NONE : NB_PLAIN;
                out = OUT_U;
            } else if (st == 3 * (P - 1)) {
                m = P - 1, colour = 0, nbmode = NB_NONE, out = OUT_U;
            } else {
                const int u = st - 3 * (P - 1) - 1;
                m = P - 2 - u / 2;
                colour = (u & 1) ? 0 : 1;
                nbmode = colour ? NB_CORR : NB_PLAIN;
                out = (m > 0) ? OUT_U : (colour ? OUT_U_AND_PLANE : OUT_PLANE);
                accu = acc;
            }
            // opaque to the optimiser, so that it keeps one copy of the step instead of cloning it
            // per branch of the decoding above to propagate the constants
            int accu_i = accu ? 1 : 0, rs_i = is_restrict ? 1 : 0;
            asm volatile("" : "+r"(m), "+r"(colour), "+r"(nbmode), "+r"(out), "+r"(accu_i), "+r"(rs_i));
            if (rs_i) restrict_level<C, K, CL>(a, c, m, warp, nw, lane);
            else relax_colour<S, C, K, CL>(a, c, fac, m, colour, plane, accu_i != 0, nbmode, out, warp, nw, lane);
            plane_sync<CL>();
            SMG_TRACE(2 + st);
        }
    }
}

// One CTA (CL = false) or one cluster of R CTAs (CL = true) per plane of the colour;
// blockIdx.y is the batch entry.
template <class S, class C, int K, bool CL>
__global__ void __launch_bounds__(512, 1) plane_relax_kernel(const __grid_constant__ PlaneRelaxArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    int pidx, rank;
    if constexpr (CL) {
        rank = static_cast<int>(cg::this_cluster().block_rank());
        pidx = static_cast<int>(blockIdx.x) / a.R;
    } else {
        rank = 0;
        pidx = static_cast<int>(blockIdx.x);
    }
    // global slot: one per CTA, or one per cluster (the plane's arrays that are not on chip)
    const long long slot = CL ? static_cast<long long>(blockIdx.y) * (gridDim.x / a.R) + pidx
                              : static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
    plane_task<S, C, K, CL>(a, pidx, static_cast<int>(blockIdx.y), slot, rank, smem_raw);
}

template <class S, class C, int K, bool CL>
int set_smem_attr(size_t smem) {
    cudaError_t e = raise_smem_attr(reinterpret_cast<const void *>(&plane_relax_kernel<S, C, K, CL>), smem);
    if (e == cudaSuccess && CL)
        e = cudaFuncSetAttribute(plane_relax_kernel<S, C, K, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return static_cast<int>(e);
}

template <class S, class C, int K, bool CL>
cudaError_t launch_pr(int nplanes, int nb, int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    if constexpr (!CL) {
        return launch_pdl(plane_relax_kernel<S, C, K, false>, dim3(nplanes, nb), dim3(threads), smem, st, a);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nplanes * a.R, nb, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = a.R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl_enabled() ? 2 : 1;
        return cudaLaunchKernelEx(&cfg, plane_relax_kernel<S, C, K, true>, a);
    }
}

}  // namespace smg
