// plane_wide.cu -- SMG plane relaxation for x-lines split over several warps: segments of
// 32 SMG_WK rows (SMG_WK rows per lane), compiled once with SMG_WK = 16 (lines of 513-2048 rows,
// longer than one warp holds) and once with SMG_WK = 8 (lines of 257-512 rows, two warps of 8
// rows per lane instead of one of 16).
//
// The plane cycle is the one of plane_relax.cuh (section "Preconditioning with SMG" of
// arXiv:1212.6680: plane relaxation as the SMG smoother, each plane by a 2D y-semicoarsening
// V-cycle with exact x-line solves); only the x-line solve changes.  A line of nx rows is cut
// into W = ceil(nx / (32 SMG_WK)) segments of 32 SMG_WK rows (the last one shorter), and a team
// of W warps owns the line, warp s holding segment s.  The exact solve of the Toeplitz
// tridiagonal system T x = d (diagonal dg, off-diagonal of, Dirichlet ends) is split as follows.
// With T_s the segment's own block and x_s its part of x,
//     T_s x_s = d_s - of v_{s-1} e_first - of u_{s+1} e_last,
// where v_{s-1} is the last value of segment s-1 and u_{s+1} the first value of segment s+1.
// So x_s = y_s - of v_{s-1} eL_s - of u_{s+1} eR_s with y_s = T_s^{-1} d_s (the warp solver of
// plane_relax.cuh on the segment alone), eL_s = T_s^{-1} e_first and eR_s = T_s^{-1} e_last.
// Taking the first and last entries of that identity for every segment gives 2W equations in
// the 2W unknowns (u_s, v_s):
//     u_s + of eL_s[0] v_{s-1} + of eR_s[0] u_{s+1} = y_s[0]
//     v_s + of eL_s[L] v_{s-1} + of eR_s[L] u_{s+1} = y_s[L]      (L = last row of segment s)
// The matrix M of that reduced system depends only on (dg, of) and the segment lengths; its
// inverse rows for v_{s-1} and u_{s+1} are formed once per line matrix, so a line solve costs
// the segment solve, one exchange of (y_s[0], y_s[L]) through shared memory, 4W FMAs and the
// correction x_s = y_s - of v_{s-1} eL_s - of u_{s+1} eR_s.  In real arithmetic this is the
// exact line solve; it differs from a one-warp solve only by rounding.
// The x-halo of a segment (the neighbouring segments' edge values, read by the couplings) is
// read from the line in memory.  One CTA per plane, or a thread-block cluster of R CTAs per
// plane: line y of an array kept on chip then belongs to CTA (y/2) mod R (local line
// ((y/2) div R)*2 + y mod 2, the layout of plan_plane_layout_cluster), which relaxes, restricts
// and assembles it, reading other CTAs' lines through distributed shared memory; the team of a
// line is always inside one CTA.  The 2D cycle runs in the general step order or in the
// shortened one of plane_lean.cuh (each step that fills a level's right-hand side also solves
// that level's even lines; the same solves on the same data, bit-identical).  The solver data of
// every 2D level's two line matrices can come from a table formed once per allocation of the
// level vectors (wide_factor_kernel), in the level's compute type: at about two FP64 FMAs per
// clock per SM, forming them costs a one-CTA FP64 plane tens of microseconds per step.
#include "plane_relax.cuh"

namespace smg {

namespace {

#ifndef SMG_WK
#error "compile with -DSMG_WK=<rows per lane in a segment: 8 or 16>"
#endif
constexpr int kWK = SMG_WK;          // rows per lane in a segment
constexpr int kSeg = 32 * kWK;       // rows per segment (one warp)
constexpr int kMaxSeg = 4;           // segments per line: nx <= 4 kSeg
constexpr int kXchg = 4;             // values a warp publishes per exchange

template <class C>
struct WideCtx {
    C *sm;        // shared memory base (coefficient table first)
    C *gw;        // this CTA's global slot
    C *g0;        // when set: the level-0 right-hand side is the plane of f itself
    int nx;
    int W;        // segments per line = warps per team
    int seg, team, nteam, warp;
    int x0, ns;   // this warp's segment: first row and number of rows
    bool vec;     // the segment is full and every line 16-byte aligned: vector access
    const int *ny, *lb;
    C *const *ub;
    C *const *gb;
    const int *uon, *gon;  // [m]: the level's u / g is on chip (spread over the cluster when R > 1)
    int R, lr, rank;       // CTAs per plane (2^lr) and this CTA's rank
    C *xb;        // exchange buffers: two of [warps][kXchg]
    const C *ftab; // this plane's precomputed solver data ([m][set][segment] entries), or null
};

// The line solver's data for one line matrix (dg, of) on this warp's segment.
// Threads of a wide-line CTA: 512 for FP64 compute; 384 for FP32 compute, which leaves 168
// registers a thread (128 at 512) for the line-solver data (fewer teams of warps per CTA, but
// measured faster on the paper's bricks).
template <class C>
constexpr int wide_threads() { return sizeof(C) == 8 ? 512 : 384; }
template <class C>
constexpr bool kWfRegs() { return sizeof(C) == 8 || kWK == 8; }

template <class C>
struct WideFac {
    TriFac<C, kWK> f;                    // factors of T_s (rows >= ns are identity rows)
    C eL[kWK], eR[kWK];                  // T_s^{-1} e_first, T_s^{-1} e_last (the lane's rows)
    C mv[2 * kMaxSeg], mu[2 * kMaxSeg];  // rows of M^{-1} giving v_{s-1} and u_{s+1}
};

template <class C>
__device__ __forceinline__ void team_sync(const WideCtx<C> &c) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + c.team), "r"(32 * c.W) : "memory");
}

// Line y of an array at `base`: in this CTA's slot or shared memory, or (a cluster's on-chip
// array) in the shared memory of the CTA that owns it.
template <class C>
__device__ __forceinline__ C *wline(const WideCtx<C> &c, C *base, int on, int y) {
    if (c.R > 1 && on) {
        const int k = y >> 1;
        const int local = ((k >> c.lr) << 1) + (y & 1);
        return cg::this_cluster().map_shared_rank(base + static_cast<long long>(local) * c.nx, k & (c.R - 1));
    }
    return base + static_cast<long long>(y) * c.nx;
}
template <class C>
__device__ __forceinline__ C *wline_u(const WideCtx<C> &c, int m, int y) {
    return wline(c, c.ub[m], c.uon[m], y);
}
template <class C>
__device__ __forceinline__ C *wline_g(const WideCtx<C> &c, int m, int y) {
    if (m == 0 && c.g0 != nullptr) return c.g0 + static_cast<long long>(y) * c.nx;
    return wline(c, c.gb[m], c.gon[m], y);
}

// The j-th line this CTA owns of a level with n lines (the pairs (2i, 2i+1) with i mod R equal to
// its rank; every line with one CTA), or n past the last: increasing in j.
template <class C>
__device__ __forceinline__ int owned_line(const WideCtx<C> &c, int j, int n) {
    const int y = 2 * (c.rank + ((j >> 1) << c.lr)) + (j & 1);
    return y < n ? y : n;
}

// The i-th item of a fused step's work list over a level of n lines: the owned even lines first
// (each carrying a line solve besides its right-hand side), then the owned odd lines, so that the
// teams share the solves evenly; n past the last.
template <class C>
__device__ __forceinline__ int fused_line(const WideCtx<C> &c, int i, int n, bool &even) {
    const int pe = (n + 1) >> 1;  // even lines of the level
    const int ne = pe > c.rank ? (pe - c.rank + c.R - 1) >> c.lr : 0;
    even = i < ne;
    const int y = even ? 2 * (c.rank + (i << c.lr)) : 2 * (c.rank + ((i - ne) << c.lr)) + 1;
    return y < n ? y : n;
}

// Row x of a line, 0 outside 0 .. nx-1.
template <class T>
__device__ __forceinline__ T wat(const T *line, int nx, int x) {
    return (x >= 0 && x < nx) ? line[x] : T(0);
}

// This warp's segment of a line (compute type), 0 beyond the segment's rows.
template <class C>
__device__ __forceinline__ void wload(C (&v)[kWK], const C *line, const WideCtx<C> &c, int lane) {
    const C *p = line + c.x0;
    if (c.vec) {
        vload<C, kWK>(v, p + lane * kWK);
        return;
    }
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        const int x = lane * kWK + j;
        v[j] = (x < c.ns) ? p[x] : C(0);
    }
}
template <class C>
__device__ __forceinline__ void wstore(C *line, const C (&v)[kWK], const WideCtx<C> &c, int lane) {
    C *p = line + c.x0;
    if (c.vec) {
        vstore<C, kWK>(p + lane * kWK, v);
        return;
    }
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        const int x = lane * kWK + j;
        if (x < c.ns) p[x] = v[j];
    }
}

// This warp's segment of line y of a plane in storage precision.
template <class C, class S>
__device__ __forceinline__ void wload_plane(C (&v)[kWK], const S *plane, int y, const WideCtx<C> &c, int lane) {
    const S *p = plane + static_cast<long long>(y) * c.nx + c.x0;
    if constexpr (vec_chunk<S, kWK>() != 0) {
        if (c.vec) {
            S sv[kWK];
            vload<S, kWK>(sv, p + lane * kWK);
#pragma unroll
            for (int j = 0; j < kWK; ++j) v[j] = ldv<C>(&sv[j]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        const int x = lane * kWK + j;
        v[j] = (x < c.ns) ? ldv<C>(p + x) : C(0);
    }
}

// d -= sc Lx v + tc v for one neighbouring line v, the x-halo of the segment given (hl for lane
// 0, hr for lane 31; only those lanes' values are read).
template <class C>
__device__ __forceinline__ void sub_coupling_h(C (&d)[kWK], const C (&v)[kWK], C sc, C tc, C hl, C hr, int lane) {
    C vl = __shfl_up_sync(0xffffffffu, v[kWK - 1], 1);
    C vr = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 0) vl = hl;
    if (lane == 31) vr = hr;
    const C ac = C(2) * sc + tc;
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        const C left = (j == 0) ? vl : v[j - 1];
        const C right = (j == kWK - 1) ? vr : v[j + 1];
        d[j] = fma(sc, left + right, fma(-ac, v[j], d[j]));
    }
}

// Segment of line y (level m) with its x-halo, the coarse correction of level m+1 added when
// `corr` (neighbour lines of an odd line going up are even lines).
template <class C>
__device__ __forceinline__ void wload_nb(C (&v)[kWK], C &hl, C &hr, const WideCtx<C> &c, int m, int y, bool corr,
                                         int lane) {
    const C *lu = wline_u(c, m, y);
    wload(v, lu, c, lane);
    const int xl = c.x0 - 1, xr = c.x0 + kSeg;
    hl = (lane == 0) ? wat(lu, c.nx, xl) : C(0);
    hr = (lane == 31) ? wat(lu, c.nx, xr) : C(0);
    if (corr) {
        const CoefRow<C> cy = coef_row<C>(c.sm + (c.lb[m] + y) * kCoefPerLine);
        const int jl = y / 2 - 1, jh = y / 2;
        if (jl >= 0) {
            const C *le = wline_u(c, m + 1, jl);
            C e[kWK];
            wload(e, le, c, lane);
#pragma unroll
            for (int j = 0; j < kWK; ++j) v[j] = fma(cy.wm, e[j], v[j]);
            if (lane == 0) hl = fma(cy.wm, wat(le, c.nx, xl), hl);
            if (lane == 31) hr = fma(cy.wm, wat(le, c.nx, xr), hr);
        }
        if (jh < c.ny[m + 1]) {
            const C *le = wline_u(c, m + 1, jh);
            C e[kWK];
            wload(e, le, c, lane);
#pragma unroll
            for (int j = 0; j < kWK; ++j) v[j] = fma(cy.wp, e[j], v[j]);
            if (lane == 0) hl = fma(cy.wp, wat(le, c.nx, xl), hl);
            if (lane == 31) hr = fma(cy.wp, wat(le, c.nx, xr), hr);
        }
    }
}

// Value of row i of the segment (held by lane i / kWK, register i % kWK), broadcast to the warp.
template <class C>
__device__ __forceinline__ C seg_value(const C (&v)[kWK], int i) {
    const int l = i / kWK, j = i - l * kWK;
    C t = C(0);
#pragma unroll
    for (int q = 0; q < kWK; ++q)
        if (q == j) t = v[q];
    return __shfl_sync(0xffffffffu, t, l);
}

// Publish n values of this warp, wait for the team, return the exchange buffer to read.
template <class C>
__device__ __forceinline__ const C *exchange(const WideCtx<C> &c, int &xp, const C *vals, int n, int lane) {
    C *b = c.xb + (xp & 1) * (16 * kXchg);
    if (lane == 0)
        for (int k = 0; k < n; ++k) b[c.warp * kXchg + k] = vals[k];
    team_sync(c);
    ++xp;  // two buffers: a warp rewrites this one only after every team warp has passed the next barrier
    return b + (c.warp - c.seg) * kXchg;  // the team's first warp
}

// One table entry per (plane, 2D level, line set, segment): the factor fields of trifac_store,
// then eL and eR (kWK x 32 each, field-major like the factors), then mv and mu.
constexpr int kWEntry = trifac_fields<double, kWK>() * 32 + 2 * kWK * 32 + 4 * kMaxSeg;

template <class C>
__device__ __forceinline__ void wfac_store(C *e, const WideFac<C> &wf, int lane) {
    trifac_store<C, kWK>(e, wf.f, lane);
    C *p = e + trifac_fields<C, kWK>() * 32;
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        p[j * 32 + lane] = wf.eL[j];
        p[(kWK + j) * 32 + lane] = wf.eR[j];
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 2 * kMaxSeg; ++q) {
            p[2 * kWK * 32 + q] = wf.mv[q];
            p[2 * kWK * 32 + 2 * kMaxSeg + q] = wf.mu[q];
        }
    }
}

template <class C>
__device__ __forceinline__ void wfac_load(WideFac<C> &wf, const C *e, int lane) {
    trifac_load<C, kWK>(wf.f, e, lane);
    const C *p = e + trifac_fields<C, kWK>() * 32;
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        wf.eL[j] = p[j * 32 + lane];
        wf.eR[j] = p[(kWK + j) * 32 + lane];
    }
#pragma unroll
    for (int q = 0; q < 2 * kMaxSeg; ++q) {
        wf.mv[q] = p[2 * kWK * 32 + q];
        wf.mu[q] = p[2 * kWK * 32 + 2 * kMaxSeg + q];
    }
}

// The line matrix (diagonal, off-diagonal) of a line with coefficient row cr.
template <class C>
__device__ __forceinline__ void line_matrix(const CoefRow<C> &cr, C &dg, C &of) {
    dg = C(2) * cr.s[1] + cr.t[1];
    of = -cr.s[1];
}

// Make wf hold the solver data of (dg, of): the segment factors, eL, eR and the two rows of the
// reduced system's inverse.  Every warp of the team calls this with the same (dg, of), so every
// warp takes the same branch below (the table's entries of one (level, set) share (dg, of)).
template <class C>
__device__ __forceinline__ void ensure_wfac(const WideCtx<C> &c, WideFac<C> &wf, C dg, C of, int &xp, int lane,
                                            int m = -1) {
    if (wf.f.dg == dg && wf.f.of == of) return;
    if (c.ftab != nullptr && m >= 0) {
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            const C *e = c.ftab + (static_cast<long long>(2 * m + set) * c.W + c.seg) * kWEntry;
            if (e[0] == dg && e[32] == of) {  // fields 0 and 1 hold the matrix (lane 0's copy)
                wfac_load<C>(wf, e, lane);
                return;
            }
        }
    }
    // the factors through the one out-of-line body (also for 8 FP32 rows per lane, which the
    // inlined form would compile differently inside the table kernel and inside the cycle), so
    // that a table entry holds the bits the cycle would form.  Formed into a copy where wf then
    // stays in registers (FP64; 8 FP32 rows per lane); with 16 FP32 rows per lane wf is left
    // in local memory, which measured faster than the spills of a register-resident copy.
    if constexpr (kWfRegs<C>()) {
        TriFac<C, kWK> tf;
        tri_factor_call<C, kWK>(tf, dg, of, c.ns, lane);
        wf.f = tf;
    } else {
        tri_factor_call<C, kWK>(wf.f, dg, of, c.ns, lane);
    }
    const int il = c.ns - 1;
    {
        C e[1][kWK];
#pragma unroll
        for (int j = 0; j < kWK; ++j) e[0][j] = (lane == 0 && j == 0) ? C(1) : C(0);
        tri_apply<C, kWK, 1>(wf.f, e, c.ns, lane);
#pragma unroll
        for (int j = 0; j < kWK; ++j) wf.eL[j] = e[0][j];
#pragma unroll
        for (int j = 0; j < kWK; ++j) e[0][j] = (lane * kWK + j == il) ? C(1) : C(0);
        tri_apply<C, kWK, 1>(wf.f, e, c.ns, lane);
#pragma unroll
        for (int j = 0; j < kWK; ++j) wf.eR[j] = e[0][j];
    }
    C ends[4];
    ends[0] = __shfl_sync(0xffffffffu, wf.eL[0], 0);
    ends[1] = seg_value(wf.eL, il);
    ends[2] = __shfl_sync(0xffffffffu, wf.eR[0], 0);
    ends[3] = seg_value(wf.eR, il);
    const C *xb = exchange(c, xp, ends, 4, lane);
    // M (2W x 2W, padded with identity to 2 kMaxSeg), unknowns (u_0, v_0, u_1, v_1, ...)
    constexpr int N = 2 * kMaxSeg;
    C M[N][N], I[N][N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            M[r][q] = (r == q) ? C(1) : C(0);
            I[r][q] = (r == q) ? C(1) : C(0);
        }
#pragma unroll
    for (int s = 0; s < kMaxSeg; ++s) {
        if (s >= c.W) break;
        const C *e = xb + s * kXchg;
        if (s > 0) {
            M[2 * s][2 * s - 1] = of * e[0];
            M[2 * s + 1][2 * s - 1] = of * e[1];
        }
        if (s + 1 < c.W) {
            M[2 * s][2 * s + 2] = of * e[2];
            M[2 * s + 1][2 * s + 2] = of * e[3];
        }
    }
    // Gauss-Jordan without pivoting (M is I plus small couplings: diagonally dominant)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const C p = recip(M[k][k]);
#pragma unroll
        for (int q = 0; q < N; ++q) {
            M[k][q] *= p;
            I[k][q] *= p;
        }
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == k) continue;
            const C f = M[r][k];
#pragma unroll
            for (int q = 0; q < N; ++q) {
                M[r][q] = fma(-f, M[k][q], M[r][q]);
                I[r][q] = fma(-f, I[k][q], I[r][q]);
            }
        }
    }
    const int rv = 2 * c.seg - 1, ru = 2 * c.seg + 2;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        C a = C(0), b = C(0);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == rv) a = I[r][q];
            if (r == ru) b = I[r][q];
        }
        wf.mv[q] = (c.seg > 0) ? a : C(0);
        wf.mu[q] = (c.seg + 1 < c.W) ? b : C(0);
    }
}

// x = T^{-1} d for the team's line (this warp's segment of d in, of x out).
template <class C>
__device__ __forceinline__ void wide_solve(const WideCtx<C> &c, const WideFac<C> &wf, C (&d)[1][kWK], int &xp,
                                           int lane) {
    tri_apply<C, kWK, 1>(wf.f, d, c.ns, lane);
    C ends[2];
    ends[0] = __shfl_sync(0xffffffffu, d[0][0], 0);
    ends[1] = seg_value(d[0], c.ns - 1);
    const C *xb = exchange(c, xp, ends, 2, lane);
    C vprev = C(0), unext = C(0);
#pragma unroll
    for (int s = 0; s < kMaxSeg; ++s) {
        if (s >= c.W) break;
        const C y0 = xb[s * kXchg], yl = xb[s * kXchg + 1];
        vprev = fma(wf.mv[2 * s], y0, fma(wf.mv[2 * s + 1], yl, vprev));
        unext = fma(wf.mu[2 * s], y0, fma(wf.mu[2 * s + 1], yl, unext));
    }
    const C al = -wf.f.of * vprev, ar = -wf.f.of * unext;
#pragma unroll
    for (int j = 0; j < kWK; ++j) d[0][j] = fma(al, wf.eL[j], fma(ar, wf.eR[j], d[0][j]));
}

// Exact relaxation of line y of 2D level m by the team (see relax_group in plane_relax.cuh for
// the modes).
template <class S, class C>
__device__ __forceinline__ void wide_relax_line(const WideCtx<C> &c, WideFac<C> &wf, int m, int y, S *plane,
                                                bool accumulate, int nbmode, int out, int &xp, int lane) {
    const int nym = c.ny[m];
    C d[1][kWK];
    const CoefRow<C> cr = coef_row<C>(c.sm + (c.lb[m] + y) * kCoefPerLine);
    wload(d[0], wline_g(c, m, y), c, lane);
    if (nbmode != NB_NONE) {
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const int yy = y + s;
            if (yy < 0 || yy >= nym) continue;
            C v[kWK], hl, hr;
            wload_nb(v, hl, hr, c, m, yy, nbmode == NB_CORR, lane);
            sub_coupling_h(d[0], v, cr.s[1 + s], cr.t[1 + s], hl, hr, lane);
        }
        if (!c.vec) {
#pragma unroll
            for (int j = 0; j < kWK; ++j)
                if (lane * kWK + j >= c.ns) d[0][j] = C(0);
        }
    }
    C dg, of;
    line_matrix<C>(cr, dg, of);
    ensure_wfac(c, wf, dg, of, xp, lane, m);
    wide_solve(c, wf, d, xp, lane);
    if (out != OUT_PLANE) wstore(wline_u(c, m, y), d[0], c, lane);
    if (out != OUT_U) {
        S *p = plane + static_cast<long long>(y) * c.nx + c.x0;
        bool done = false;
        if constexpr (vec_chunk<S, kWK>() != 0) {
            if (c.vec) {
                S sv[kWK];
                if (accumulate) {
                    vload<S, kWK>(sv, p + lane * kWK);
#pragma unroll
                    for (int j = 0; j < kWK; ++j) stv<S, C>(&sv[j], ldv<C>(&sv[j]) + d[0][j]);
                } else {
#pragma unroll
                    for (int j = 0; j < kWK; ++j) stv<S, C>(&sv[j], d[0][j]);
                }
                vstore<S, kWK>(p + lane * kWK, sv);
                done = true;
            }
        }
        if (!done) {
#pragma unroll
            for (int j = 0; j < kWK; ++j) {
                const int x = lane * kWK + j;
                if (x < c.ns) {
                    const C v = accumulate ? ldv<C>(p + x) + d[0][j] : d[0][j];
                    stv<S, C>(p + x, v);
                }
            }
        }
    }
}

// g_{m+1}[j] from the odd lines 2j-1, 2j+1, 2j+3 of level m (restrict_combine of
// plane_relax.cuh with the segment's x-halo).
template <class C>
__device__ __forceinline__ void wide_restrict_line(const WideCtx<C> &c, int m, int jc, int lane) {
    const int nym = c.ny[m], e0 = 2 * jc;
    const bool ha = e0 >= 1, h1 = e0 + 2 < nym, hc = e0 + 3 < nym;
    const CoefRow<C> c0 = coef_row<C>(c.sm + (c.lb[m] + e0) * kCoefPerLine);
    const CoefRow<C> c1 = coef_row<C>(c.sm + (c.lb[m] + (h1 ? e0 + 2 : e0)) * kCoefPerLine);
    C acc[kWK];
#pragma unroll
    for (int q = 0; q < kWK; ++q) acc[q] = C(0);
    const C w0 = c0.wp;
    C v[kWK], hl, hr;
    if (ha) {
        wload_nb(v, hl, hr, c, m, e0 - 1, false, lane);
        sub_coupling_h(acc, v, w0 * c0.s[0], w0 * c0.t[0], hl, hr, lane);
    }
    C sb = w0 * c0.s[2], tb = w0 * c0.t[2], w1 = C(0);
    if (h1) {
        w1 = c1.wm;
        sb = fma(w1, c1.s[0], sb);
        tb = fma(w1, c1.t[0], tb);
    }
    wload_nb(v, hl, hr, c, m, e0 + 1, false, lane);
    sub_coupling_h(acc, v, sb, tb, hl, hr, lane);
    if (h1 && hc) {
        wload_nb(v, hl, hr, c, m, e0 + 3, false, lane);
        sub_coupling_h(acc, v, w1 * c1.s[2], w1 * c1.t[2], hl, hr, lane);
    }
    wstore(wline_g(c, m + 1, jc), acc, c, lane);
}

// d -= M (4c - c_{x-1} - c_{x+1} - c_{y-1} - c_{y+1}) + Kc c for plane pl at line y.
template <class C, class S>
__device__ __forceinline__ void wide_sub_plane_term(C (&d)[kWK], const S *pl, int y, int ny, C Mc, C Kc,
                                                    const WideCtx<C> &c, int lane) {
    C cv[kWK], up[kWK], dn[kWK];
    wload_plane<C, S>(cv, pl, y, c, lane);
#pragma unroll
    for (int j = 0; j < kWK; ++j) { up[j] = C(0); dn[j] = C(0); }
    if (y > 0) wload_plane<C, S>(up, pl, y - 1, c, lane);
    if (y + 1 < ny) wload_plane<C, S>(dn, pl, y + 1, c, lane);
    const S *row = pl + static_cast<long long>(y) * c.nx;
    C vl = __shfl_up_sync(0xffffffffu, cv[kWK - 1], 1);
    C vr = __shfl_down_sync(0xffffffffu, cv[0], 1);
    if (lane == 0) vl = (c.x0 > 0) ? ldv<C>(row + c.x0 - 1) : C(0);
    if (lane == 31) vr = (c.x0 + kSeg < c.nx) ? ldv<C>(row + c.x0 + kSeg) : C(0);
#pragma unroll
    for (int j = 0; j < kWK; ++j) {
        const C left = (j == 0) ? vl : cv[j - 1];
        const C right = (j == kWK - 1) ? vr : cv[j + 1];
        d[j] -= Mc * (C(4) * cv[j] - left - right - up[j] - dn[j]) + Kc * cv[j];
    }
}

// g_0 line y = f_z - sum_dz A_{z,z+dz} u_{z+dz} (mode 1: own plane zero; mode 2: all).
template <class S, class C>
__device__ __forceinline__ void wide_rhs_line(const PlaneRelaxArgs &a, const WideCtx<C> &c, int y, int mode,
                                              const S *fpl, const S *ub, int z, const C *zc, int lane) {
    const long long np = static_cast<long long>(a.nx) * a.ny;
    C d[kWK];
    wload_plane<C, S>(d, fpl, y, c, lane);
    if (mode >= 1 && z > 0) wide_sub_plane_term<C, S>(d, ub + (z - 1) * np, y, a.ny, zc[0], zc[3], c, lane);
    if (mode >= 1 && z + 1 < a.nz) wide_sub_plane_term<C, S>(d, ub + (z + 1) * np, y, a.ny, zc[2], zc[5], c, lane);
    if (mode == 2) wide_sub_plane_term<C, S>(d, ub + z * np, y, a.ny, zc[1], zc[4], c, lane);
    wstore(wline_g(c, 0, y), d, c, lane);
}

// One CTA (CL = false) or one cluster of a.R CTAs (CL = true) per plane of the colour; blockIdx.y
// is the batch entry.
template <class S, class C, bool CL>
__global__ void __launch_bounds__(wide_threads<C>(), 1) plane_wide_kernel(const __grid_constant__ PlaneRelaxArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) C s_xb[2 * 16 * kXchg];
    __shared__ int s_ny[kMaxPlaneLevels], s_lb[kMaxPlaneLevels], s_uon[kMaxPlaneLevels], s_gon[kMaxPlaneLevels];
    __shared__ C *s_ub[kMaxPlaneLevels], *s_gb[kMaxPlaneLevels];
    pdl_trigger();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    int pidx, rank;
    if constexpr (CL) {
        rank = static_cast<int>(cg::this_cluster().block_rank());
        pidx = static_cast<int>(blockIdx.x) / a.R;
    } else {
        rank = 0;
        pidx = static_cast<int>(blockIdx.x);
    }
    const int b = static_cast<int>(blockIdx.y);
    const long long slot = CL ? static_cast<long long>(blockIdx.y) * (gridDim.x / a.R) + pidx
                              : static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
    auto step_sync = [&]() {
        if constexpr (CL) cg::this_cluster().sync();
        else __syncthreads();
    };
    WideCtx<C> c;
    c.sm = reinterpret_cast<C *>(smem_raw);
    c.gw = reinterpret_cast<C *>(a.gws) + slot * a.ws_per_plane;
    c.g0 = nullptr;
    c.nx = a.nx;
    c.W = a.W;
    c.warp = warp;
    c.seg = warp % a.W;
    c.team = warp / a.W;
    c.nteam = nw / a.W;
    c.x0 = c.seg * kSeg;
    c.ns = min(kSeg, a.nx - c.x0);
    c.vec = a.vec != 0 && c.ns == kSeg;
    c.xb = s_xb;
    c.R = CL ? a.R : 1;
    c.lr = CL ? __ffs(a.R) - 1 : 0;
    c.rank = rank;
    c.ftab = nullptr;
    if (a.wftab != nullptr) {  // a table of the compute type C (the host passes the matching one)
        const int zp = a.colour + 2 * pidx;  // the plane's index in its z-level
        const int slot = (a.wfslot != nullptr) ? a.wfslot[zp] : zp;
        c.ftab = static_cast<const C *>(a.wftab) + static_cast<long long>(slot) * 2 * a.P * a.W * kWEntry;
    }
    const bool active = c.team < c.nteam;
    if (tid < a.P) {
        s_ny[tid] = a.ny_m[tid];
        s_lb[tid] = a.line_base[tid];
        s_uon[tid] = static_cast<int>((a.smem_u_mask >> tid) & 1u);
        s_gon[tid] = static_cast<int>((a.smem_g_mask >> tid) & 1u);
        s_ub[tid] = (s_uon[tid] ? c.sm : c.gw) + a.off_u[tid];
        s_gb[tid] = (s_gon[tid] ? c.sm : c.gw) + a.off_g[tid];
    }
    c.ny = s_ny;
    c.lb = s_lb;
    c.ub = s_ub;
    c.gb = s_gb;
    c.uon = s_uon;
    c.gon = s_gon;
    const int nx = a.nx, ny = a.ny;
    const long long np = static_cast<long long>(nx) * ny;
    const int z = a.colour + 2 * pidx;
    const S *fb = reinterpret_cast<const S *>(a.f) + static_cast<long long>(b) * a.vstride;
    S *ub = reinterpret_cast<S *>(a.u) + static_cast<long long>(b) * a.vstride;
    S *plane = ub + static_cast<long long>(z) * np;
    const C *zc = coef_table<C>(a.zcoef, a.zcoef32) + static_cast<long long>(z) * kCoefPerPlane;
    {
        const C *pc = coef_table<C>(a.pcoef, a.pcoef32) + static_cast<long long>(z) * a.sum_ny * kCoefPerLine;
        for (int i = tid; i < a.sum_ny * kCoefPerLine; i += nt) c.sm[i] = pc[i];
    }
    __syncthreads();
    pdl_wait();
    step_sync();  // (cluster) every CTA's level table and shared memory are set up
    SMG_TRACE(0);
    WideFac<C> wf;
    wf.f.dg = C(0);  // no real line matrix has a zero diagonal: the first line always factors
    wf.f.of = C(0);
    int xp = 0;
    const int P = a.P;
    const bool fuse = a.lean != 0 && P > 1;  // the shortened step order (4P - 3 steps)
    for (int it = 0; it < a.iters; ++it) {
        const int mode = (it == 0) ? a.mode : 2;
        const S *fpl = fb + static_cast<long long>(z) * np;
        c.g0 = nullptr;
        if constexpr (std::is_same<S, C>::value) {
            if (mode == 0) c.g0 = const_cast<C *>(reinterpret_cast<const C *>(fpl));
        }
        const bool acc = (mode == 2);
        const bool rhs = (c.g0 == nullptr);
        // step -1 forms the right-hand side of level 0 (where the plane of f is not used
        // directly); then the 2D cycle's steps in the order of plane_task (plane_relax.cuh):
        // down-sweep steps (even lines, odd lines, restriction per level, then the coarsest
        // level's lines) and up-sweep steps (odd lines with the coarse correction, even lines per
        // level).  In the shortened order every step that fills a level's right-hand side (step
        // -1, each restriction) also solves that level's even lines, which start from zero and
        // read no coupling.
        const int down = fuse ? 2 * (P - 1) : 3 * (P - 1) + 1;
        const int nsteps = (P == 1) ? 1 : down + 2 * (P - 1);
        for (int st = -1; st < nsteps; ++st) {
            int m = 0, colour = 0, nbmode = NB_NONE, out = OUT_U;
            bool accu = false, solve = true;
            int pre = 0;  // 1: the right-hand side of each listed line, 2: its restriction
            if (st < 0) {
                pre = rhs ? 1 : 0;
                solve = fuse;
            } else if (P == 1) {
                out = OUT_PLANE, accu = acc;
            } else if (st < down) {
                if (fuse) {
                    m = (st >> 1) + (st & 1);
                    if (st & 1) pre = 2;
                    else colour = 1, nbmode = NB_PLAIN;
                } else if (st < 3 * (P - 1)) {
                    m = st / 3;
                    const int k = st - 3 * m;
                    if (k == 2) {
                        m += 1, pre = 2, solve = false;
                    } else {
                        colour = k;
                        nbmode = (k == 0) ? NB_NONE : NB_PLAIN;
                    }
                } else {
                    m = P - 1;
                }
            } else {
                const int u = st - down;
                m = P - 2 - u / 2;
                colour = (u & 1) ? 0 : 1;
                nbmode = colour ? NB_CORR : NB_PLAIN;
                out = (m > 0) ? OUT_U : (colour ? OUT_U_AND_PLANE : OUT_PLANE);
                accu = acc;
            }
            if (active && (pre != 0 || solve)) {
                // a filling step lists every owned line of level m (even ones first) and solves
                // the even ones; a relaxation lists the owned lines of its colour (line
                // colour + 2i belongs to CTA i mod R)
                const int n = c.ny[m];
                for (int i = c.team;; i += c.nteam) {
                    bool even = true;
                    const int y = pre ? fused_line(c, i, n, even) : colour + 2 * (c.rank + (i << c.lr));
                    if (y >= n) break;
                    if (pre == 1) wide_rhs_line<S, C>(a, c, y, mode, fpl, ub, z, zc, lane);
                    else if (pre == 2) wide_restrict_line<C>(c, m - 1, y, lane);
                    if (solve && even) wide_relax_line<S, C>(c, wf, m, y, plane, accu, nbmode, out, xp, lane);
                }
            }
            step_sync();
            SMG_TRACE(st + 2);
        }
    }
}

// The solver data of one (plane, 2D level m, line set) for all W segments: one warp per segment,
// the same ensure_wfac as inside the plane cycle.  Grid (slots, 2P), W warps per CTA.
struct WideFactorArgs {
    int nx, W, P, sum_ny;
    int ny_m[kMaxPlaneLevels];
    int line_base[kMaxPlaneLevels];
    const int *planes;    // the plane of each slot (null: slot s is plane s)
    const double *pcoef;  // the planes' coefficient tables (sum_ny lines x kCoefPerLine each)
    const float *pcoef32; // the same rounded to FP32
    void *tab;            // out: 2P W kWEntry values of the compute type per slot
};

template <class C>
__global__ void wide_factor_kernel(const __grid_constant__ WideFactorArgs a) {
    __shared__ __align__(16) C s_xb[2 * 16 * kXchg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = blockIdx.x, pair = blockIdx.y, m = pair >> 1, set = pair & 1;
    const int p = (a.planes != nullptr) ? a.planes[slot] : slot;
    WideCtx<C> c;
    c.sm = nullptr;
    c.gw = nullptr;
    c.g0 = nullptr;
    c.nx = a.nx;
    c.W = a.W;
    c.warp = warp;
    c.seg = warp;
    c.team = 0;
    c.nteam = 1;
    c.x0 = c.seg * kSeg;
    c.ns = min(kSeg, a.nx - c.x0);
    c.vec = false;
    c.ny = nullptr;
    c.lb = nullptr;
    c.ub = nullptr;
    c.gb = nullptr;
    c.uon = nullptr;
    c.gon = nullptr;
    c.R = 1;
    c.lr = 0;
    c.rank = 0;
    c.xb = s_xb;
    c.ftab = nullptr;
    const int y = set ? a.ny_m[m] - 1 : 0;
    const CoefRow<C> cr = coef_row<C>(coef_table<C>(a.pcoef, a.pcoef32) +
                                      (static_cast<long long>(p) * a.sum_ny + a.line_base[m] + y) * kCoefPerLine);
    C dg, of;
    line_matrix<C>(cr, dg, of);
    WideFac<C> wf;
    wf.f.dg = C(0);
    wf.f.of = C(0);
    int xp = 0;
    ensure_wfac<C>(c, wf, dg, of, xp, lane);
    wfac_store<C>(static_cast<C *>(a.tab) + ((static_cast<long long>(slot) * 2 * a.P + pair) * a.W + c.seg) * kWEntry,
                  wf, lane);
}

template <class S, class C>
cudaError_t launch_wide(int nplanes, int nb, int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    threads = std::min(threads, wide_threads<C>());
    if (a.R <= 1) return launch_pdl(plane_wide_kernel<S, C, false>, dim3(nplanes, nb), dim3(threads), smem, st, a);
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
    return cudaLaunchKernelEx(&cfg, plane_wide_kernel<S, C, true>, a);
}

template <class S, class C>
int wide_smem_attr(bool cl, size_t smem) {
    if (!cl)
        return static_cast<int>(raise_smem_attr(reinterpret_cast<const void *>(&plane_wide_kernel<S, C, false>), smem));
    cudaError_t e = raise_smem_attr(reinterpret_cast<const void *>(&plane_wide_kernel<S, C, true>), smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(plane_wide_kernel<S, C, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return static_cast<int>(e);
}

template <class S, class C>
bool wide_resident(int R, int threads, size_t smem) {
    threads = std::min(threads, wide_threads<C>());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, plane_wide_kernel<S, C, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

}  // namespace

#define SMG_WCAT(a, b) a##b
#define SMG_WCAT2(a, b) SMG_WCAT(a, b)
#define SMG_WNAME(base) SMG_WCAT2(base##_w, SMG_WK)

long long SMG_WNAME(wide_factor_values)(int P, int W) { return 2LL * P * W * kWEntry; }

cudaError_t SMG_WNAME(launch_wide_factor_table)(int nx, int W, int P, int sum_ny, const int *ny_m, const int *line_base,
                                     int nslots, const int *planes, const double *pcoef, const float *pcoef32,
                                     bool f64, void *tab, cudaStream_t st) {
    if (W < 2 || W > kMaxSeg || P < 1 || P > kMaxPlaneLevels || nslots < 1) return cudaErrorInvalidValue;
    WideFactorArgs a;
    a.nx = nx;
    a.W = W;
    a.P = P;
    a.sum_ny = sum_ny;
    for (int m = 0; m < kMaxPlaneLevels; ++m) {
        a.ny_m[m] = m < P ? ny_m[m] : 0;
        a.line_base[m] = m < P ? line_base[m] : 0;
    }
    a.planes = planes;
    a.pcoef = pcoef;
    a.pcoef32 = pcoef32;
    a.tab = tab;
    if (f64) wide_factor_kernel<double><<<dim3(nslots, 2 * P), 32 * W, 0, st>>>(a);
    else wide_factor_kernel<float><<<dim3(nslots, 2 * P), 32 * W, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t SMG_WNAME(launch_plane_wide)(Prec storage, bool f64, int nplanes, int nb, int threads, const PlaneRelaxArgs &a,
                              size_t smem, cudaStream_t st) {
    if (a.W < 2 || a.W > kMaxSeg || threads / 32 < a.W || threads > 512 || a.R < 1 || a.R > 16 || (a.R & (a.R - 1)))
        return cudaErrorInvalidValue;
    switch (storage) {
    case Prec::F64: return launch_wide<double, double>(nplanes, nb, threads, a, smem, st);
    case Prec::F32:
        return f64 ? launch_wide<float, double>(nplanes, nb, threads, a, smem, st)
                   : launch_wide<float, float>(nplanes, nb, threads, a, smem, st);
    case Prec::BF16:
        return f64 ? launch_wide<__nv_bfloat16, double>(nplanes, nb, threads, a, smem, st)
                   : launch_wide<__nv_bfloat16, float>(nplanes, nb, threads, a, smem, st);
    }
    return cudaErrorInvalidValue;
}

int SMG_WNAME(set_plane_wide_smem)(Prec storage, bool f64, bool cl, size_t smem) {
    switch (storage) {
    case Prec::F64: return wide_smem_attr<double, double>(cl, smem);
    case Prec::F32: return f64 ? wide_smem_attr<float, double>(cl, smem) : wide_smem_attr<float, float>(cl, smem);
    case Prec::BF16:
        return f64 ? wide_smem_attr<__nv_bfloat16, double>(cl, smem) : wide_smem_attr<__nv_bfloat16, float>(cl, smem);
    }
    return static_cast<int>(cudaErrorInvalidValue);
}

bool SMG_WNAME(wide_cluster_resident)(Prec storage, bool f64, int R, int threads, size_t smem) {
    switch (storage) {
    case Prec::F64: return wide_resident<double, double>(R, threads, smem);
    case Prec::F32: return f64 ? wide_resident<float, double>(R, threads, smem) : wide_resident<float, float>(R, threads, smem);
    case Prec::BF16:
        return f64 ? wide_resident<__nv_bfloat16, double>(R, threads, smem)
                   : wide_resident<__nv_bfloat16, float>(R, threads, smem);
    }
    return false;
}

}  // namespace smg
