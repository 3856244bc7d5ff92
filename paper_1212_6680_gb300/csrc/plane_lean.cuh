// plane_lean.cuh -- the plane relaxation of one z-plane by one CTA (or one thread-block cluster),
// with the 2D cycle's dependent steps shortened (section "Preconditioning with SMG" of
// arXiv:1212.6680: plane relaxation as the smoother of the SMG V-cycle).
//
// It computes what plane_task<S, C, K, CL> (plane_relax.cuh) computes -- the same line solves on
// the same right-hand sides, with the same operations in the same order -- but it regroups the
// work into fewer barrier-separated steps.  Every line solve of the cycle depends on lines that
// other warps produce, so each step ends in a barrier (CTA-wide, or cluster-wide when the plane
// is spread over a cluster), and on GB300 each step costs about a thousand cycles whatever
// little work it holds.  Two regroupings cut the number of steps from 5P - 3 to 4P - 3 (P 2D
// levels):
//   * the plane's right-hand side is assembled line by line, and the warp that assembles an even
//     line solves it at once (going down, even lines of level 0 have zero neighbours);
//   * the warp that restricts coarse line j of level m+1 solves it at once when j is even (even
//     lines of level m+1 going down also have zero neighbours), so the restriction and the next
//     level's even-line relaxation are one step.
// The step list (P >= 2):
//   S0            right-hand side g_0 of every line; even lines of level 0 solved
//   m = 0..P-2:   odd lines of level m;  restriction to level m+1 with its even lines solved
//                 (the single line of level P-1 is solved in the last restriction step)
//   m = P-2..0:   odd lines of level m (neighbours + coarse correction);  even lines of level m
// Level 0 writes the plane (accumulating in correction form).  Per-level addresses, sizes and
// factor sets are read from a table in shared memory built once per CTA; a line uses its level's
// interior factor set, or the last line's set for y = ny_m - 1 (the host only launches this
// kernel when every line's matrix equals the set it is given).
//
// With a cluster of R CTAs (CL = true) line y of a level kept on chip belongs to CTA
// ((y/2) mod R), stored there at local line ((y/2) div R)*2 + (y mod 2) (the layout of
// plan_plane_layout_cluster); a CTA relaxes, restricts and assembles only the lines (pairs) it
// owns and reads the others' lines through distributed shared memory.  The coarse levels from
// a.solo_from on belong whole to CTA 0 (line y at local line y): the steps that touch only those
// levels run on CTA 0 alone and end in a CTA barrier instead of a cluster barrier; the other CTAs
// wait at the next cluster barrier.
#pragma once

#include "plane_relax.cuh"

namespace smg {

// One 2D level, as the steps read it.
template <class C>
struct LeanLevel {
    C *u;             // u_m lines (this CTA's shared memory, or the global slot)
    C *g;             // g_m lines
    const C *fs;      // the level's two factor sets (interior lines, then the last line)
    int ny;           // lines
    int lb;           // first row of the level in the coefficient table
    int uon, gon;     // u_m / g_m: 0 in the global slot, 1 on chip (cluster addressing applies),
                      // 2 on chip with every line on CTA 0 (a solo level)
    int solo;         // the level belongs whole to CTA 0 of the cluster
};

template <class C, int K>
struct LeanEnv {
    const C *coef;          // the plane's coefficient table (shared memory)
    const LeanLevel<C> *lv; // [P] (shared memory)
    int nx;
    bool vec;               // nx == 32 K and every array 16-byte aligned
    int lane, warp, nw;
    int lr, rank;           // cluster size 2^lr and this CTA's rank (0, 0 without a cluster)
};

// Address of line y of an array at `base` (on chip or not).
template <class C, int K, bool CL>
__device__ __forceinline__ C *lean_line(const LeanEnv<C, K> &e, C *base, int on_chip, int y) {
    if constexpr (!CL) {
        return base + y * e.nx;
    } else {
        if (!on_chip) return base + y * e.nx;
        if (on_chip == 2) return cg::this_cluster().map_shared_rank(base + y * e.nx, 0);
        const int k = y >> 1;
        const int owner = k & ((1 << e.lr) - 1);
        const int local = ((k >> e.lr) << 1) + (y & 1);
        return cg::this_cluster().map_shared_rank(base + local * e.nx, owner);
    }
}

template <bool CL>
__device__ __forceinline__ void lean_sync() {
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
}

// Lines two at a time while a lane's share of two lines fits in 16 bytes, else one.
template <class C, int K>
constexpr int lean_pair() {
    return (sizeof(C) * K <= 16) ? 2 : 1;
}

// Make fac hold factor set `set` (0: interior lines, 1: last line) of level m.
template <class C, int K>
__device__ __forceinline__ void lean_fac(TriFac<C, K> &fac, int &key, const LeanLevel<C> &L, int m, int set, int lane) {
    const int k = 2 * m + set;
    if (key == k) return;
    trifac_load<C, K>(fac, L.fs + set * trifac_fields<C, K>() * 32, lane);
    key = k;
}

// Store a solved line: into u_m, into the plane (level 0, accumulating in correction form), or both.
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void lean_store(const LeanEnv<C, K> &e, const LeanLevel<C> &L, int y, const C (&d)[K],
                                           S *plane, bool acc, int out) {
    if (out != OUT_PLANE) store_line<C, K>(lean_line<C, K, CL>(e, L.u, L.uon, y), d, e.nx, e.vec, e.lane);
    if (out == OUT_U) return;
    S *p = plane + y * e.nx;
    if constexpr (vec_chunk<S, K>() != 0) {
        if (e.vec) {
            S sv[K];
            if (acc) {
                vload<S, K>(sv, p + e.lane * K);
#pragma unroll
                for (int j = 0; j < K; ++j) stv<S, C>(&sv[j], ldv<C>(&sv[j]) + d[j]);
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) stv<S, C>(&sv[j], d[j]);
            }
            vstore<S, K>(p + e.lane * K, sv);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = e.lane * K + j;
        if (x < e.nx) stv<S, C>(p + x, acc ? ldv<C>(p + x) + d[j] : d[j]);
    }
}

// Exact relaxation of NL lines ys[] of one colour of level m by one warp (lines of one colour do
// not couple to each other).  nbmode: the neighbouring lines are zero (NB_NONE), read
// (NB_PLAIN), or read with the coarse correction P u_{m+1} added (NB_CORR, the neighbours are
// even lines).
template <class S, class C, int K, bool CL, int NL>
__device__ __forceinline__ void lean_relax(const LeanEnv<C, K> &e, TriFac<C, K> &fac, int &key, int m,
                                           const int (&ys)[NL], int nbmode, int out, S *plane, bool acc) {
    const LeanLevel<C> L = e.lv[m];
    const int nx = e.nx, lane = e.lane;
    C d[NL][K];
    CoefRow<C> cr[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        cr[l] = coef_row<C>(e.coef + (L.lb + ys[l]) * kCoefPerLine);
        load_line<C, K>(d[l], lean_line<C, K, CL>(e, L.g, L.gon, ys[l]), nx, e.vec, lane);
    }
    if (nbmode != NB_NONE) {
        LeanLevel<C> Lc;
        Lc.u = nullptr;
        Lc.ny = 0;
        Lc.uon = 0;
        if (nbmode == NB_CORR) Lc = e.lv[m + 1];
        const int nyc = Lc.ny;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int y = ys[l];
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                const int yy = y + s;
                if (yy < 0 || yy >= L.ny) continue;
                C v[K];
                load_line<C, K>(v, lean_line<C, K, CL>(e, L.u, L.uon, yy), nx, e.vec, lane);
                if (nbmode == NB_CORR) {  // neighbour yy is an even line: add P e from level m+1
                    const CoefRow<C> cy = coef_row<C>(e.coef + (L.lb + yy) * kCoefPerLine);
                    const int jl = yy / 2 - 1, jh = yy / 2;
                    if (jl >= 0) {
                        C c[K];
                        load_line<C, K>(c, lean_line<C, K, CL>(e, Lc.u, Lc.uon, jl), nx, e.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fma(cy.wm, c[j], v[j]);
                    }
                    if (jh < nyc) {
                        C c[K];
                        load_line<C, K>(c, lean_line<C, K, CL>(e, Lc.u, Lc.uon, jh), nx, e.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fma(cy.wp, c[j], v[j]);
                    }
                }
                sub_coupling<C, K>(d[l], v, cr[l].s[1 + s], cr[l].t[1 + s], lane);
            }
            if (!e.vec) {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (lane * K + j >= nx) d[l][j] = C(0);
            }
        }
    }
    // every line of a group but the level's last shares the interior matrix
    const int set = (ys[NL - 1] == L.ny - 1) ? 1 : 0;
    if (NL == 1 || set == 0) {
        lean_fac<C, K>(fac, key, L, m, set, lane);
        tri_apply<C, K, NL>(fac, d, nx, lane);
    } else {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            lean_fac<C, K>(fac, key, L, m, ys[l] == L.ny - 1 ? 1 : 0, lane);
            C dl[1][K];
#pragma unroll
            for (int j = 0; j < K; ++j) dl[0][j] = d[l][j];
            tri_apply<C, K, 1>(fac, dl, nx, lane);
#pragma unroll
            for (int j = 0; j < K; ++j) d[l][j] = dl[0][j];
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) lean_store<S, C, K, CL>(e, L, ys[l], d[l], plane, acc, out);
}

// The lines of one colour of level m this CTA owns, colour + 2k with k = rank + R i, warp w
// taking i = w, w + nw, ...: two at a time while two are left (when a lane's share of two lines
// fits in 16 bytes), then one.
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void lean_colour(const LeanEnv<C, K> &e, TriFac<C, K> &fac, int &key, int m, int colour,
                                            int nbmode, int out, S *plane, bool acc) {
    const int nl = (e.lv[m].ny - colour + 1) / 2;
    const bool dist = CL && !e.lv[m].solo;  // lines spread over the cluster
    int nown = nl;
    if constexpr (CL) {
        if (dist) nown = (nl > e.rank) ? ((nl - e.rank + (1 << e.lr) - 1) >> e.lr) : 0;
        else if (e.rank != 0) nown = 0;
    }
    auto Y = [&](int i) { return dist ? colour + 2 * (e.rank + (i << e.lr)) : colour + 2 * i; };
    int i = e.warp;
    if constexpr (lean_pair<C, K>() == 2) {
        for (; i + e.nw < nown; i += 2 * e.nw) {
            const int ys[2] = {Y(i), Y(i + e.nw)};
            lean_relax<S, C, K, CL, 2>(e, fac, key, m, ys, nbmode, out, plane, acc);
        }
    }
    for (; i < nown; i += e.nw) {
        const int ys[1] = {Y(i)};
        lean_relax<S, C, K, CL, 1>(e, fac, key, m, ys, nbmode, out, plane, acc);
    }
}

// g_{m+1}[j] from the odd lines 2j-1, 2j+1, 2j+3 of level m (restrict_combine: the residual of
// level m after its down-sweep); the result stays in registers.
template <class C, int K, bool CL>
__device__ __forceinline__ void lean_restrict_line(const LeanEnv<C, K> &e, const LeanLevel<C> &L, int j, C (&acc)[K]) {
    const int nx = e.nx, lane = e.lane, e0 = 2 * j;
    const bool ha = e0 >= 1, h1 = e0 + 2 < L.ny, hc = e0 + 3 < L.ny;
    C va[K], vb[K], vc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) { va[q] = C(0); vc[q] = C(0); }
    if (ha) load_line<C, K>(va, lean_line<C, K, CL>(e, L.u, L.uon, e0 - 1), nx, e.vec, lane);
    load_line<C, K>(vb, lean_line<C, K, CL>(e, L.u, L.uon, e0 + 1), nx, e.vec, lane);
    if (hc) load_line<C, K>(vc, lean_line<C, K, CL>(e, L.u, L.uon, e0 + 3), nx, e.vec, lane);
    const CoefRow<C> c0 = coef_row<C>(e.coef + (L.lb + e0) * kCoefPerLine);
    const CoefRow<C> c1 = coef_row<C>(e.coef + (L.lb + (h1 ? e0 + 2 : e0)) * kCoefPerLine);
    restrict_combine<C, K>(acc, va, vb, vc, c0, c1, ha, h1, hc, lane);
}

// Restriction from level m to level m+1 over the coarse line pairs (2k, 2k+1) this CTA owns
// (k = rank + R i); every coarse line's g is stored, and the even one of the pair is solved at
// once (level m+1's down-sweep relaxes its even lines with zero neighbours).  While the CTA owns
// at most half as many pairs as it has warps, the two lines of a pair go to two warps (w takes
// the even line, w + nw/2 the odd one) so that neither waits for the other's restriction;
// otherwise warp w takes whole pairs i = w, w + nw, ...
template <class C, int K, bool CL>
__device__ __forceinline__ void lean_restrict_solve(const LeanEnv<C, K> &e, TriFac<C, K> &fac, int &key, int m) {
    const LeanLevel<C> L = e.lv[m], Lc = e.lv[m + 1];
    const int nx = e.nx, lane = e.lane;
    const int npairs = (Lc.ny + 1) / 2;
    const bool dist = CL && !Lc.solo;  // coarse line pairs spread over the cluster
    int nown = npairs;
    if constexpr (CL) {
        if (dist) nown = (npairs > e.rank) ? ((npairs - e.rank + (1 << e.lr) - 1) >> e.lr) : 0;
        else if (e.rank != 0) nown = 0;
    }
    const int half = e.nw >> 1;
    if (2 * nown <= e.nw) {
        const bool odd = e.warp >= half;
        const int i = odd ? e.warp - half : e.warp;
        if (i >= nown) return;
        const int k = dist ? e.rank + (i << e.lr) : i;
        const int j = 2 * k + (odd ? 1 : 0);
        if (j >= Lc.ny) return;
        C g[1][K];
        lean_restrict_line<C, K, CL>(e, L, j, g[0]);
        store_line<C, K>(lean_line<C, K, CL>(e, Lc.g, Lc.gon, j), g[0], nx, e.vec, lane);
        if (odd) return;
        lean_fac<C, K>(fac, key, Lc, m + 1, j == Lc.ny - 1 ? 1 : 0, lane);
        tri_apply<C, K, 1>(fac, g, nx, lane);
        store_line<C, K>(lean_line<C, K, CL>(e, Lc.u, Lc.uon, j), g[0], nx, e.vec, lane);
        return;
    }
    for (int i = e.warp; i < nown; i += e.nw) {
        const int k = dist ? e.rank + (i << e.lr) : i;
        const int j0 = 2 * k, j1 = 2 * k + 1;
        C g0[1][K], g1[K];
        lean_restrict_line<C, K, CL>(e, L, j0, g0[0]);
        if (j1 < Lc.ny) lean_restrict_line<C, K, CL>(e, L, j1, g1);
        store_line<C, K>(lean_line<C, K, CL>(e, Lc.g, Lc.gon, j0), g0[0], nx, e.vec, lane);
        if (j1 < Lc.ny) store_line<C, K>(lean_line<C, K, CL>(e, Lc.g, Lc.gon, j1), g1, nx, e.vec, lane);
        lean_fac<C, K>(fac, key, Lc, m + 1, j0 == Lc.ny - 1 ? 1 : 0, lane);
        tri_apply<C, K, 1>(fac, g0, nx, lane);
        store_line<C, K>(lean_line<C, K, CL>(e, Lc.u, Lc.uon, j0), g0[0], nx, e.vec, lane);
    }
}

// S0: the right-hand side g_0 = f_z - sum_dz A_{z,z+dz} u_{z+dz} of every line this CTA owns
// (mode 0: f_z; mode 1: the own plane is zero; mode 2: all terms), stored unless g_0 is f_z
// itself; even lines are solved at once (into u_0, or into the plane when the plane has a
// single line).  Lines in pairs (2k, 2k+1), k = rank + R i.
//
// d -= Mc (4 c - c_{x-1} - c_{x+1} - up - dn) + Kc c for one plane line c with its y-neighbours up
// and dn already loaded (the arithmetic of sub_plane_term).
template <class C, int K>
__device__ __forceinline__ void lean_plane_term(C (&d)[K], const C (&cv)[K], const C (&up)[K], const C (&dn)[K], C Mc,
                                                C Kc, int lane) {
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

// Lines y0 and y0 + 1 (when `two`) of g_0 = f_z - sum_dz A_{z,z+dz} u_{z+dz} (mode 1: own plane
// zero; mode 2: all).  Lines y0 - 1 .. y0 + 2 of each plane the pair needs are loaded once for both
// lines and before any arithmetic, so their latencies overlap; per line the terms are subtracted
// in the order of rhs_group (plane z-1, z+1, then z).
template <class C, class S, int K>
__device__ __forceinline__ void lean_rhs_pair(C (&d)[2][K], const S *fpl, const S *ub, int z, int nz, int y0, bool two,
                                              int ny, int nx, long long np, const C *zc, int mode, bool vec, int lane) {
    load_plane_line<C, S, K>(d[0], fpl, y0, nx, vec, lane);
    if (two) load_plane_line<C, S, K>(d[1], fpl, y0 + 1, nx, vec, lane);
    auto rows = [&](C (&r)[4][K], const S *pl) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int y = y0 - 1 + t;
            if (y >= 0 && y < ny && (t < 3 || two)) {
                load_plane_line<C, S, K>(r[t], pl, y, nx, vec, lane);
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) r[t][j] = C(0);
            }
        }
    };
    auto apply = [&](const C (&r)[4][K], C Mc, C Kc) {
        lean_plane_term<C, K>(d[0], r[1], r[0], r[2], Mc, Kc, lane);
        if (two) lean_plane_term<C, K>(d[1], r[2], r[1], r[3], Mc, Kc, lane);
    };
    const bool lo = mode >= 1 && z > 0, hi = mode >= 1 && z + 1 < nz;
    if (lo && hi) {
        C ra[4][K], rb[4][K];
        rows(ra, ub + (z - 1) * np);
        rows(rb, ub + (z + 1) * np);
        apply(ra, zc[0], zc[3]);
        apply(rb, zc[2], zc[5]);
    } else if (lo || hi) {
        C ra[4][K];
        rows(ra, ub + (lo ? z - 1 : z + 1) * np);
        if (lo) apply(ra, zc[0], zc[3]);
        else apply(ra, zc[2], zc[5]);
    }
    if (mode == 2) {
        C ra[4][K];
        rows(ra, ub + z * np);
        apply(ra, zc[1], zc[4]);
    }
}

template <class S, class C, int K, bool CL>
__device__ __forceinline__ void lean_rhs_even(const LeanEnv<C, K> &e, TriFac<C, K> &fac, int &key,
                                              const PlaneRelaxArgs &a, int mode, bool g0_is_f, const S *fpl,
                                              const S *ub, int z, const C *zc, S *plane, bool acc, int P) {
    const LeanLevel<C> L = e.lv[0];
    const int nx = a.nx, ny = a.ny, lane = e.lane;
    const long long np = static_cast<long long>(nx) * ny;
    const int npairs = (ny + 1) / 2;
    int nown = npairs;
    if constexpr (CL) nown = (npairs > e.rank) ? ((npairs - e.rank + (1 << e.lr) - 1) >> e.lr) : 0;
    for (int i = e.warp; i < nown; i += e.nw) {
        const int k = CL ? e.rank + (i << e.lr) : i;
        C d[2][K];
        if constexpr (sizeof(C) == 4 && sizeof(C) * K <= 16) {
            // FP32 with a lane's share of a line in at most 16 bytes (nx <= 128): the pair's plane lines
            // loaded together (with wider shares the extra registers spill, so the lines are
            // assembled one after the other there)
            const bool two = 2 * k + 1 < ny;
            lean_rhs_pair<C, S, K>(d, fpl, ub, z, a.nz, 2 * k, two, ny, nx, np, zc, mode, e.vec, lane);
            if (!g0_is_f) {
                store_line<C, K>(lean_line<C, K, CL>(e, L.g, L.gon, 2 * k), d[0], nx, e.vec, lane);
                if (two) store_line<C, K>(lean_line<C, K, CL>(e, L.g, L.gon, 2 * k + 1), d[1], nx, e.vec, lane);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int y = 2 * k + t;
                if (y >= ny) break;
                load_plane_line<C, S, K>(d[t], fpl, y, nx, e.vec, lane);
                if (mode >= 1 && z > 0)
                    sub_plane_term<C, S, K>(d[t], ub + (z - 1) * np, y, nx, ny, zc[0], zc[3], e.vec, lane);
                if (mode >= 1 && z + 1 < a.nz)
                    sub_plane_term<C, S, K>(d[t], ub + (z + 1) * np, y, nx, ny, zc[2], zc[5], e.vec, lane);
                if (mode == 2) sub_plane_term<C, S, K>(d[t], ub + z * np, y, nx, ny, zc[1], zc[4], e.vec, lane);
                if (!g0_is_f) store_line<C, K>(lean_line<C, K, CL>(e, L.g, L.gon, y), d[t], nx, e.vec, lane);
            }
        }
        C dv[1][K];
#pragma unroll
        for (int j = 0; j < K; ++j) dv[0][j] = d[0][j];
        lean_fac<C, K>(fac, key, L, 0, 2 * k == ny - 1 ? 1 : 0, lane);
        tri_apply<C, K, 1>(fac, dv, nx, lane);
        lean_store<S, C, K, CL>(e, L, 2 * k, dv[0], plane, acc, P == 1 ? OUT_PLANE : OUT_U);
    }
}

// The relaxation of the pidx-th plane of the colour (batch entry b) by one CTA (CL = false) or by
// this CTA's share of a cluster (CL = true, rank `rank`); `slot` selects the global workspace.
template <class S, class C, int K, bool CL>
__device__ __forceinline__ void plane_lean_task(const PlaneRelaxArgs &a, int pidx, int b, long long slot, int rank,
                                                unsigned char *smem_raw) {
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int nx = a.nx, ny = a.ny, P = a.P;
    const long long np = static_cast<long long>(nx) * ny;
    const int z = a.colour + 2 * pidx;
    const int tid = threadIdx.x, nt = blockDim.x;
    LeanEnv<C, K> e;
    e.lane = tid & 31;
    e.warp = tid >> 5;
    e.nw = nt >> 5;
    e.nx = nx;
    e.vec = a.vec != 0;
    e.coef = sm;
    e.rank = CL ? rank : 0;
    e.lr = CL ? __ffs(a.R) - 1 : 0;
    C *gw = reinterpret_cast<C *>(a.gws) + slot * a.ws_per_plane;
    const S *fb = reinterpret_cast<const S *>(a.f) + static_cast<long long>(b) * a.vstride;
    S *ub = reinterpret_cast<S *>(a.u) + static_cast<long long>(b) * a.vstride;
    S *plane = ub + static_cast<long long>(z) * np;
    const C *zc = coef_table<C>(a.zcoef, a.zcoef32) + static_cast<long long>(z) * kCoefPerPlane;
    __shared__ LeanLevel<C> s_lv[kMaxPlaneLevels];
    {
        const C *pc = coef_table<C>(a.pcoef, a.pcoef32) + static_cast<long long>(z) * a.sum_ny * kCoefPerLine;
        for (int i = tid; i < a.sum_ny * kCoefPerLine; i += nt) sm[i] = pc[i];
        if (tid < P) {
            LeanLevel<C> L;
            L.solo = (CL && tid >= a.solo_from) ? 1 : 0;
            L.uon = static_cast<int>((a.smem_u_mask >> tid) & 1u) * (L.solo ? 2 : 1);
            L.gon = static_cast<int>((a.smem_g_mask >> tid) & 1u) * (L.solo ? 2 : 1);
            L.u = (L.uon ? sm : gw) + a.off_u[tid];
            L.g = (L.gon ? sm : gw) + a.off_g[tid];
            L.fs = sm + a.off_fs + 2 * tid * trifac_fields<C, K>() * 32;
            L.ny = a.ny_m[tid];
            L.lb = a.line_base[tid];
            s_lv[tid] = L;
        }
    }
    e.lv = s_lv;
    TriFac<C, K> fac;
    __syncthreads();
    // the two factor sets of every 2D level (interior line, last line), by warps in parallel
    for (int sidx = e.warp; sidx < 2 * P; sidx += e.nw) {
        const int mm = sidx >> 1;
        const int y = (sidx & 1) ? a.ny_m[mm] - 1 : 0;
        const C *lc = sm + (a.line_base[mm] + y) * kCoefPerLine;
        tri_factor<C, K>(fac, C(2) * lc[1] + lc[4], -lc[1], nx, e.lane);
        trifac_store<C, K>(sm + a.off_fs + sidx * trifac_fields<C, K>() * 32, fac, e.lane);
    }
    // everything above reads only the hierarchy's tables (overlapping the previous kernel under
    // programmatic dependent launch); from here on the planes are read and written
    pdl_wait();
    lean_sync<CL>();
    SMG_TRACE(0);
    int key = -1;
    for (int it = 0; it < a.iters; ++it) {
        const int mode = (it == 0) ? a.mode : 2;
        const bool acc = (mode == 2);
        const S *fpl = fb + static_cast<long long>(z) * np;
        // g_0 is f_z itself for the first red sweep when f is in the compute precision (level 0's
        // table entry then points at f, in global memory); otherwise it is assembled into g_0
        bool g0_is_f = false;
        if constexpr (std::is_same<S, C>::value) g0_is_f = (mode == 0);
        if (tid == 0) {
            if (g0_is_f) {
                s_lv[0].g = const_cast<C *>(reinterpret_cast<const C *>(fpl));
                s_lv[0].gon = 0;
            } else {
                s_lv[0].gon = static_cast<int>(a.smem_g_mask & 1u);
                s_lv[0].g = (s_lv[0].gon ? sm : gw) + a.off_g[0];
            }
        }
        __syncthreads();
        lean_rhs_even<S, C, K, CL>(e, fac, key, a, mode, g0_is_f, fpl, ub, z, zc, plane, acc, P);
        lean_sync<CL>();
        SMG_TRACE(1);
        if (P == 1) continue;
        // a step runs on CTA 0 alone when the level it writes is solo (odd and even lines of level
        // m: m >= solo_from; restriction to level m+1: m+1 >= solo_from); the barrier between two
        // such steps is CTA 0's own
        const int sf = CL ? a.solo_from : P;
        auto step_sync = [&](bool solo_pair) {
            if constexpr (CL) {
                if (solo_pair) {
                    if (e.rank == 0) __syncthreads();
                    return;
                }
            }
            lean_sync<CL>();
        };
        for (int m = 0; m + 1 < P; ++m) {
            lean_colour<S, C, K, CL>(e, fac, key, m, 1, NB_PLAIN, OUT_U, plane, false);
            step_sync(m >= sf);  // odd(m) down -> restrict(m)
            SMG_TRACE(2 + 2 * m);
            lean_restrict_solve<C, K, CL>(e, fac, key, m);
            // restrict(m) runs on CTA 0 alone when level m+1 is solo; the next step is odd(m+1)
            // down, or odd(P-2) up after the last restriction
            step_sync(m + 1 < P - 1 ? m + 1 >= sf : m >= sf);
            SMG_TRACE(3 + 2 * m);
        }
        for (int m = P - 2; m >= 0; --m) {
            lean_colour<S, C, K, CL>(e, fac, key, m, 1, NB_CORR, m > 0 ? OUT_U : OUT_U_AND_PLANE, plane, acc);
            step_sync(m >= sf);  // odd(m) up -> even(m) up
            SMG_TRACE(2 * P + 2 * (P - 2 - m));
            lean_colour<S, C, K, CL>(e, fac, key, m, 0, NB_PLAIN, m > 0 ? OUT_U : OUT_PLANE, plane, acc);
            step_sync(m >= sf && m - 1 >= sf);  // even(m) up -> odd(m-1) up
            SMG_TRACE(2 * P + 1 + 2 * (P - 2 - m));
        }
    }
}

// One CTA (CL = false) or one cluster of R CTAs (CL = true) per plane of the colour; blockIdx.y
// is the batch entry.
// Threads of a shortened-step CTA: 512 for FP32 compute; 384 for FP64 compute, which leaves 168
// registers a thread for the FP64 line factors instead of spilling them (measured faster on the
// FP64 cycle and the FP64 coarsest plane; the cycle is bit-identical for any warp count).
template <class C>
constexpr int lean_threads() { return sizeof(C) == 8 ? 384 : 512; }

template <class S, class C, int K, bool CL>
__global__ void __launch_bounds__(lean_threads<C>(), 1) plane_lean_kernel(const __grid_constant__ PlaneRelaxArgs a) {
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
    const long long slot = CL ? static_cast<long long>(blockIdx.y) * (gridDim.x / a.R) + pidx
                              : static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
    plane_lean_task<S, C, K, CL>(a, pidx, static_cast<int>(blockIdx.y), slot, rank, smem_raw);
}

template <class S, class C, int K, bool CL>
cudaError_t launch_lean(int nplanes, int nb, int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    threads = std::min(threads, lean_threads<C>());
    if constexpr (!CL) {
        return launch_pdl(plane_lean_kernel<S, C, K, false>, dim3(nplanes, nb), dim3(threads), smem, st, a);
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
        return cudaLaunchKernelEx(&cfg, plane_lean_kernel<S, C, K, true>, a);
    }
}

template <class S, class C, int K, bool CL>
int set_lean_smem_attr(size_t smem) {
    cudaError_t e = raise_smem_attr(reinterpret_cast<const void *>(&plane_lean_kernel<S, C, K, CL>), smem);
    if (e == cudaSuccess && CL)
        e = cudaFuncSetAttribute(plane_lean_kernel<S, C, K, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return static_cast<int>(e);
}

template <class S, class C, int K>
bool lean_cluster_resident(int R, int threads, size_t smem) {
    threads = std::min(threads, lean_threads<C>());
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
    if (cudaOccupancyMaxActiveClusters(&n, plane_lean_kernel<S, C, K, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

}  // namespace smg
