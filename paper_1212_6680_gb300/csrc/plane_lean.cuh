// plane_lean.cuh -- the plane relaxation of one z-plane by one CTA in FP32 arithmetic, with the
// 2D cycle's dependent steps shortened (section "Preconditioning with SMG" of arXiv:1212.6680:
// plane relaxation as the smoother of the SMG V-cycle).
//
// It computes exactly what plane_task<S, float, K, false> (plane_relax.cuh) computes -- the same
// line solves on the same right-hand sides, with the same operations in the same order -- but it
// regroups the work into fewer barrier-separated steps.  Every line solve of the cycle depends
// on lines that other warps produce, so each step ends in a CTA barrier, and on GB300 each step
// costs about a thousand cycles whatever little work it holds.  Two regroupings cut the number
// of steps from 5P - 3 to 4P - 3 (P 2D levels):
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
#pragma once

#include "plane_relax.cuh"

namespace smg {

// One 2D level, as the steps read it.
struct LeanLevel {
    float *u;         // u_m lines (shared memory, or the CTA's global slot)
    float *g;         // g_m lines
    const float *fs;  // the level's two factor sets (interior lines, then the last line)
    int ny;           // lines
    int lb;           // first row of the level in the coefficient table
};

template <int K>
struct LeanEnv {
    const float *coef;    // the plane's coefficient table (shared memory)
    const LeanLevel *lv;  // [P] (shared memory)
    int nx;
    bool vec;             // nx == 32 K and every array 16-byte aligned
    int lane, warp, nw;
};

// Make fac hold factor set `set` (0: interior lines, 1: last line) of level m.
template <int K>
__device__ __forceinline__ void lean_fac(TriFac<float, K> &fac, int &key, const LeanLevel &L, int m, int set, int lane) {
    const int k = 2 * m + set;
    if (key == k) return;
    trifac_load<float, K>(fac, L.fs + set * trifac_fields<float, K>() * 32, lane);
    key = k;
}

// Store a solved line: into u_m, into the plane (level 0, accumulating in correction form), or both.
template <class S, int K>
__device__ __forceinline__ void lean_store(const LeanEnv<K> &e, const LeanLevel &L, int y, const float (&d)[K],
                                           S *plane, bool acc, int out) {
    if (out != OUT_PLANE) store_line<float, K>(L.u + y * e.nx, d, e.nx, e.vec, e.lane);
    if (out == OUT_U) return;
    S *p = plane + y * e.nx;
    if constexpr (vec_chunk<S, K>() != 0) {
        if (e.vec) {
            S sv[K];
            if (acc) {
                vload<S, K>(sv, p + e.lane * K);
#pragma unroll
                for (int j = 0; j < K; ++j) stv<S, float>(&sv[j], ldv<float>(&sv[j]) + d[j]);
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) stv<S, float>(&sv[j], d[j]);
            }
            vstore<S, K>(p + e.lane * K, sv);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = e.lane * K + j;
        if (x < e.nx) stv<S, float>(p + x, acc ? ldv<float>(p + x) + d[j] : d[j]);
    }
}

// Exact relaxation of NL lines ys[0 .. nvalid) of one colour of level m by one warp (entries past
// nvalid repeat a valid line: solved, not stored).  nbmode: neighbours zero (NB_NONE), read
// (NB_PLAIN), or read with the coarse correction of level m+1 added (NB_CORR).
template <class S, int K, int NL>
__device__ __forceinline__ void lean_relax(const LeanEnv<K> &e, TriFac<float, K> &fac, int &key, int m,
                                           const int (&ys)[NL], int nvalid, int nbmode, int out, S *plane, bool acc) {
    const LeanLevel L = e.lv[m];
    const int nx = e.nx, lane = e.lane;
    float d[NL][K];
    CoefRow<float> cr[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        cr[l] = coef_row<float>(e.coef + (L.lb + ys[l]) * kCoefPerLine);
        load_line<float, K>(d[l], L.g + ys[l] * nx, nx, e.vec, lane);
    }
    if (nbmode != NB_NONE) {
        LeanLevel Lc;
        Lc.u = nullptr;
        Lc.ny = 0;
        if (nbmode == NB_CORR) Lc = e.lv[m + 1];
        const int nyc = Lc.ny;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int y = ys[l];
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                const int yy = y + s;
                if (yy < 0 || yy >= L.ny) continue;
                float v[K];
                load_line<float, K>(v, L.u + yy * nx, nx, e.vec, lane);
                if (nbmode == NB_CORR) {  // neighbour yy is an even line: add P e from level m+1
                    const CoefRow<float> cy = coef_row<float>(e.coef + (L.lb + yy) * kCoefPerLine);
                    const int jl = yy / 2 - 1, jh = yy / 2;
                    if (jl >= 0) {
                        float c[K];
                        load_line<float, K>(c, Lc.u + jl * nx, nx, e.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fmaf(cy.wm, c[j], v[j]);
                    }
                    if (jh < nyc) {
                        float c[K];
                        load_line<float, K>(c, Lc.u + jh * nx, nx, e.vec, lane);
#pragma unroll
                        for (int j = 0; j < K; ++j) v[j] = fmaf(cy.wp, c[j], v[j]);
                    }
                }
                sub_coupling<float, K>(d[l], v, cr[l].s[1 + s], cr[l].t[1 + s], lane);
            }
            if (!e.vec) {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (lane * K + j >= nx) d[l][j] = 0.0f;
            }
        }
    }
    // every line of a group but the level's last shares the interior matrix
    const int set = (ys[NL - 1] == L.ny - 1) ? 1 : 0;
    if (NL == 1 || set == 0) {
        lean_fac<K>(fac, key, L, m, set, lane);
        tri_apply<float, K, NL>(fac, d, nx, lane);
    } else {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            lean_fac<K>(fac, key, L, m, ys[l] == L.ny - 1 ? 1 : 0, lane);
            float dl[1][K];
#pragma unroll
            for (int j = 0; j < K; ++j) dl[0][j] = d[l][j];
            tri_apply<float, K, 1>(fac, dl, nx, lane);
#pragma unroll
            for (int j = 0; j < K; ++j) d[l][j] = dl[0][j];
        }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (l >= nvalid) break;
        lean_store<S, K>(e, L, ys[l], d[l], plane, acc, out);
    }
}

// Lines of one colour of level m, warp w taking colour + 2(w + i nw): two at a time while two
// are left (a lane's share of a line is at most 16 bytes here), then one.
template <class S, int K>
__device__ __forceinline__ void lean_colour(const LeanEnv<K> &e, TriFac<float, K> &fac, int &key, int m, int colour,
                                            int nbmode, int out, S *plane, bool acc) {
    const int nl = (e.lv[m].ny - colour + 1) / 2;
    int i = e.warp;
    for (; i + e.nw < nl; i += 2 * e.nw) {
        const int ys[2] = {colour + 2 * i, colour + 2 * (i + e.nw)};
        lean_relax<S, K, 2>(e, fac, key, m, ys, 2, nbmode, out, plane, acc);
    }
    if (i < nl) {
        const int ys[1] = {colour + 2 * i};
        lean_relax<S, K, 1>(e, fac, key, m, ys, 1, nbmode, out, plane, acc);
    }
}

// g_{m+1}[j] from the odd lines 2j-1, 2j+1, 2j+3 of level m (restrict_combine: the residual of
// level m after its down-sweep); the result stays in registers.
template <int K>
__device__ __forceinline__ void lean_restrict_line(const LeanEnv<K> &e, const LeanLevel &L, int j, float (&acc)[K]) {
    const int nx = e.nx, lane = e.lane, e0 = 2 * j;
    const bool ha = e0 >= 1, h1 = e0 + 2 < L.ny, hc = e0 + 3 < L.ny;
    float va[K], vb[K], vc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) { va[q] = 0.0f; vc[q] = 0.0f; }
    if (ha) load_line<float, K>(va, L.u + (e0 - 1) * nx, nx, e.vec, lane);
    load_line<float, K>(vb, L.u + (e0 + 1) * nx, nx, e.vec, lane);
    if (hc) load_line<float, K>(vc, L.u + (e0 + 3) * nx, nx, e.vec, lane);
    const CoefRow<float> c0 = coef_row<float>(e.coef + (L.lb + e0) * kCoefPerLine);
    const CoefRow<float> c1 = coef_row<float>(e.coef + (L.lb + (h1 ? e0 + 2 : e0)) * kCoefPerLine);
    restrict_combine<float, K>(acc, va, vb, vc, c0, c1, ha, h1, hc, lane);
}

// Restriction from level m to level m+1, coarse lines in pairs (2k, 2k+1) with k = w + i nw;
// every coarse line's g is stored, and the even one of the pair is solved at once (level m+1's
// down-sweep relaxes its even lines with zero neighbours).
template <int K>
__device__ __forceinline__ void lean_restrict_solve(const LeanEnv<K> &e, TriFac<float, K> &fac, int &key, int m) {
    const LeanLevel L = e.lv[m], Lc = e.lv[m + 1];
    const int nx = e.nx, lane = e.lane;
    const int npairs = (Lc.ny + 1) / 2;
    for (int k = e.warp; k < npairs; k += e.nw) {
        const int j0 = 2 * k, j1 = 2 * k + 1;
        float g0[1][K];
        lean_restrict_line<K>(e, L, j0, g0[0]);
        store_line<float, K>(Lc.g + j0 * nx, g0[0], nx, e.vec, lane);
        if (j1 < Lc.ny) {
            float g1[K];
            lean_restrict_line<K>(e, L, j1, g1);
            store_line<float, K>(Lc.g + j1 * nx, g1, nx, e.vec, lane);
        }
        lean_fac<K>(fac, key, Lc, m + 1, j0 == Lc.ny - 1 ? 1 : 0, lane);
        tri_apply<float, K, 1>(fac, g0, nx, lane);
        store_line<float, K>(Lc.u + j0 * nx, g0[0], nx, e.vec, lane);
    }
}

// S0: the right-hand side g_0 = f_z - sum_dz A_{z,z+dz} u_{z+dz} of every line (mode 0: f_z; mode
// 1: the own plane is zero; mode 2: all terms), stored unless g_0 is f_z itself; even lines are
// solved at once (into u_0, or into the plane when the plane has a single line).  Lines in pairs
// (2k, 2k+1), k = w + i nw.
template <class S, int K>
__device__ __forceinline__ void lean_rhs_even(const LeanEnv<K> &e, TriFac<float, K> &fac, int &key, const PlaneRelaxArgs &a,
                                              int mode, bool g0_is_f, const S *fpl, const S *ub, int z,
                                              const float *zc, S *plane, bool acc, int P) {
    const LeanLevel L = e.lv[0];
    const int nx = a.nx, ny = a.ny, lane = e.lane;
    const long long np = static_cast<long long>(nx) * ny;
    const int npairs = (ny + 1) / 2;
    for (int k = e.warp; k < npairs; k += e.nw) {
        float d[2][K];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int y = 2 * k + t;
            if (y >= ny) break;
            load_plane_line<float, S, K>(d[t], fpl, y, nx, e.vec, lane);
            if (mode >= 1 && z > 0)
                sub_plane_term<float, S, K>(d[t], ub + (z - 1) * np, y, nx, ny, zc[0], zc[3], e.vec, lane);
            if (mode >= 1 && z + 1 < a.nz)
                sub_plane_term<float, S, K>(d[t], ub + (z + 1) * np, y, nx, ny, zc[2], zc[5], e.vec, lane);
            if (mode == 2) sub_plane_term<float, S, K>(d[t], ub + z * np, y, nx, ny, zc[1], zc[4], e.vec, lane);
            if (!g0_is_f) store_line<float, K>(L.g + y * nx, d[t], nx, e.vec, lane);
        }
        float dv[1][K];
#pragma unroll
        for (int j = 0; j < K; ++j) dv[0][j] = d[0][j];
        lean_fac<K>(fac, key, L, 0, 2 * k == ny - 1 ? 1 : 0, lane);
        tri_apply<float, K, 1>(fac, dv, nx, lane);
        lean_store<S, K>(e, L, 2 * k, dv[0], plane, acc, P == 1 ? OUT_PLANE : OUT_U);
    }
}

// The relaxation of the pidx-th plane of the colour (batch entry b) by one CTA.
template <class S, int K>
__device__ __forceinline__ void plane_lean_task(const PlaneRelaxArgs &a, int pidx, int b, long long slot,
                                                unsigned char *smem_raw) {
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int nx = a.nx, ny = a.ny, P = a.P;
    const long long np = static_cast<long long>(nx) * ny;
    const int z = a.colour + 2 * pidx;
    const int tid = threadIdx.x, nt = blockDim.x;
    LeanEnv<K> e;
    e.lane = tid & 31;
    e.warp = tid >> 5;
    e.nw = nt >> 5;
    e.nx = nx;
    e.vec = a.vec != 0;
    e.coef = sm;
    float *gw = reinterpret_cast<float *>(a.gws) + slot * a.ws_per_plane;
    const S *fb = reinterpret_cast<const S *>(a.f) + static_cast<long long>(b) * a.vstride;
    S *ub = reinterpret_cast<S *>(a.u) + static_cast<long long>(b) * a.vstride;
    S *plane = ub + static_cast<long long>(z) * np;
    const float *zc = a.zcoef32 + static_cast<long long>(z) * kCoefPerPlane;
    __shared__ LeanLevel s_lv[kMaxPlaneLevels];
    {
        const float *pc = a.pcoef32 + static_cast<long long>(z) * a.sum_ny * kCoefPerLine;
        for (int i = tid; i < a.sum_ny * kCoefPerLine; i += nt) sm[i] = pc[i];
        if (tid < P) {
            LeanLevel L;
            L.u = (((a.smem_u_mask >> tid) & 1u) ? sm : gw) + a.off_u[tid];
            L.g = (((a.smem_g_mask >> tid) & 1u) ? sm : gw) + a.off_g[tid];
            L.fs = sm + a.off_fs + 2 * tid * trifac_fields<float, K>() * 32;
            L.ny = a.ny_m[tid];
            L.lb = a.line_base[tid];
            s_lv[tid] = L;
        }
    }
    e.lv = s_lv;
    TriFac<float, K> fac;
    __syncthreads();
    // the two factor sets of every 2D level (interior line, last line), by warps in parallel
    for (int sidx = e.warp; sidx < 2 * P; sidx += e.nw) {
        const int mm = sidx >> 1;
        const int y = (sidx & 1) ? a.ny_m[mm] - 1 : 0;
        const float *lc = sm + (a.line_base[mm] + y) * kCoefPerLine;
        tri_factor<float, K>(fac, 2.0f * lc[1] + lc[4], -lc[1], nx, e.lane);
        trifac_store<float, K>(sm + a.off_fs + sidx * trifac_fields<float, K>() * 32, fac, e.lane);
    }
    // everything above reads only the hierarchy's tables (overlapping the previous kernel under
    // programmatic dependent launch); from here on the planes are read and written
    pdl_wait();
    __syncthreads();
    SMG_TRACE(0);
    int key = -1;
    for (int it = 0; it < a.iters; ++it) {
        const int mode = (it == 0) ? a.mode : 2;
        const bool acc = (mode == 2);
        const S *fpl = fb + static_cast<long long>(z) * np;
        // g_0 is f_z itself for the first red sweep when f is FP32 (the host then points u_0's
        // table entry's g at f); otherwise it is assembled into the level's g array
        bool g0_is_f = false;
        if constexpr (std::is_same<S, float>::value) g0_is_f = (mode == 0);
        if (g0_is_f && tid == 0) s_lv[0].g = const_cast<float *>(reinterpret_cast<const float *>(fpl));
        if (!g0_is_f && tid == 0) s_lv[0].g = (((a.smem_g_mask) & 1u) ? sm : gw) + a.off_g[0];
        __syncthreads();
        lean_rhs_even<S, K>(e, fac, key, a, mode, g0_is_f, fpl, ub, z, zc, plane, acc, P);
        __syncthreads();
        SMG_TRACE(1);
        if (P == 1) continue;
        for (int m = 0; m + 1 < P; ++m) {
            lean_colour<S, K>(e, fac, key, m, 1, NB_PLAIN, OUT_U, plane, false);
            __syncthreads();
            SMG_TRACE(2 + 2 * m);
            lean_restrict_solve<K>(e, fac, key, m);
            __syncthreads();
            SMG_TRACE(3 + 2 * m);
        }
        for (int m = P - 2; m >= 0; --m) {
            lean_colour<S, K>(e, fac, key, m, 1, NB_CORR, m > 0 ? OUT_U : OUT_U_AND_PLANE, plane, acc);
            __syncthreads();
            SMG_TRACE(2 * P + 2 * (P - 2 - m));
            lean_colour<S, K>(e, fac, key, m, 0, NB_PLAIN, m > 0 ? OUT_U : OUT_PLANE, plane, acc);
            __syncthreads();
            SMG_TRACE(2 * P + 1 + 2 * (P - 2 - m));
        }
    }
}

template <class S, int K>
__global__ void __launch_bounds__(512, 1) plane_lean_kernel(const __grid_constant__ PlaneRelaxArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    const long long slot = static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
    plane_lean_task<S, K>(a, static_cast<int>(blockIdx.x), static_cast<int>(blockIdx.y), slot, smem_raw);
}

}  // namespace smg
