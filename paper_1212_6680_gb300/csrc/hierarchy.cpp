// hierarchy.cpp -- host construction of the SMG hierarchy in FP64 (setup, done once).
//
// SMG (section "Preconditioning with SMG" of arXiv:1212.6680) coarsens in z; each plane is
// relaxed by a 2D cycle that coarsens in y with exact x-line solves.  The paper leaves the
// internals open; the library uses this semicoarsening reading:
//   * coarse points are the odd 0-based indices, n_{l+1} = floor(n_l / 2), down to 1;
//   * interpolation injects coarse points and gives each even fine point the weights
//     -X(i, i+-1) / X(i, i) of the coupling matrix X obtained by collapsing the interior
//     stencil across the non-coarsened directions (for z: X = K_l; for y: X = T_m);
//   * restriction is the transpose and coarse operators are Galerkin products P^T A P.
// Operators keep the Kronecker form
//   (A_l u)_z = sum_dz M_l(z,z+dz) L2D u_{z+dz} + K_l(z,z+dz) u_{z+dz},   M_0 = I, K_0 = tridiag(-1,2,-1)
//   (B_m u)_y = sum_dy S_m(y,y+dy) Lx u_{y+dy} + T_m(y,y+dy) u_{y+dy},   S_0 = c I, T_0 = c Ly + d I
// with c = M_l(z,z), d = K_l(z,z) for the plane operator B = c L2D + d I of plane z.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "smg_internal.h"

namespace smg {
namespace {

// Tridiagonal matrix as three diagonals: lo[i] = X(i,i-1), di[i] = X(i,i), up[i] = X(i,i+1).
struct Tridiag {
    std::vector<double> lo, di, up;
    explicit Tridiag(int n = 0) : lo(n, 0.0), di(n, 0.0), up(n, 0.0) {}
    int size() const { return static_cast<int>(di.size()); }
};

struct Weights {
    std::vector<double> wm, wp;  // per fine point; zero for coarse (odd) points
};

Weights collapse_weights(const Tridiag &X) {
    const int n = X.size();
    Weights w{std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};
    for (int i = 0; i < n; i += 2) {
        if (i > 0) w.wm[i] = -X.lo[i] / X.di[i];
        if (i + 1 < n) w.wp[i] = -X.up[i] / X.di[i];
    }
    return w;
}

// Galerkin product P^T X P for the interpolation given by w.  P has, in column j (coarse
// point j <-> fine 2j+1): 1 at row 2j+1, wp(2j) at row 2j, wm(2j+2) at row 2j+2.
Tridiag galerkin(const Tridiag &X, const Weights &w) {
    const int n = X.size(), nc = n / 2;
    Tridiag C(nc);
    // column j of P as (row, weight) triples
    auto col = [&](int j, std::array<std::pair<int, double>, 3> &out) {
        int cnt = 0;
        out[cnt++] = {2 * j + 1, 1.0};
        out[cnt++] = {2 * j, w.wp[2 * j]};
        if (2 * j + 2 < n) out[cnt++] = {2 * j + 2, w.wm[2 * j + 2]};
        else out[cnt++] = {-1, 0.0};
        return cnt;
    };
    auto xget = [&](int i, int k) -> double {
        if (i < 0 || k < 0 || i >= n || k >= n) return 0.0;
        if (k == i) return X.di[i];
        if (k == i - 1) return X.lo[i];
        if (k == i + 1) return X.up[i];
        return 0.0;
    };
    for (int i = 0; i < nc; ++i) {
        std::array<std::pair<int, double>, 3> ci, cj;
        col(i, ci);
        for (int j = std::max(0, i - 1); j <= std::min(nc - 1, i + 1); ++j) {
            col(j, cj);
            double v = 0.0;
            for (auto &a : ci) {
                if (a.first < 0) continue;
                for (auto &b : cj) {
                    if (b.first < 0) continue;
                    v += a.second * xget(a.first, b.first) * b.second;
                }
            }
            if (j == i) C.di[i] = v;
            else if (j == i - 1) C.lo[i] = v;
            else C.up[i] = v;
        }
    }
    return C;
}

int num_levels(int n) {
    int c = 1;
    while (n > 1) {
        n /= 2;
        ++c;
    }
    return c;
}

}  // namespace

int hierarchy_levels(int n) { return num_levels(n); }

void build_hierarchy(int nx, int ny, int nz, HostHierarchy &H) {
    H = HostHierarchy();
    H.nx = nx;
    H.ny = ny;
    H.nz = nz;
    H.L = num_levels(nz);
    H.P = num_levels(ny);
    H.nz_l.resize(H.L);
    H.plane_base.resize(H.L);
    H.ny_m.resize(H.P);
    H.line_base.resize(H.P);
    {
        int n = ny, base = 0;
        for (int m = 0; m < H.P; ++m) {
            H.ny_m[m] = n;
            H.line_base[m] = base;
            base += n;
            n /= 2;
        }
        H.sum_ny = base;
    }
    {
        int n = nz, base = 0;
        for (int l = 0; l < H.L; ++l) {
            H.nz_l[l] = n;
            H.plane_base[l] = base;
            base += n;
            n /= 2;
        }
        H.nplanes_total = base;
    }
    H.zcoef.assign(static_cast<size_t>(H.nplanes_total) * kCoefPerPlane, 0.0);
    H.pcoef.assign(static_cast<size_t>(H.nplanes_total) * H.sum_ny * kCoefPerLine, 0.0);

    Tridiag M(nz), K(nz);
    for (int z = 0; z < nz; ++z) {
        M.di[z] = 1.0;
        K.di[z] = 2.0;
        if (z > 0) K.lo[z] = -1.0;
        if (z + 1 < nz) K.up[z] = -1.0;
    }
    for (int l = 0; l < H.L; ++l) {
        const int n = M.size();
        Weights w = (l + 1 < H.L) ? collapse_weights(K)
                                  : Weights{std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};
        for (int z = 0; z < n; ++z) {
            double *zc = &H.zcoef[static_cast<size_t>(H.plane_base[l] + z) * kCoefPerPlane];
            zc[0] = M.lo[z];
            zc[1] = M.di[z];
            zc[2] = M.up[z];
            zc[3] = K.lo[z];
            zc[4] = K.di[z];
            zc[5] = K.up[z];
            zc[6] = w.wm[z];
            zc[7] = w.wp[z];
            // the plane's 2D hierarchy for B = c L2D + d I
            const double c = M.di[z], d = K.di[z];
            Tridiag S(ny), T(ny);
            for (int y = 0; y < ny; ++y) {
                S.di[y] = c;
                T.di[y] = 2.0 * c + d;
                if (y > 0) T.lo[y] = -c;
                if (y + 1 < ny) T.up[y] = -c;
            }
            double *pc = &H.pcoef[static_cast<size_t>(H.plane_base[l] + z) * H.sum_ny * kCoefPerLine];
            for (int m = 0; m < H.P; ++m) {
                const int nym = S.size();
                Weights wy = (m + 1 < H.P) ? collapse_weights(T)
                                           : Weights{std::vector<double>(nym, 0.0), std::vector<double>(nym, 0.0)};
                for (int y = 0; y < nym; ++y) {
                    double *lc = pc + static_cast<size_t>(H.line_base[m] + y) * kCoefPerLine;
                    lc[0] = S.lo[y];
                    lc[1] = S.di[y];
                    lc[2] = S.up[y];
                    lc[3] = T.lo[y];
                    lc[4] = T.di[y];
                    lc[5] = T.up[y];
                    lc[6] = wy.wm[y];
                    lc[7] = wy.wp[y];
                }
                if (m + 1 < H.P) {
                    Tridiag Sc = galerkin(S, wy), Tc = galerkin(T, wy);
                    S = Sc;
                    T = Tc;
                }
            }
        }
        if (l + 1 < H.L) {
            Tridiag Mc = galerkin(M, w), Kc = galerkin(K, w);
            M = Mc;
            K = Kc;
        }
    }
}

bool lean_uniform_level(const HostHierarchy &H, int l) {
    for (int z = 0; z < H.nz_l[l]; ++z) {
        const double *pc = &H.pcoef[static_cast<size_t>(H.plane_base[l] + z) * H.sum_ny * kCoefPerLine];
        for (int m = 0; m < H.P; ++m) {
            const double *l0 = pc + static_cast<size_t>(H.line_base[m]) * kCoefPerLine;
            for (int y = 1; y + 1 < H.ny_m[m]; ++y) {
                const double *ly = pc + static_cast<size_t>(H.line_base[m] + y) * kCoefPerLine;
                if (ly[1] != l0[1] || ly[4] != l0[4]) return false;
            }
        }
    }
    return true;
}

int plane_classes(const HostHierarchy &H, int l, std::vector<int> &slot, std::vector<int> &rep) {
    const size_t per = static_cast<size_t>(H.sum_ny) * kCoefPerLine;
    const double *base = &H.pcoef[static_cast<size_t>(H.plane_base[l]) * per];
    slot.assign(H.nz_l[l], -1);
    rep.clear();
    for (int z = 0; z < H.nz_l[l]; ++z) {
        for (size_t c = 0; c < rep.size() && slot[z] < 0; ++c)
            if (std::memcmp(base + z * per, base + static_cast<size_t>(rep[c]) * per, per * sizeof(double)) == 0)
                slot[z] = static_cast<int>(c);
        if (slot[z] < 0) {
            slot[z] = static_cast<int>(rep.size());
            rep.push_back(z);
        }
    }
    return static_cast<int>(rep.size());
}

// Greedy placement of the 2D-cycle arrays: the coefficient table first, then the coarsest
// levels (latency-bound, few lines) and finally the finest; u_m before g_m at each level
// (the iterate is touched more often than the right-hand side).  What does not fit in
// `smem_budget` goes to a global slot per CTA (L2-resident for the sizes of interest).
// Instantiated x-line chunk size for nx (rows per lane): 1, 2, 3, 4, 6, 8 or 16.
// Factor sets kept in shared memory: every 2D level (the single-line coarsest included), unless
// they would take more than a third of the budget; then only the finest MF levels keep theirs
// and the others factor on the fly.
static int factor_levels(const HostHierarchy &H, int K, size_t elem_bytes, size_t smem_budget) {
    const size_t set_bytes = 2 * static_cast<size_t>(trifac_set_elems(K)) * elem_bytes;  // two per level
    int mf = std::min(H.P, kMaxFactorLevels);
    while (mf > 0 && static_cast<size_t>(mf) * set_bytes > smem_budget / 3) --mf;
    return mf;
}

static int chunk_K(int nx) {
    const int k = (nx + 31) / 32;
    if (k <= 4) return k;
    if (k <= 6) return 6;
    if (k <= 8) return 8;
    return 16;
}

// Placement priority of the 2D-cycle arrays: both arrays of levels >= 2 (coarse to fine), then
// u_1, u_0, g_1, g_0.  Entries are (level, 0 = u / 1 = g).
static std::vector<std::pair<int, int>> layout_order(const HostHierarchy &H) {
    std::vector<std::pair<int, int>> order;
    for (int m = H.P - 1; m >= 2; --m) {
        order.push_back({m, 0});
        order.push_back({m, 1});
    }
    if (H.P > 1) order.push_back({1, 0});
    order.push_back({0, 0});
    if (H.P > 1) order.push_back({1, 1});
    order.push_back({0, 1});
    return order;
}

// Shared memory starts with the plane's coefficient table and the factor sets of the interior
// line matrices of the first MF 2D levels (the levels with many lines; the others factor on
// the fly), then the 2D-cycle arrays, placed greedily: the coarsest levels first (latency-bound,
// few lines) and finally the finest; u_m before g_m at each level (the iterate is touched more
// often).  What does not fit in `smem_budget` goes to a global slot per CTA (L2-resident for
// the sizes of interest).
PlaneLayout plan_plane_layout(const HostHierarchy &H, size_t elem_bytes, size_t smem_budget, int K, bool all_sets,
                              bool no_sets) {
    PlaneLayout P;
    P.K = K > 0 ? K : chunk_K(H.nx);
    auto align4 = [](size_t v) { return (v + 3) & ~static_cast<size_t>(3); };
    size_t smem_elems = align4(static_cast<size_t>(H.sum_ny) * kCoefPerLine);
    P.MF = no_sets ? 0
                   : (all_sets ? std::min(H.P, kMaxFactorLevels) : factor_levels(H, P.K, elem_bytes, smem_budget));
    P.off_fs = static_cast<int>(smem_elems);
    smem_elems += 2 * static_cast<size_t>(P.MF) * trifac_set_elems(P.K);
    long long gl = 0;
    const size_t budget_elems = smem_budget / elem_bytes;
    for (const auto &o : layout_order(H)) {
        const int m = o.first;
        const size_t sz = align4(static_cast<size_t>(H.nx) * H.ny_m[m]);
        if (smem_elems + sz <= budget_elems) {
            if (o.second == 0) {
                P.off_u[m] = static_cast<int>(smem_elems);
                P.smem_u_mask |= 1u << m;
            } else {
                P.off_g[m] = static_cast<int>(smem_elems);
                P.smem_g_mask |= 1u << m;
            }
            smem_elems += sz;
        } else {
            if (o.second == 0) P.off_u[m] = static_cast<int>(gl);
            else P.off_g[m] = static_cast<int>(gl);
            gl += static_cast<long long>(sz);
        }
    }
    P.smem_bytes = smem_elems * elem_bytes;
    P.ws_per_plane = gl;
    return P;
}

PlaneLayout plan_plane_layout_cluster(const HostHierarchy &H, size_t elem_bytes, size_t smem_budget, int R,
                                      bool all_sets, int solo_from, bool no_sets) {
    PlaneLayout P;
    P.K = chunk_K(H.nx);
    P.solo_from = solo_from;
    auto align4 = [](size_t v) { return (v + 3) & ~static_cast<size_t>(3); };
    size_t smem_elems = align4(static_cast<size_t>(H.sum_ny) * kCoefPerLine);
    P.MF = no_sets ? 0
                   : (all_sets ? std::min(H.P, kMaxFactorLevels) : factor_levels(H, P.K, elem_bytes, smem_budget));
    P.off_fs = static_cast<int>(smem_elems);
    smem_elems += 2 * static_cast<size_t>(P.MF) * trifac_set_elems(P.K);
    const size_t budget_elems = smem_budget / elem_bytes;
    if (smem_elems > budget_elems) {
        P.smem_bytes = 0;
        return P;
    }
    // the same priority as one CTA per plane; each CTA holds its share of an on-chip array, and
    // an array that does not fit lives whole in the cluster's global slot
    long long gl = 0;
    for (const auto &o : layout_order(H)) {
        const int m = o.first;
        const int pairs = (H.ny_m[m] + 1) / 2;
        const size_t nloc = (m >= solo_from) ? static_cast<size_t>(H.ny_m[m]) : 2 * static_cast<size_t>((pairs + R - 1) / R);
        const size_t sz = align4(static_cast<size_t>(H.nx) * nloc);
        int &off = (o.second == 0) ? P.off_u[m] : P.off_g[m];
        unsigned &mask = (o.second == 0) ? P.smem_u_mask : P.smem_g_mask;
        if (smem_elems + sz <= budget_elems) {
            off = static_cast<int>(smem_elems);
            mask |= 1u << m;
            smem_elems += sz;
        } else {
            off = static_cast<int>(gl);
            gl += static_cast<long long>(align4(static_cast<size_t>(H.nx) * H.ny_m[m]));
        }
    }
    P.smem_bytes = smem_elems * elem_bytes;
    P.ws_per_plane = gl;
    return P;
}

}  // namespace smg
