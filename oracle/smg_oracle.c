/*
 * smg_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see smg_oracle.h).
 *
 * What it computes, and where each piece comes from:
 *
 *  - Model operator: the 3D negative Laplacian, 7-point stencil, unit grid spacing,
 *    homogeneous Dirichlet boundary (section "PSD and PCG methods", model problem;
 *    section "Preconditioning of LOBPCG with SMG" repeats it).
 *  - Algorithm 1 (PSD / PCG), with beta from eq. (1) (standard PCG), eq. (2) (flexible
 *    PCG, which needs the extra vector r_k - r_{k-1}) or beta = 0 (PSD).
 *  - The SMG preconditioner T (section "Preconditioning with SMG"): a V-cycle with plane
 *    relaxation and -v npre npost smoothing counts.  The paper does not give SMG's
 *    internals; this file fixes the following reading of them (semicoarsening multigrid):
 *
 *    z-hierarchy.  Level 0 is the fine grid.  nz_{l+1} = floor(nz_l / 2); the coarse planes
 *    are the odd 0-based fine planes (coarse j <-> fine 2j+1); the last level has one plane.
 *    Every level operator has the form
 *        (A_l u)_z = sum_{dz=-1..1} [ M_l(z,z+dz) * L2D u_{z+dz} + K_l(z,z+dz) * u_{z+dz} ]
 *    with L2D the 5-point 2D Dirichlet Laplacian of one plane and M_l, K_l tridiagonal
 *    nz_l x nz_l matrices; M_0 = I, K_0 = tridiag(-1, 2, -1).
 *    Prolongation P_l: coarse planes are injected; an even fine plane z takes
 *    wm(z) e_{z-1} + wp(z) e_{z+1} with w(z) = -K_l(z,z+-1) / K_l(z,z), i.e. the stencil
 *    collapsed in-plane (interior stencil: the in-plane row sum of L2D is zero, so the
 *    collapsed coupling is K_l); a neighbour outside the brick contributes nothing.
 *    Restriction R = P^T and Galerkin coarse operators A_{l+1} = P^T A_l P, which keeps the
 *    form above with M_{l+1} = P^T M_l P and K_{l+1} = P^T K_l P (15-point stencils).
 *
 *    Plane solve.  The plane operator of plane z is B = c*L2D + d*I with c = M_l(z,z),
 *    d = K_l(z,z).  It is solved approximately by one 2D V-cycle, zero initial guess, that
 *    coarsens in y exactly as above (operators (B_m u)_y = sum_dy [S_m(y,y+dy) Lx u_{y+dy}
 *    + T_m(y,y+dy) u_{y+dy}], S_0 = c I, T_0 = c Ly + d I, y-weights -T_m(y,y+-1)/T_m(y,y)),
 *    relaxes even then odd y-lines going down and odd then even going up, each line solved
 *    exactly (Thomas), and solves the single line left at the bottom exactly.
 *
 *    3D cycle.  From u = 0 on every level: npre sweeps of red (even z) then black (odd z)
 *    plane relaxation, u_z += C_z (f - A_l u)_z; residual, restriction; recursion;
 *    prolongation and correction; npost sweeps of black then red.  The level with one plane
 *    applies coarse_iters steps u += C (f - A u) of the plane cycle.
 *
 * Every loop below is the definition written out; no blocking, fusion or reordering.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "smg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX3(x, y, z, nx, ny) ((((size_t)(z)) * (size_t)(ny) + (size_t)(y)) * (size_t)(nx) + (size_t)(x))

/* ------------------------------------------------------------------------------------ */
/* Model operator                                                                        */
/* ------------------------------------------------------------------------------------ */

void orc_apply_A(int nx, int ny, int nz, const double *u, double *out)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nz > 4)
#endif
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double v = 6.0 * u[IDX3(x, y, z, nx, ny)];
                if (x > 0) v -= u[IDX3(x - 1, y, z, nx, ny)];
                if (x < nx - 1) v -= u[IDX3(x + 1, y, z, nx, ny)];
                if (y > 0) v -= u[IDX3(x, y - 1, z, nx, ny)];
                if (y < ny - 1) v -= u[IDX3(x, y + 1, z, nx, ny)];
                if (z > 0) v -= u[IDX3(x, y, z - 1, nx, ny)];
                if (z < nz - 1) v -= u[IDX3(x, y, z + 1, nx, ny)];
                out[IDX3(x, y, z, nx, ny)] = v;
            }
}

/* ------------------------------------------------------------------------------------ */
/* Thomas algorithm (textbook LU without pivoting of a tridiagonal matrix)               */
/* ------------------------------------------------------------------------------------ */

void orc_thomas(int n, const double *a, const double *b, const double *c,
                const double *d, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double den = b[i] - (i > 0 ? a[i] * cp[i - 1] : 0.0);
        cp[i] = (i < n - 1 ? c[i] : 0.0) / den;
        dp[i] = (d[i] - (i > 0 ? a[i] * dp[i - 1] : 0.0)) / den;
    }
    for (int i = n - 1; i >= 0; --i)
        x[i] = dp[i] - (i < n - 1 ? cp[i] * x[i + 1] : 0.0);
    free(cp);
    free(dp);
}

/* ------------------------------------------------------------------------------------ */
/* 1D semicoarsening pieces: tridiagonal matrices, interpolation, Galerkin product        */
/* ------------------------------------------------------------------------------------ */

/* Tridiagonal n x n matrix stored as e[3*i + (j - i + 1)] = X(i, j), |i - j| <= 1. */
typedef struct {
    int n;
    double *e;
} tri_t;

static tri_t tri_new(int n)
{
    tri_t t;
    t.n = n;
    t.e = (double *)calloc((size_t)3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    return t;
}

static double tri_get(const tri_t *t, int i, int j)
{
    if (i < 0 || j < 0 || i >= t->n || j >= t->n || abs(i - j) > 1) return 0.0;
    return t->e[3 * i + (j - i + 1)];
}

static void tri_add(tri_t *t, int i, int j, double v)
{
    t->e[3 * i + (j - i + 1)] += v;
}

/* Interpolation weights of the fine points from the collapsed coupling matrix X:
 * w-(i) = -X(i,i-1)/X(i,i), w+(i) = -X(i,i+1)/X(i,i) for even i; a neighbour outside
 * [0, n) gives weight 0.  Odd i are the coarse points (injection); their entries are 0. */
static void interp_weights(const tri_t *X, double *wm, double *wp)
{
    for (int i = 0; i < X->n; ++i) {
        wm[i] = 0.0;
        wp[i] = 0.0;
        if (i % 2 == 0) {
            double di = tri_get(X, i, i);
            if (i - 1 >= 0) wm[i] = -tri_get(X, i, i - 1) / di;
            if (i + 1 < X->n) wp[i] = -tri_get(X, i, i + 1) / di;
        }
    }
}

/* Row i of the prolongation P (n_fine x n_fine/2): up to two (coarse index, weight) pairs. */
static int prolong_row(int i, int n, const double *wm, const double *wp, int *cj, double *cw)
{
    int nc = n / 2, cnt = 0;
    if (i % 2 == 1) {
        cj[cnt] = (i - 1) / 2;
        cw[cnt++] = 1.0;
    } else {
        if (i - 1 >= 0) {
            cj[cnt] = i / 2 - 1;
            cw[cnt++] = wm[i];
        }
        if (i + 1 < n && i / 2 < nc) {
            cj[cnt] = i / 2;
            cw[cnt++] = wp[i];
        }
    }
    return cnt;
}

/* Galerkin triple product Xc = P^T X P, summed entry by entry over the nonzeros. */
static tri_t galerkin(const tri_t *X, const double *wm, const double *wp)
{
    int n = X->n, nc = n / 2;
    tri_t Xc = tri_new(nc);
    for (int a = 0; a < n; ++a) {
        int ca[2], cb[2];
        double wa[2], wb[2];
        int na = prolong_row(a, n, wm, wp, ca, wa);
        for (int b = a - 1; b <= a + 1; ++b) {
            if (b < 0 || b >= n) continue;
            double xab = tri_get(X, a, b);
            int nb = prolong_row(b, n, wm, wp, cb, wb);
            for (int p = 0; p < na; ++p)
                for (int q = 0; q < nb; ++q)
                    tri_add(&Xc, ca[p], cb[q], wa[p] * xab * wb[q]);
        }
    }
    return Xc;
}

/* ------------------------------------------------------------------------------------ */
/* The 2D plane hierarchy and plane cycle                                                */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int nx, nlev;   /* nlev 2D levels, ny_m halving down to 1 */
    int *ny;        /* [nlev] */
    tri_t *S, *T;   /* [nlev] operators (B_m u)_y = sum S(y,y') Lx u_y' + T(y,y') u_y' */
    double **wm, **wp; /* [nlev] y-interpolation weights (from T) */
} plane_h;

static int count_levels(int n)
{
    int c = 1;
    while (n > 1) {
        n /= 2;
        ++c;
    }
    return c;
}

static void plane_build(plane_h *ph, int nx, int ny, double c, double d)
{
    ph->nx = nx;
    ph->nlev = count_levels(ny);
    ph->ny = (int *)malloc(sizeof(int) * (size_t)ph->nlev);
    ph->S = (tri_t *)malloc(sizeof(tri_t) * (size_t)ph->nlev);
    ph->T = (tri_t *)malloc(sizeof(tri_t) * (size_t)ph->nlev);
    ph->wm = (double **)malloc(sizeof(double *) * (size_t)ph->nlev);
    ph->wp = (double **)malloc(sizeof(double *) * (size_t)ph->nlev);
    int n = ny;
    ph->S[0] = tri_new(n);
    ph->T[0] = tri_new(n);
    for (int y = 0; y < n; ++y) {
        tri_add(&ph->S[0], y, y, c);
        tri_add(&ph->T[0], y, y, 2.0 * c + d);
        if (y > 0) tri_add(&ph->T[0], y, y - 1, -c);
        if (y < n - 1) tri_add(&ph->T[0], y, y + 1, -c);
    }
    for (int m = 0; m < ph->nlev; ++m) {
        ph->ny[m] = n;
        ph->wm[m] = (double *)calloc((size_t)n, sizeof(double));
        ph->wp[m] = (double *)calloc((size_t)n, sizeof(double));
        if (m + 1 < ph->nlev) {
            interp_weights(&ph->T[m], ph->wm[m], ph->wp[m]);
            ph->S[m + 1] = galerkin(&ph->S[m], ph->wm[m], ph->wp[m]);
            ph->T[m + 1] = galerkin(&ph->T[m], ph->wm[m], ph->wp[m]);
            n /= 2;
        }
    }
}

static void plane_free(plane_h *ph)
{
    for (int m = 0; m < ph->nlev; ++m) {
        free(ph->S[m].e);
        free(ph->T[m].e);
        free(ph->wm[m]);
        free(ph->wp[m]);
    }
    free(ph->ny);
    free(ph->S);
    free(ph->T);
    free(ph->wm);
    free(ph->wp);
}

/* (B_m u) on one 2D level: out_y = sum_dy S(y,y+dy) Lx u_{y+dy} + T(y,y+dy) u_{y+dy}. */
static void plane_apply(const plane_h *ph, int m, const double *u, double *out)
{
    int nx = ph->nx, ny = ph->ny[m];
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double v = 0.0;
            for (int yy = y - 1; yy <= y + 1; ++yy) {
                if (yy < 0 || yy >= ny) continue;
                const double *uy = u + (size_t)yy * nx;
                double lx = 2.0 * uy[x] - (x > 0 ? uy[x - 1] : 0.0) - (x < nx - 1 ? uy[x + 1] : 0.0);
                v += tri_get(&ph->S[m], y, yy) * lx + tri_get(&ph->T[m], y, yy) * uy[x];
            }
            out[(size_t)y * nx + x] = v;
        }
}

/* Exact relaxation of line y: (S(y,y) Lx + T(y,y) I) u_y = g_y - sum_{dy=+-1} B_{y,y+dy} u_{y+dy}. */
static void line_relax(const plane_h *ph, int m, int y, const double *g, double *u)
{
    int nx = ph->nx, ny = ph->ny[m];
    double *a = (double *)malloc(sizeof(double) * (size_t)nx);
    double *b = (double *)malloc(sizeof(double) * (size_t)nx);
    double *c = (double *)malloc(sizeof(double) * (size_t)nx);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)nx);
    double syy = tri_get(&ph->S[m], y, y), tyy = tri_get(&ph->T[m], y, y);
    for (int x = 0; x < nx; ++x) {
        double v = g[(size_t)y * nx + x];
        for (int yy = y - 1; yy <= y + 1; yy += 2) {
            if (yy < 0 || yy >= ny) continue;
            const double *uy = u + (size_t)yy * nx;
            double lx = 2.0 * uy[x] - (x > 0 ? uy[x - 1] : 0.0) - (x < nx - 1 ? uy[x + 1] : 0.0);
            v -= tri_get(&ph->S[m], y, yy) * lx + tri_get(&ph->T[m], y, yy) * uy[x];
        }
        rhs[x] = v;
        a[x] = -syy;
        b[x] = 2.0 * syy + tyy;
        c[x] = -syy;
    }
    orc_thomas(nx, a, b, c, rhs, u + (size_t)y * nx);
    free(a);
    free(b);
    free(c);
    free(rhs);
}

#ifdef _OPENMP
#define ORC_PAR_LINES _Pragma("omp parallel for schedule(dynamic, 1) if (!omp_in_parallel() && ny > 8)")
#else
#define ORC_PAR_LINES
#endif

/* One 2D V-cycle on level m: u = C_m g, zero initial guess. */
static void plane_vcycle(const plane_h *ph, int m, const double *g, double *u)
{
    int nx = ph->nx, ny = ph->ny[m];
    size_t np = (size_t)nx * (size_t)ny;
    memset(u, 0, sizeof(double) * np);
    if (m == ph->nlev - 1) { /* one line left: exact solve */
        for (int y = 0; y < ny; ++y) line_relax(ph, m, y, g, u);
        return;
    }
    /* pre-relaxation: even lines, then odd lines (the lines of one colour are independent; with
       OpenMP they are shared among threads when no outer loop already is) */
    ORC_PAR_LINES
    for (int y = 0; y < ny; y += 2) line_relax(ph, m, y, g, u);
    ORC_PAR_LINES
    for (int y = 1; y < ny; y += 2) line_relax(ph, m, y, g, u);
    /* residual and restriction g_c = P^T (g - B u) */
    double *r = (double *)malloc(sizeof(double) * np);
    plane_apply(ph, m, u, r);
    for (size_t i = 0; i < np; ++i) r[i] = g[i] - r[i];
    int nyc = ph->ny[m + 1];
    size_t npc = (size_t)nx * (size_t)nyc;
    double *gc = (double *)calloc(npc, sizeof(double));
    double *uc = (double *)calloc(npc, sizeof(double));
    for (int y = 0; y < ny; ++y) {
        int cj[2];
        double cw[2];
        int cnt = prolong_row(y, ny, ph->wm[m], ph->wp[m], cj, cw);
        for (int p = 0; p < cnt; ++p)
            for (int x = 0; x < nx; ++x)
                gc[(size_t)cj[p] * nx + x] += cw[p] * r[(size_t)y * nx + x];
    }
    plane_vcycle(ph, m + 1, gc, uc);
    /* prolongation and correction u += P u_c */
    for (int y = 0; y < ny; ++y) {
        int cj[2];
        double cw[2];
        int cnt = prolong_row(y, ny, ph->wm[m], ph->wp[m], cj, cw);
        for (int p = 0; p < cnt; ++p)
            for (int x = 0; x < nx; ++x)
                u[(size_t)y * nx + x] += cw[p] * uc[(size_t)cj[p] * nx + x];
    }
    /* post-relaxation: odd lines, then even lines */
    ORC_PAR_LINES
    for (int y = 1; y < ny; y += 2) line_relax(ph, m, y, g, u);
    ORC_PAR_LINES
    for (int y = 0; y < ny; y += 2) line_relax(ph, m, y, g, u);
    free(r);
    free(gc);
    free(uc);
}

void orc_plane_cycle(int nx, int ny, double c, double d, const double *g, double *v)
{
    plane_h ph;
    plane_build(&ph, nx, ny, c, d);
    plane_vcycle(&ph, 0, g, v);
    plane_free(&ph);
}

/* ------------------------------------------------------------------------------------ */
/* The 3D SMG hierarchy and V-cycle                                                      */
/* ------------------------------------------------------------------------------------ */

struct orc_smg {
    int nx, ny, nz, npre, npost, coarse_iters;
    int L;                /* number of z-levels */
    int *nz_l;            /* [L] */
    tri_t *M, *K;         /* [L] */
    double **wm, **wp;    /* [L] z-interpolation weights */
    plane_h **ph;         /* [L][nz_l] plane hierarchies */
    double *learned;      /* NULL, or the 7776 weights of the learned post-correction */
    long long learned_accepted, learned_calls;
};

orc_smg *orc_smg_setup(int nx, int ny, int nz, int npre, int npost, int coarse_iters)
{
    if (nx < 1 || ny < 1 || nz < 1 || npre < 1 || npost < 0 || coarse_iters < 1) return NULL;
    orc_smg *h = (orc_smg *)calloc(1, sizeof(orc_smg));
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->npre = npre;
    h->npost = npost;
    h->coarse_iters = coarse_iters;
    h->L = count_levels(nz);
    h->nz_l = (int *)malloc(sizeof(int) * (size_t)h->L);
    h->M = (tri_t *)malloc(sizeof(tri_t) * (size_t)h->L);
    h->K = (tri_t *)malloc(sizeof(tri_t) * (size_t)h->L);
    h->wm = (double **)malloc(sizeof(double *) * (size_t)h->L);
    h->wp = (double **)malloc(sizeof(double *) * (size_t)h->L);
    h->ph = (plane_h **)malloc(sizeof(plane_h *) * (size_t)h->L);
    int n = nz;
    h->M[0] = tri_new(n);
    h->K[0] = tri_new(n);
    for (int z = 0; z < n; ++z) {
        tri_add(&h->M[0], z, z, 1.0);
        tri_add(&h->K[0], z, z, 2.0);
        if (z > 0) tri_add(&h->K[0], z, z - 1, -1.0);
        if (z < n - 1) tri_add(&h->K[0], z, z + 1, -1.0);
    }
    for (int l = 0; l < h->L; ++l) {
        h->nz_l[l] = n;
        h->wm[l] = (double *)calloc((size_t)n, sizeof(double));
        h->wp[l] = (double *)calloc((size_t)n, sizeof(double));
        h->ph[l] = (plane_h *)malloc(sizeof(plane_h) * (size_t)n);
        for (int z = 0; z < n; ++z)
            plane_build(&h->ph[l][z], nx, ny, tri_get(&h->M[l], z, z), tri_get(&h->K[l], z, z));
        if (l + 1 < h->L) {
            interp_weights(&h->K[l], h->wm[l], h->wp[l]);
            h->M[l + 1] = galerkin(&h->M[l], h->wm[l], h->wp[l]);
            h->K[l + 1] = galerkin(&h->K[l], h->wm[l], h->wp[l]);
            n /= 2;
        }
    }
    return h;
}

void orc_smg_free(orc_smg *h)
{
    if (!h) return;
    for (int l = 0; l < h->L; ++l) {
        for (int z = 0; z < h->nz_l[l]; ++z) plane_free(&h->ph[l][z]);
        free(h->ph[l]);
        free(h->M[l].e);
        free(h->K[l].e);
        free(h->wm[l]);
        free(h->wp[l]);
    }
    free(h->ph);
    free(h->M);
    free(h->K);
    free(h->wm);
    free(h->wp);
    free(h->nz_l);
    free(h->learned);
    free(h);
}

/* 2D 5-point Dirichlet Laplacian of one plane. */
static void l2d(int nx, int ny, const double *u, double *out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            double v = 4.0 * u[i];
            if (x > 0) v -= u[i - 1];
            if (x < nx - 1) v -= u[i + 1];
            if (y > 0) v -= u[i - nx];
            if (y < ny - 1) v -= u[i + nx];
            out[i] = v;
        }
}

/* Row block z of the level operator: out = sum_dz M(z,z+dz) L2D u_{z+dz} + K(z,z+dz) u_{z+dz}. */
static void level_apply_plane(const orc_smg *h, int l, int z, const double *u, double *out, double *tmp)
{
    int nx = h->nx, ny = h->ny, nzl = h->nz_l[l];
    size_t np = (size_t)nx * (size_t)ny;
    for (size_t i = 0; i < np; ++i) out[i] = 0.0;
    for (int zz = z - 1; zz <= z + 1; ++zz) {
        if (zz < 0 || zz >= nzl) continue;
        const double *uz = u + (size_t)zz * np;
        double m = tri_get(&h->M[l], z, zz), k = tri_get(&h->K[l], z, zz);
        l2d(nx, ny, uz, tmp);
        for (size_t i = 0; i < np; ++i) out[i] += m * tmp[i] + k * uz[i];
    }
}

/* Plane relaxation in correction form: u_z += C_z (f - A_l u)_z. */
static void plane_relax(const orc_smg *h, int l, int z, const double *f, double *u,
                        double *g, double *v, double *tmp)
{
    size_t np = (size_t)h->nx * (size_t)h->ny;
    level_apply_plane(h, l, z, u, g, tmp);
    for (size_t i = 0; i < np; ++i) g[i] = f[(size_t)z * np + i] - g[i];
    plane_vcycle(&h->ph[l][z], 0, g, v);
    for (size_t i = 0; i < np; ++i) u[(size_t)z * np + i] += v[i];
}

/* The planes z0, z0 + 2, ... < nzl of one colour, relaxed independently (each reads only the
   other colour's planes); with OpenMP they are shared among threads, each with its own scratch. */
static void relax_colour(const orc_smg *h, int l, int z0, const double *f, double *u)
{
    int nzl = h->nz_l[l];
    size_t np = (size_t)h->nx * (size_t)h->ny;
#ifdef _OPENMP
#pragma omp parallel if (nzl > 2)
#endif
    {
        double *g = (double *)malloc(sizeof(double) * np);
        double *v = (double *)malloc(sizeof(double) * np);
        double *tmp = (double *)malloc(sizeof(double) * np);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int z = z0; z < nzl; z += 2) plane_relax(h, l, z, f, u, g, v, tmp);
        free(g);
        free(v);
        free(tmp);
    }
}

/* One 3D V-cycle on level l: u = T_l f, zero initial guess. */
static void smg_vcycle(const orc_smg *h, int l, const double *f, double *u)
{
    int nx = h->nx, ny = h->ny, nzl = h->nz_l[l];
    size_t np = (size_t)nx * (size_t)ny, nl = np * (size_t)nzl;
    double *g = (double *)malloc(sizeof(double) * np);
    double *v = (double *)malloc(sizeof(double) * np);
    double *tmp = (double *)malloc(sizeof(double) * np);
    memset(u, 0, sizeof(double) * nl);
    if (l == h->L - 1) { /* coarsest level: one plane */
        for (int it = 0; it < h->coarse_iters; ++it)
            for (int z = 0; z < nzl; ++z) plane_relax(h, l, z, f, u, g, v, tmp);
        free(g);
        free(v);
        free(tmp);
        return;
    }
    for (int s = 0; s < h->npre; ++s) {
        relax_colour(h, l, 0, f, u);
        relax_colour(h, l, 1, f, u);
    }
    /* residual r = f - A_l u and restriction f_c = P^T r */
    double *r = (double *)malloc(sizeof(double) * nl);
#ifdef _OPENMP
#pragma omp parallel if (nzl > 2)
#endif
    {
        double *gz = (double *)malloc(sizeof(double) * np);
        double *tz = (double *)malloc(sizeof(double) * np);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int z = 0; z < nzl; ++z) {
            level_apply_plane(h, l, z, u, gz, tz);
            for (size_t i = 0; i < np; ++i) r[(size_t)z * np + i] = f[(size_t)z * np + i] - gz[i];
        }
        free(gz);
        free(tz);
    }
    int nzc = h->nz_l[l + 1];
    double *fc = (double *)calloc(np * (size_t)nzc, sizeof(double));
    double *uc = (double *)calloc(np * (size_t)nzc, sizeof(double));
    /* every point sums its fine planes in plane order (the order does not depend on threads) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (size_t i = 0; i < np; ++i)
        for (int z = 0; z < nzl; ++z) {
            int cj[2];
            double cw[2];
            int cnt = prolong_row(z, nzl, h->wm[l], h->wp[l], cj, cw);
            for (int p = 0; p < cnt; ++p) fc[(size_t)cj[p] * np + i] += cw[p] * r[(size_t)z * np + i];
        }
    smg_vcycle(h, l + 1, fc, uc);
    /* prolongation and correction u += P u_c */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (size_t i = 0; i < np; ++i)
        for (int z = 0; z < nzl; ++z) {
            int cj[2];
            double cw[2];
            int cnt = prolong_row(z, nzl, h->wm[l], h->wp[l], cj, cw);
            for (int p = 0; p < cnt; ++p) u[(size_t)z * np + i] += cw[p] * uc[(size_t)cj[p] * np + i];
        }
    for (int s = 0; s < h->npost; ++s) {
        relax_colour(h, l, 1, f, u);
        relax_colour(h, l, 0, f, u);
    }
    free(r);
    free(fc);
    free(uc);
    free(g);
    free(v);
    free(tmp);
}

/* Threads the oracle's loops may use (OpenMP builds; 1 = plain sequential execution).  The results
   do not depend on it: every parallel loop writes disjoint outputs whose values are computed in a
   fixed order. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_smg_apply(const orc_smg *h, const double *r, double *s)
{
    smg_vcycle(h, 0, r, s);
    if (h->learned) {
        /* the learned post-correction of net_oracle.c; the counters are bookkeeping only */
        orc_smg *hm = (orc_smg *)h;
        hm->learned_calls += 1;
        hm->learned_accepted += orc_learned_correct(h->nx, h->ny, h->nz, h->learned, r, s);
    }
}

int orc_smg_set_learned(orc_smg *h, const double *w)
{
    if (!h) return -1;
    free(h->learned);
    h->learned = NULL;
    h->learned_calls = h->learned_accepted = 0;
    if (w) {
        h->learned = (double *)malloc(sizeof(double) * ORC_NET_WEIGHTS);
        memcpy(h->learned, w, sizeof(double) * ORC_NET_WEIGHTS);
    }
    return 0;
}

void orc_smg_learned_stats(const orc_smg *h, long long *calls, long long *accepted)
{
    *calls = h->learned_calls;
    *accepted = h->learned_accepted;
}

int orc_smg_num_levels(const orc_smg *h) { return h->L; }
int orc_smg_level_nz(const orc_smg *h, int l) { return h->nz_l[l]; }

void orc_smg_level_coefs(const orc_smg *h, int l, double *M, double *K, double *wm, double *wp)
{
    for (int z = 0; z < h->nz_l[l]; ++z) {
        for (int k = 0; k < 3; ++k) {
            M[3 * z + k] = tri_get(&h->M[l], z, z + k - 1);
            K[3 * z + k] = tri_get(&h->K[l], z, z + k - 1);
        }
        wm[z] = h->wm[l][z];
        wp[z] = h->wp[l][z];
    }
}

int orc_smg_plane_num_levels(const orc_smg *h) { return h->ph[0][0].nlev; }
int orc_smg_plane_level_ny(const orc_smg *h, int m) { return h->ph[0][0].ny[m]; }

void orc_smg_plane_coefs(const orc_smg *h, int l, int z, int m,
                         double *S, double *T, double *wm, double *wp)
{
    const plane_h *ph = &h->ph[l][z];
    for (int y = 0; y < ph->ny[m]; ++y) {
        for (int k = 0; k < 3; ++k) {
            S[3 * y + k] = tri_get(&ph->S[m], y, y + k - 1);
            T[3 * y + k] = tri_get(&ph->T[m], y, y + k - 1);
        }
        wm[y] = ph->wm[m][y];
        wp[y] = ph->wp[m][y];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1: PSD and PCG with beta from eq. (1) or eq. (2)                            */
/* ------------------------------------------------------------------------------------ */

static double dot(size_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

int orc_krylov(const orc_smg *h, int nx, int ny, int nz, int variant,
               const double *b, double *x, double tol, int maxit,
               int *iters, double *relres, double *hist, double *xs, double *rs)
{
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    double *r = (double *)malloc(sizeof(double) * n);
    double *s = (double *)malloc(sizeof(double) * n);
    double *p = (double *)calloc(n, sizeof(double));
    double *q = (double *)malloc(sizeof(double) * n);
    double *dr = (double *)calloc(n, sizeof(double)); /* r_k - r_{k-1} (eq. (2)) */
    int status = -3, k = 0, restart = 1;
    double rho_prev = 0.0;

    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    orc_apply_A(nx, ny, nz, x, q);
    for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];

    for (k = 0;; ++k) {
        double rn = sqrt(dot(n, r, r));
        if (hist) hist[k] = rn / bn;
        if (xs) memcpy(xs + (size_t)k * n, x, sizeof(double) * n);
        if (rs) memcpy(rs + (size_t)k * n, r, sizeof(double) * n);
        if (!isfinite(rn)) {
            status = -6;
            break;
        }
        if (rn / bn <= tol) {
            /* confirm with the true residual; if it fails, continue from it (restart) */
            orc_apply_A(nx, ny, nz, x, q);
            double tn = 0.0;
            for (size_t i = 0; i < n; ++i) {
                double t = b[i] - q[i];
                tn += t * t;
            }
            if (sqrt(tn) / bn <= tol) {
                status = 0;
                break;
            }
            for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
            restart = 1;
        }
        if (k >= maxit) {
            status = -3;
            break;
        }
        /* s_k = T r_k */
        if (h)
            orc_smg_apply(h, r, s);
        else
            memcpy(s, r, sizeof(double) * n);
        double rho = dot(n, s, r);
        double beta = 0.0;
        if (!restart && variant != 2) {
            if (rho_prev == 0.0) {
                status = -4;
                break;
            }
            if (variant == 0)
                beta = rho / rho_prev;                 /* eq. (1) */
            else
                beta = dot(n, s, dr) / rho_prev;       /* eq. (2) */
        }
        for (size_t i = 0; i < n; ++i) p[i] = s[i] + beta * p[i];
        orc_apply_A(nx, ny, nz, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) {
            status = (pq == pq) ? -4 : -6;
            break;
        }
        double alpha = rho / pq;
        for (size_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            double rnew = r[i] - alpha * q[i];
            dr[i] = rnew - r[i];
            r[i] = rnew;
        }
        rho_prev = rho;
        restart = 0;
    }

    orc_apply_A(nx, ny, nz, x, q);
    double tn = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double t = b[i] - q[i];
        tn += t * t;
    }
    *iters = k;
    *relres = sqrt(tn) / bn;
    free(r);
    free(s);
    free(p);
    free(q);
    free(dr);
    return status;
}
