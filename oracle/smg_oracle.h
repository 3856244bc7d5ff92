/*
 * smg_oracle.h -- plain FP64 CPU oracle for the SMG-preconditioned Krylov solvers of
 * Bouwmeester, Dougherty, Knyazev, "Nonsymmetric multigrid preconditioning for conjugate
 * gradient methods" (arXiv:1212.6680).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * code; only the test suite, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Grid convention: interior points of an nx x ny x nz brick, index (z*ny + y)*nx + x,
 * x fastest, spacing 1, homogeneous Dirichlet boundary (values outside the brick are 0).
 */
#ifndef SMG_ORACLE_H
#define SMG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_smg orc_smg;

/* Model operator: 7-point negative Laplacian, section "PSD and PCG methods" (model problem). */
void orc_apply_A(int nx, int ny, int nz, const double *u, double *out);

/* Thomas algorithm for a general tridiagonal system
 *   a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],  i = 0..n-1  (a[0], c[n-1] ignored). */
void orc_thomas(int n, const double *a, const double *b, const double *c,
                const double *d, double *x);

/* SMG hierarchy (section "Preconditioning with SMG"; the reading of its internals is the one
 * documented in smg_oracle.c).  Returns NULL on bad arguments. */
orc_smg *orc_smg_setup(int nx, int ny, int nz, int npre, int npost, int coarse_iters);
void orc_smg_free(orc_smg *h);
/* s = T r : one V-cycle with zero initial guess. */
void orc_smg_apply(const orc_smg *h, const double *r, double *s);

/* Introspection for the Galerkin / interpolation pins. */
int orc_smg_num_levels(const orc_smg *h);
int orc_smg_level_nz(const orc_smg *h, int l);
/* M, K: [nz_l][3] entries (z, z-1), (z, z), (z, z+1); wm, wp: [nz_l] interpolation weights. */
void orc_smg_level_coefs(const orc_smg *h, int l, double *M, double *K, double *wm, double *wp);
int orc_smg_plane_num_levels(const orc_smg *h);
int orc_smg_plane_level_ny(const orc_smg *h, int m);
/* S, T: [ny_m][3] entries (y, y-1), (y, y), (y, y+1); wm, wp: [ny_m]. */
void orc_smg_plane_coefs(const orc_smg *h, int l, int z, int m,
                         double *S, double *T, double *wm, double *wp);

/* The 2D plane cycle alone, for the plane operator c*L2D + d*I on an nx x ny plane:
 * v = C g (one 2D V-cycle, zero initial guess). */
void orc_plane_cycle(int nx, int ny, double c, double d, const double *g, double *v);

/* Algorithm 1 with beta from eq. (1) (variant 0, standard PCG), eq. (2) (variant 1, flexible
 * PCG) or beta = 0 (variant 2, PSD).  h == NULL means T = I (no preconditioner).
 * x holds x0 on entry and the last iterate on exit.  iters, relres (true residual) always
 * written.  hist (optional, maxit+1 entries) receives ||r_k||/||b|| of the recurrence.
 * xs, rs (optional, (maxit+1)*N each) receive the iterates x_k and residuals r_k.
 * Returns 0 converged, -3 not converged in maxit, -4 breakdown, -6 NaN/Inf. */
int orc_krylov(const orc_smg *h, int nx, int ny, int nz, int variant,
               const double *b, double *x, double tol, int maxit,
               int *iters, double *relres, double *hist, double *xs, double *rs);

#ifdef __cplusplus
}
#endif
#endif
