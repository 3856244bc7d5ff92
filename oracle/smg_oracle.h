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
/* Threads the oracle may use (built with OpenMP: the planes of a colour, the lines of a colour,
 * the points of a transfer are shared among threads; every output is computed in a fixed order,
 * so results are bitwise independent of the count).  n >= 1 sets it; returns the count in force. */
int orc_set_threads(int n);

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

/* ---- learned post-correction (net_oracle.c; not in the paper) ---------------------------- */
#define ORC_NET_WEIGHTS 7776 /* 16*1*27 + 16*16*27 + 1*16*27 */

/* 3x3x3 convolution (cross-correlation), zero padding, no bias.  w: [cout][cin][27],
 * tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); in: [cin][N]; out: [cout][N]. */
void orc_conv3d(int nx, int ny, int nz, int cin, int cout, const double *w, const double *in, double *out);
/* Its adjoint in the input: gin = conv^T gout. */
void orc_conv3d_adj(int nx, int ny, int nz, int cin, int cout, const double *w, const double *gout, double *gin);
/* Its gradient in the weights of sum <gout, out>. */
void orc_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const double *in, const double *gout, double *gw);
/* delta = rms(rho) * Net(rho / rms(rho)). */
void orc_net_forward(int nx, int ny, int nz, const double *w, const double *rho, double *delta);
/* L = (e - delta)^T A (e - delta) / e^T A e and, if grad != NULL, dL/dw (7776). */
double orc_net_loss_grad(int nx, int ny, int nz, const double *w, const double *rho, const double *e, double *grad);
/* The same two with the hidden activations rounded to BF16 when act_bf16 = 1. */
void orc_net_forward_ex(int nx, int ny, int nz, const double *w, const double *rho, double *delta, int act_bf16);
double orc_net_loss_grad_ex(int nx, int ny, int nz, const double *w, const double *rho, const double *e, double *grad,
                            int act_bf16);
/* Round to binary32, then to the nearest BF16 (ties to even). */
double orc_round_bf16(double v);
/* s += delta(r - A s) when the judge accepts it; returns 1 if accepted. */
int orc_learned_correct(int nx, int ny, int nz, const double *w, const double *r, double *s);
/* Attach (w != NULL, copied) or detach (NULL) the learned post-correction of a handle:
 * orc_smg_apply then returns s0 + delta or s0 as the judge decides. */
int orc_smg_set_learned(orc_smg *h, const double *w);
void orc_smg_learned_stats(const orc_smg *h, long long *calls, long long *accepted);

#ifdef __cplusplus
}
#endif
#endif
