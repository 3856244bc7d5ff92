/*
 * smg.h -- C ABI of libsmg: SMG-preconditioned PCG / flexible PCG / PSD and LOBPCG for the
 * 7-point 3D Dirichlet Laplacian, on one GB300 GPU (sm_103a).
 *
 * Method: Bouwmeester, Dougherty, Knyazev, "Nonsymmetric multigrid preconditioning for
 * conjugate gradient methods", arXiv:1212.6680.
 *   - Algorithm 1 (section "PSD and PCG methods"), beta from eq. (1) (standard PCG),
 *     eq. (2) (flexible PCG) or beta = 0 (PSD).
 *   - SMG preconditioner T with -v npre npost relaxation (section "Preconditioning with SMG").
 *   - LOBPCG preconditioned by SMG (section "Preconditioning of LOBPCG with SMG").
 * The model problem (section "PSD and PCG methods"): negative Laplacian, 7-point stencil,
 * grid spacing one, homogeneous Dirichlet boundary, on the interior points of an
 * nx x ny x nz brick.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Layout.  A grid vector holds N = nx*ny*nz doubles, index (z*ny + y)*nx + x (x fastest).
 *           A block of m vectors is column-major N x m: vector j starts at element j*N.
 *  Memory.  Vector pointers are caller-owned.  Unless an entry point says otherwise they are
 *           device pointers (e.g. PyTorch CUDA tensors) on the current device.  The handle owns
 *           the hierarchy and all scratch space; smg_setup allocates them and smg_destroy
 *           frees them.
 *  Streams. `stream` is a cudaStream_t (NULL = the legacy default stream).  Work on one handle
 *           is stream-ordered.  A handle is not thread-safe: one host thread at a time.
 *  Errors.  Every entry point returns SMG_OK (0) or a negative SMG_ERR_* code.  Invalid
 *           arguments return SMG_ERR_ARG before anything is launched or written.
 *           smg_last_error() gives a message for the calling thread's last failure.
 */
#ifndef SMG_H
#define SMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smg_ctx *smg_handle; /* opaque; owns the hierarchy and workspace */

enum {
    SMG_OK = 0,
    SMG_ERR_ARG = -1,       /* invalid argument; nothing was launched */
    SMG_ERR_CUDA = -2,      /* a CUDA call failed (message in smg_last_error) */
    SMG_ERR_NOCONV = -3,    /* maxit reached; the last iterate is returned */
    SMG_ERR_BREAKDOWN = -4, /* (p, Ap) <= 0 or (s_{k-1}, r_{k-1}) = 0 in Algorithm 1 */
    SMG_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    SMG_ERR_NAN = -6,       /* NaN or Inf met in a residual norm or inner product */
    SMG_ERR_HOST = -7       /* a host allocation failed (message in smg_last_error) */
};

enum { SMG_PCG = 0, SMG_FPCG = 1, SMG_PSD = 2 };       /* eq. (1), eq. (2), beta = 0 */
enum { SMG_FP64 = 0, SMG_FP32 = 1, SMG_BF16 = 2 };     /* V-cycle storage precision */

/* Options for smg_set_option. */
enum {
    SMG_OPT_COARSE_ITERS = 0, /* plane-cycle steps on the one-plane coarsest level (>= 1, default 1) */
    SMG_OPT_THREADS = 1,      /* threads per CTA of the plane-relaxation kernels: 256 or 512
                                 (default 512; the shortened-step kernel with FP64 compute and the
                                 wide-line kernel with FP32 compute use at most 384, for registers) */
    SMG_OPT_PROFILE = 2,      /* time plane-relaxation launches with CUDA events: 0 off,
                                 1 the finest level's launches only, 2 every launch */
    SMG_OPT_CLUSTER_MAX = 3,  /* largest thread-block cluster (CTAs per plane) for the FP64
                                 plane relaxations: 1, 2, 4, 8 or 16 (default 16; levels other
                                 than the one-plane coarsest use at most 8) */
    SMG_OPT_CLUSTER_MAX32 = 4, /* the same for the FP32-compute plane relaxations of the FP32 and
                                 BF16 cycles: 1, 2, 4, 8 or 16, or 0 (default) for 8 with x-lines
                                 split over several warps, else 1 while a plane's 2D-cycle iterate
                                 fits in one CTA's shared memory and 4 when it does not */
    SMG_OPT_PRECOND = 5,      /* the preconditioner krylov_solve applies: 1 (default) the SMG cycle,
                                 0 none (T = I: plain CG by eq. (1) or (2), steepest descent for PSD;
                                 section 2, figures 1-2); lobpcg_solve always uses the cycle */
    SMG_OPT_LEAN = 6,         /* 1 (default): plane relaxations with x-lines of at most 256 rows
                                 whose layout keeps every 2D level's factor sets on chip (FP32 or
                                 FP64 compute, one CTA or a cluster per plane) run the 2D cycle
                                 with fewer barrier-separated steps (the restriction fused with the
                                 next level's even lines; the same line solves in the same order,
                                 bit-identical), and the wide-line kernel (longer x-lines) runs its
                                 cycle in the same shortened step order (bit-identical); 0: the
                                 general kernel and the general step order */
    SMG_OPT_GRAM_TC = 7,      /* lobpcg_solve's Gram products with both block widths >= value (and
                                 <= 64) run on the tensor cores (smg_gram's digit splitting); the
                                 others, and all of them with value 0, on the CUDA cores in
                                 double-float arithmetic (default 16) */
    SMG_OPT_GRAPH = 8,        /* 1 (default): krylov_solve runs its iterations as one CUDA graph
                                 whose conditional while node repeats V-cycle + Krylov kernels on
                                 the device until the recurrence residual meets tol, maxit is
                                 reached or a breakdown is flagged (the host then checks the true
                                 residual as in the host loop); the graph is rebuilt after any
                                 option, precision or weight change and when x changes.  Not used
                                 with the learned correction, pair capture or profiling.  0: the
                                 host launches every iteration and reads the scalars after each */
    SMG_OPT_FUSED_TAIL = 9    /* 1: the Krylov part of an iteration (Algorithm 1's dots, p update,
                                 A p and x/r update) runs as one cooperative kernel with bounded
                                 grid-wide barriers between its phases when its CTAs all fit on the
                                 GPU (nx % 4 == 0, aligned vectors); bit-identical to 0 (default),
                                 four kernels chained by programmatic dependent launch, which is
                                 faster on GB300 (the barriers cost more than the kernel
                                 boundaries).  A barrier wait that gives up returns SMG_ERR_TIMEOUT
                                 from krylov_solve */,
    SMG_OPT_SOLO = 10         /* T in [0, 512] (default 8): when the shortened-step plane cycle
                                 runs on a thread-block cluster, the 2D levels of at most T lines
                                 are held whole by the cluster's first CTA, whose steps on them
                                 end in a CTA barrier instead of a cluster barrier; the same
                                 results as 0 (every level spread over the cluster) */,
    SMG_OPT_RESTRICT_COLUMN = 11 /* 1 (default): with FP64 storage, or from 4M coarse points per
                                 launch, each thread of the residual + restriction walks four
                                 coarse planes, computing each fine residual (and each plane's
                                 in-plane stencil) once; smaller FP32 / BF16 launches, and every
                                 launch with 0, use one coarse plane per thread, recomputing the
                                 residual of every even fine plane for both coarse planes it
                                 feeds.  Bit-identical results */,
    SMG_OPT_WIDE_FACTORS = 12 /* 1 (default): planes whose x-lines run on the wide-line kernel
                                 (see SMG_OPT_WIDE_MIN_ROWS) read the line solver's data of every
                                 2D level's two line matrices (segment factors, the segments'
                                 responses to their end values, the reduced system's rows) from
                                 tables formed once, in the compute precision, when the level
                                 vectors are allocated, one per class of planes with equal
                                 coefficients (smg_plane_classes; the coarsest level always, the
                                 others while the tables take at most 512 MB); 0: formed inside the plane
                                 cycle at every change of line matrix.  Bit-identical results */,
    SMG_OPT_WIDE_MIN_ROWS = 13 /* 257 (default) or 513: x-lines of at least this many rows (and at
                                 most 512) are split over two warps of 8 rows per lane (the
                                 wide-line kernel, with its clusters and tables) instead of one
                                 warp of 16 (the general plane cycle); lines longer than 512 rows
                                 always take the wide-line kernel.  The two differ by rounding */
};

/*
 * smg_setup -- build the SMG hierarchy for the nx x ny x nz brick (section "Preconditioning
 * with SMG": -v npre npost).  npre >= 1 pre-relaxation sweeps, npost >= 0 post-relaxation
 * sweeps (npost = 0 is the paper's nonsymmetric "no post-relaxation" cycle).  The hierarchy
 * is computed on the host in FP64 (z-semicoarsening, Galerkin coarse operators, per-plane
 * y-hierarchies) and copied to the current device; work vectors for one right-hand side are
 * allocated.  Sizes: 1 <= nx <= 2048, 1 <= ny <= 512, 1 <= nz <= 4096.  x-lines of up to 256
 * rows are solved by one warp; longer ones (the paper's 16n x n x n bricks up to n = 128) are cut
 * into segments of 256 rows (lines of 257-512 rows) or 512 rows (longer lines), one warp each,
 * joined exactly through a reduced system of the segment ends (SMG_OPT_WIDE_MIN_ROWS = 513 keeps
 * lines of up to 512 rows on one warp); a plane of such lines runs on one CTA or on a cluster of
 * CTAs that own its lines in pairs, without the shortened-step cycle.  *out receives the handle.
 * The cycle precision starts as SMG_FP64.
 */
int smg_setup(int nx, int ny, int nz, int npre, int npost, smg_handle *out);

/* smg_set_precision -- storage precision of the V-cycle: SMG_FP64, SMG_FP32 or SMG_BF16.
 * FP32 computes in FP32; BF16 stores level vectors in bfloat16 and computes in FP32.  The
 * one-plane coarsest level always computes in FP64.  Krylov recurrences, inner products and
 * norms stay FP64. */
int smg_set_precision(smg_handle h, int prec);

/* smg_set_option -- set one SMG_OPT_* option (see the enum). */
int smg_set_option(smg_handle h, int option, int value);

/*
 * smg_apply -- s = T r, one V-cycle with zero initial guess (the preconditioner of
 * Algorithm 1).  r and s: device, N doubles each, must not overlap.
 */
int smg_apply(smg_handle h, const double *r, double *s, void *stream);

/*
 * smg_apply_batched -- S = T R for nb right-hand sides at once (R, S: device, N x nb
 * column-major).  All nb cycles run in the same launches.  1 <= nb <= 64.
 */
int smg_apply_batched(smg_handle h, int nb, const double *R, double *S, void *stream);

/* smg_apply_A -- out = A u, the 7-point operator in FP64 (device, N doubles each). */
int smg_apply_A(smg_handle h, const double *u, double *out, void *stream);

/*
 * krylov_solve -- Algorithm 1 with T = SMG: variant SMG_PCG (eq. (1)), SMG_FPCG (eq. (2)) or
 * SMG_PSD (beta = 0).  x holds x0 on entry and the solution on exit.  Stops when the FP64 true
 * residual satisfies ||b - A x||_2 <= tol ||b||_2 (the recurrence residual is tested first;
 * if the true residual then fails, the solver continues from it with beta = 0).
 * b and x may be device pointers or host pointers (pageable or pinned); for host pointers
 * the library copies b and x0 to the device and x back, inside the call, and returns after
 * the copy back.  *iters (preconditioner applications) and *relres (true relative residual)
 * are always written.  Returns SMG_ERR_NOCONV after maxit iterations (last iterate in x).
 * tol > 0, maxit >= 0.  Synchronises `stream` once per iteration (8-byte residual readback).
 */
int krylov_solve(smg_handle h, int variant, const double *b, double *x, double tol, int maxit,
                 int *iters, double *relres, void *stream);

/*
 * lobpcg_solve -- the m smallest eigenpairs of A by LOBPCG preconditioned with T (section
 * "Preconditioning of LOBPCG with SMG"; m = 1 in the paper).  X (device, N x m column-major)
 * holds the initial block on entry and the eigenvector approximations on exit; lambda (host,
 * m doubles) receives the Ritz values in ascending order.  Converged when every column has
 * ||A x_i - lambda_i x_i||_2 <= tol * lambda_i * ||x_i||_2.  1 <= m <= 64, 3m <= N.
 */
int lobpcg_solve(smg_handle h, int m, double *X, double *lambda, double tol, int maxit,
                 int *iters, void *stream);

/*
 * Batched solver: nsys independent systems, each the model problem on its own brick
 * (dims[3s], dims[3s+1], dims[3s+2] = nx, ny, nz of system s), solved together by Algorithm 1
 * (PCG eq. (1), flexible PCG eq. (2) or PSD) preconditioned by SMG with -v npre npost.  Per
 * iteration, one CUDA graph runs one persistent kernel that performs every step of every
 * system's V-cycle (levels aligned from the finest, a bounded grid barrier between steps) and
 * the FP64 Krylov kernels of all systems; converged systems are masked out on the device.
 *
 * smg_batched_setup -- builds the hierarchies, allocates every buffer, chooses the schedule
 * (threads per CTA, task order within a step) by timing one V-cycle per candidate (cached per
 * set of grids for the life of the process) and captures the per-iteration graph.
 *   dims:  host, 3*nsys ints; 1 <= nx <= 128, 1 <= ny <= 512, 1 <= nz <= 4096; 1 <= nsys <= 4096.
 *   npre, npost: 1 <= npre <= 8, 0 <= npost <= 8.
 *   prec:  SMG_FP32 (FP32 cycle, FP64 coarsest plane, FP64 Krylov); others return SMG_ERR_ARG.
 *   *out:  receives the handle (NULL on failure).  Synchronises `stream`.
 *
 * smg_batched_solve -- one solve of all systems.
 *   b, x:   host arrays of nsys device pointers (system s has nx*ny*nz doubles, layout as
 *           smg_apply); x holds x0 on entry.  Caller-owned.
 *   iters:  host, nsys ints, always written (preconditioner applications per system).
 *   relres: host, nsys doubles (NULL allowed): final true relative residual per system.
 * Stops each system at ||b - A x||_2 <= tol ||b||_2 (true residual); returns SMG_ERR_NOCONV
 * when some system did not reach it in maxit iterations, SMG_ERR_TIMEOUT when a grid-barrier
 * wait gave up, SMG_ERR_BREAKDOWN / SMG_ERR_NAN as krylov_solve.  Synchronises `stream` once
 * per iteration.  Calls on one handle must not overlap.
 *
 * smg_batched_apply -- s_s = T_s r_s for every system s: one application of each system's SMG
 *   V-cycle (section 3: the fixed, linear preconditioner of Algorithm 1) with the handle's
 *   npre/npost, storage precision and tuned schedule, all systems together in exactly one launch
 *   of the persistent V-cycle kernel -- the launch each iteration of smg_batched_solve makes.
 *   r, s:   host arrays of nsys device pointers (system s: nx*ny*nz doubles, layout as
 *           smg_apply); r is rounded to the storage precision on entry, s receives the cycle's
 *           output widened exactly to FP64.  Caller-owned.
 *   Returns SMG_ERR_TIMEOUT when a grid-barrier wait gave up.  Synchronises `stream`.  Calls on
 *   one handle must not overlap (the handle's level vectors are shared).
 *
 * smg_batched_destroy -- frees the handle (NULL accepted).  Synchronises the device.
 */
typedef struct smg_batched_ctx *smg_batched_handle;
int smg_batched_setup(int nsys, const int *dims, int npre, int npost, int prec, smg_batched_handle *out,
                      void *stream);
int smg_batched_solve(smg_batched_handle h, int variant, const double *const *b, double *const *x, double tol,
                      int maxit, int *iters, double *relres, void *stream);
int smg_batched_apply(smg_batched_handle h, const double *const *r, double *const *s, void *stream);
int smg_batched_destroy(smg_batched_handle h);

/*
 * smg_batched_info -- the schedule the set-up's autotuner chose by timing every candidate
 * V-cycle: x-line tile (rows_per_lane K: a warp holds 32 K rows of a line, K from the narrowest
 * that holds every system's lines up to 4), threads per CTA (256 or 512), persistent CTAs
 * (`blocks`: a multiple of the SM count, 1 up to the occupancy limit per SM) and task order
 * (0 system order, 1 longest plane first); also the tasks per V-cycle and the kernel launches the
 * handle has issued so far (the persistent V-cycle counts once per launch).  Host outputs.
 */
int smg_batched_info(smg_batched_handle h, int *threads, int *order, int *blocks, long long *tasks,
                     long long *launches, int *rows_per_lane);

/*
 * smg_batched_set_profile / smg_batched_profile_read -- with profiling on, each iteration's
 * graph replay is timed by its event nodes: class 0 the persistent V-cycle kernel, class 1 the
 * Krylov kernels.  Read returns replays, total device milliseconds and, for class 0, the
 * algorithmic bytes of the V-cycles performed (storage words each active system's cycle must
 * read and write: 2.5 words per point per relaxation sweep, 5 per point for residual +
 * restriction + prolongation, 2 per point on the coarsest plane); reading resets the class.
 */
int smg_batched_set_profile(smg_batched_handle h, int on);
int smg_batched_profile_read(smg_batched_handle h, int which, long long *launches, double *ms, double *bytes);

/*
 * krylov_solve_batched -- one-shot form: smg_batched_setup, smg_batched_solve with flexible PCG
 * (eq. (2)) and relres = NULL, smg_batched_destroy.  Arguments as above.
 */
int krylov_solve_batched(int nsys, const int *dims, int npre, int npost, int prec, const double *const *b,
                         double *const *x, double tol, int maxit, int *iters, void *stream);

/*
 * smg_barrier_selftest -- runs a small persistent kernel of 4 CTAs whose grid barrier waits for
 * 4 + extra_blocks CTAs, with a wait limit of about limit_seconds (0 < limit_seconds <= 10).
 * *status (host) receives SMG_OK when the barriers complete (extra_blocks = 0) and
 * SMG_ERR_TIMEOUT when a wait gave up (extra_blocks > 0): the failure path of the barrier that
 * krylov_solve_batched relies on, exercised without faulting or hanging the device.
 */
int smg_barrier_selftest(int extra_blocks, double limit_seconds, int *status, void *stream);

/*
 * Learned post-correction (not in the paper; eq. (2), flexible PCG, is what admits a nonlinear
 * preconditioner, and PSD admits one too).  After the SMG cycle s0 = T r, the residual
 * rho = r - A s0 goes through a small network -- 3x3x3 convolutions 1 -> 16 -> 16 -> 1 channels,
 * zero padding, no bias, ReLU after the first two layers, input divided by its RMS and output
 * multiplied back -- giving delta; the result is s0 + delta when ||rho - A delta||_2 < ||rho||_2
 * and s0 otherwise.  Weights: SMG_NET_WEIGHTS values, layer 1 [16][1][27], layer 2 [16][16][27],
 * layer 3 [1][16][27], each [out channel][in channel][tap], tap (dz+1)*9 + (dy+1)*3 + (dx+1)
 * weighting the input at (x+dx, y+dy, z+dz).  Activations are BF16 with FP32 accumulation
 * (SMG_FP32 activations are offered by the handle-free calls for accuracy checks).
 */
#define SMG_NET_WEIGHTS 7776

/* smg_set_learned -- attach (enable = 1) the correction with weights_bf16 (host, SMG_NET_WEIGHTS
 * BF16 bit patterns, copied) to every smg_apply and krylov_solve of the handle, or detach it
 * (enable = 0, weights ignored).  Meant for handles with npost = 0.  Resets the judge counters. */
int smg_set_learned(smg_handle h, const void *weights_bf16, int enable);

/* smg_learned_stats -- how many corrections were computed and how many the judge kept (host
 * outputs; synchronises the device). */
int smg_learned_stats(smg_handle h, long long *calls, long long *accepted);

/*
 * smg_collect_pairs -- training pairs along one flexible PCG solve of A x = b from x0 = 0 with
 * the handle's cycle: before the k-th update, with s_k = T r_k,
 *   rho_out[k] = r_k - A s_k   and   e_out[k] = xstar - x_k - s_k     (FP32, N values each),
 * so that e_out[k] is the error left after the cycle when xstar solves A x = b.  b, xstar: device
 * FP64; rho_out, e_out: device, max_pairs * N floats.  *npairs (host) receives the number of pairs
 * written (at most max_pairs).  Stops at tol or maxit like krylov_solve; not converging is not
 * an error here.
 */
int smg_collect_pairs(smg_handle h, const double *b, const double *xstar, double tol, int maxit, float *rho_out,
                      float *e_out, int max_pairs, int *npairs, void *stream);

/* smg_net_forward -- delta = rms(rho) Net(rho / rms(rho)) on an nx x ny x nz grid.  w: host
 * FP32 [SMG_NET_WEIGHTS] (rounded to BF16 when act_prec = SMG_BF16); rho, delta: device FP64.
 * act_prec: SMG_BF16 or SMG_FP32 activations.  Synchronises `stream`. */
int smg_net_forward(int nx, int ny, int nz, int act_prec, const float *w, const double *rho, double *delta,
                    void *stream);

/* smg_net_loss_grad -- L = (e - delta)^T A (e - delta) / e^T A e for delta = the network's
 * correction of rho, and dL/dw.  rho, e: device FP64; *loss: host; grad: host FP32
 * [SMG_NET_WEIGHTS].  Synchronises `stream`. */
int smg_net_loss_grad(int nx, int ny, int nz, int act_prec, const float *w, const double *rho, const double *e,
                      double *loss, float *grad, void *stream);

/* smg_net_train -- Adam (beta 0.9, 0.999, eps 1e-8, step size lr) over npairs pairs, one pair per
 * step, `epochs` passes in an order shuffled from `seed`.  dims: host, 3 ints per pair; rho[i],
 * e[i]: device FP32 arrays of pair i (layout of smg_collect_pairs).  w: host FP32
 * [SMG_NET_WEIGHTS], initial weights in, trained weights out.  loss_hist: host, `epochs` mean
 * losses.  Synchronises `stream` once per epoch. */
int smg_net_train(int npairs, const int *dims, const float *const *rho, const float *const *e, int epochs, double lr,
                  unsigned long long seed, int act_prec, float *w, double *loss_hist, void *stream);

/* smg_net_set_tensor_cores -- process-wide choice for the BF16 16 -> 16 channel layer: 1 (the
 * default) runs it on the tcgen05 tensor cores, 0 on the CUDA cores (FP32 FMAs, the same BF16
 * inputs and rounding).  Takes effect at the next launch; not for concurrent use with solves. */
int smg_net_set_tensor_cores(int on);

/* smg_net_tc_status -- *err (host) = 1 if a tensor-core layer launch gave up waiting for its
 * accumulators (bounded wait; its output is then incomplete) since the last call, else 0; clears
 * the flag.  Synchronises the device. */
int smg_net_tc_status(int *err);

/* smg_destroy -- free the handle and everything it owns (NULL is accepted). */
int smg_destroy(smg_handle h);

/* smg_last_error -- message of the calling thread's last failed call ("" if none). */
const char *smg_last_error(void);

/*
 * smg_profile_read -- when SMG_OPT_PROFILE is on, the plane-relaxation launches timed so far
 * on this handle: launches, total device milliseconds (CUDA events on the launch stream) and
 * algorithmic bytes (vector elements the launches must read and write), by class `which`:
 * 0 plane relaxation on the finest level, 1 plane relaxation on the other levels except the
 * coarsest, 2 the one-plane coarsest solve, 3 restriction and prolongation, 4 the Krylov
 * kernels of each iteration, 5 the learned post-correction of each iteration (its "bytes" are
 * the convolutions' flops, 2 x 27 x 288 per point) (classes 1-4 are timed only with
 * SMG_OPT_PROFILE = 2; classes 0 and 5 with either 1 or 2).
 * Reading resets the counters of that class.  Synchronises the device.
 */
int smg_profile_read(smg_handle h, int which, long long *launches, double *ms, double *bytes);

/*
 * smg_check_conversions -- diagnostic for the library's own FP32 <-> FP64 conversions (the
 * paper has no counterpart; the conversions are the ones the mixed-precision cycle and the
 * Krylov kernels use).  For each of the n device doubles in src it compares the integer-pipe
 * narrowing (round to nearest even) with the hardware conversion, and the widening of the
 * rounded value with the hardware widening, bit for bit.  mismatches: device int[2], set to the
 * narrowing and widening mismatch counts.  Asynchronous on `stream`.
 */
int smg_check_conversions(long long n, const double *src, int *mismatches, void *stream);

/*
 * smg_krylov_history -- the relative recurrence residuals ||r_k||_2 / ||b||_2, k = 0 .. iters, of
 * the handle's last krylov_solve (the quantity figures 2 and 5 of section 3 plot, in the 2-norm):
 * entry k is read at the top of iteration k, before the stopping test (a restart from the true
 * residual keeps the recurrence value of that step).  Copies min(max, count) values into hist
 * (host) and sets *count (host) to the number recorded.
 */
int smg_krylov_history(smg_handle h, double *hist, int max, int *count);

/* smg_launch_count -- number of CUDA kernel launches this handle has issued so far. */
int smg_launch_count(smg_handle h, long long *count);

/*
 * smg_gram -- G = U^T V for tall-skinny blocks in FP64 accuracy on the tensor cores: the dense
 * inner products of block LOBPCG (section 4, "Preconditioning of LOBPCG with SMG": the
 * Rayleigh-Ritz matrices S^T A S, S^T S and the orthogonalisation products).  Each entry is split
 * into seven 7-bit integer digits relative to a power of two per column; digit products run as
 * BF16 tcgen05 MMAs whose FP32 sums over 64 rows are exact, and are combined in 64-bit integers
 * and FP64.  The error is about 1e-15 of ||u_i|| ||v_j||.
 *   n:      rows (>= 1).
 *   U, V:   device, column-major n x k1 and n x k2 (column j at U + j n), 1 <= k1, k2 <= 64.
 *   G:      device, k1 x k2 doubles, row-major (G[i k2 + j] = u_i . v_j).  Caller-owned.
 * Allocates and frees its workspace (about 64 KB per 2048 rows) and synchronises `stream`;
 * returns SMG_ERR_TIMEOUT when a bounded wait for the tensor cores gave up.
 */
int smg_gram(long long n, int k1, const double *U, int k2, const double *V, double *G, void *stream);

/*
 * smg_apply_A_dot_static -- out = A u and *dot = (u, A u), allocating nothing.
 * The paper has no counterpart: this is the 7-point operator with its fused inner product
 * (u, A u), in a form for callers that cannot allocate device memory where they need it
 * (a host framework that owns every device allocation and lends the library only input and
 * output buffers, or a section where cudaMalloc / cudaFree must not run because they can
 * synchronise the device).  No handle is needed.
 *   nx, ny, nz: grid sizes, >= 1, with nx*ny*nz <= 33,554,432 (the capacity of the scratch);
 *               larger grids return SMG_ERR_ARG with a message and launch nothing.
 *   u, out:     device, nx*ny*nz doubles each, caller-owned, must not overlap.
 *   dot:        device, one double, caller-owned.
 * Scratch: the per-CTA partial sums live in a file-scope device array (about 32 KB) that every
 * GPU which loads the library holds until the process exits.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) for that device; make that first
 * call before any stream capture.  Every call shares the array and clears its counter first:
 * calls that overlap on the GPU (for example on two streams at once) race and give wrong
 * results; calls ordered on one stream are safe.  Asynchronous on `stream`.
 */
int smg_apply_A_dot_static(int nx, int ny, int nz, const double *u, double *out, double *dot, void *stream);

/*
 * smg_setup_coefs -- the SMG set-up as smg_setup builds it, on the host only (no device, no
 * handle): section 3's semicoarsening hierarchy under the readings the library states (odd
 * planes and lines coarse, interpolation weights from the stencil collapsed in-plane, Galerkin
 * coarse operators).  For z-level l, plane z of that level and 2D level m of the plane:
 *   zc:    8 doubles (host, caller-owned): the plane's z-coupling M(z,z-1), M(z,z), M(z,z+1),
 *          K(z,z-1), K(z,z), K(z,z+1) and its interpolation weights wm(z), wp(z), where level l's
 *          operator is (A_l u)_z = sum_dz M(z,z+dz) L2D u_(z+dz) + K(z,z+dz) u_(z+dz);
 *   lines: ny_m x 8 doubles (host, caller-owned), line y of 2D level m: S(y,y-1), S(y,y),
 *          S(y,y+1), T(y,y-1), T(y,y), T(y,y+1), wm(y), wp(y), where the plane operator on that
 *          level is (B v)_y = sum_dy S(y,y+dy) Lx v_(y+dy) + T(y,y+dy) v_(y+dy);
 *   nz_l, ny_m: (host, may be NULL) the number of planes of level l and lines of 2D level m.
 * Any index out of range (l >= number of z-levels, z >= nz_l, m >= number of 2D levels) or a
 * grid that smg_setup refuses (a size < 1 or above its limits) returns SMG_ERR_ARG and writes
 * nothing; the sizes and l, m are checked before anything is allocated.  Each call builds the
 * whole host hierarchy (about 32 nz ny doubles of host memory, freed before it returns; a failed
 * host allocation returns SMG_ERR_HOST): meant for inspection and tests, not for a hot loop.
 */
int smg_setup_coefs(int nx, int ny, int nz, int l, int z, int m, double *zc, double *lines, int *nz_l, int *ny_m);

/*
 * smg_plane_classes -- the planes of z-level l that share one set of line-solver data, on the
 * host only (no device, no handle).  Planes whose 2D hierarchies (the `lines` of
 * smg_setup_coefs, every 2D level) are bit for bit equal form one class; the wide-line plane
 * relaxation (x-lines of more than 256 rows) forms its line-solver table once per class.
 *   cls: nz_l ints (host, caller-owned): the class of each plane of level l, numbered in order
 *        of first appearance (so cls[0] = 0).
 * Returns the number of classes (>= 1), or SMG_ERR_ARG (a grid smg_setup refuses, l out of
 * range, cls NULL; nothing written) or SMG_ERR_HOST (host allocation).  Builds the whole host
 * hierarchy like smg_setup_coefs: for inspection and tests.
 */
int smg_plane_classes(int nx, int ny, int nz, int l, int *cls);

/*
 * smg_plane_layout -- where the plane-relaxation kernel keeps the arrays of a plane's 2D cycle
 * (host only, no device): the layout the library plans for an nx x ny plane computed in
 * elem_bytes-byte arithmetic (4 or 8) by one CTA (R = 1) or by a cluster of R = 2, 4, 8 or 16
 * CTAs.  Shared memory holds the plane's coefficient table (sum_ny lines x coef_per_line values)
 * at offset 0, then the line-solver factor sets of the first MF 2D levels (two sets of
 * set_elems values each, from off_fs), then the 2D-cycle arrays u_m and g_m that fit; the others
 * live in a global slot of ws_elems values per CTA (per cluster when R > 1).  Offsets and sizes
 * are in elements.
 *   out: host, caller-owned, 64 long longs:
 *     [0] P (2D levels)  [1] K (x-line rows per lane)  [2] MF  [3] smem_bytes (0: the cluster
 *     layout does not fit)  [4] ws_elems  [5] off_fs  [6] on-chip mask of the u_m  [7] on-chip
 *     mask of the g_m  [8] sum_ny  [9] coef_per_line  [10] set_elems
 *     [16 + m] offset of u_m, [32 + m] offset of g_m, [48 + m] ny_m  (m < P <= 16)
 * Sizes outside the library's limits (nx, ny in 1..512), elem_bytes other than 4 or 8, or
 * another R return SMG_ERR_ARG and write nothing.
 */
int smg_plane_layout(int nx, int ny, int elem_bytes, int R, long long *out);

/*
 * smg_plane_layout_kind -- smg_plane_layout for each plane-cycle kernel's own layout (host only):
 *   kind 0: the general cycle (smg_plane_layout's plan);
 *   kind 1: the shortened-step cycle, nx <= 256: every 2D level's factor sets on chip (MF = P);
 *           on a cluster (R > 1) the 2D levels of at most `solo` lines from the first such level
 *           on are held whole by the cluster's first CTA where that keeps on chip every array the
 *           spread plan keeps (solo = 0: none);
 *   kind 2: the wide-line cycle, 257 <= nx <= 2048 (K = 8 rows per lane up to 512 rows, else 16):
 *           no factor sets on chip (MF = 0), 2 KB of the shared memory left to the kernel's
 *           static arrays.
 * out as smg_plane_layout's, plus [11] the first 2D level held whole by the first CTA (P when
 * none).  A level held whole keeps all ny_m lines on every CTA's plan (CTA 0 uses them); a spread
 * level keeps 2 ceil(ceil(ny_m / 2) / R) lines.  Residency of the cluster on the GPU is not
 * checked here (the library falls back to the spread plan, or a smaller cluster, at run time).
 * Arguments outside these ranges (and those smg_plane_layout refuses) return SMG_ERR_ARG.
 */
int smg_plane_layout_kind(int nx, int ny, int elem_bytes, int R, int kind, int solo, long long *out);

#ifdef __cplusplus
}
#endif
#endif
