/*
 * nle.h -- C ABI of the GB300 (sm_103a) DACG-Newton eigensolver.
 *
 * Computes the p leftmost eigenpairs of a large sparse symmetric positive
 * definite matrix A by the method of Bergamaschi & Martinez, "Efficiently
 * preconditioned Inexact Newton methods for large symmetric eigenvalue
 * problems" (arXiv:1312.1553):
 *   - Newton on the unit sphere for A u = q(u) u (Section 1, eq. "nonlinear",
 *     eq. "gras"), one eigenpair at a time, deflated against the converged
 *     ones (Section 3.2, eq. "precQ");
 *   - the correction equation solved by PCG restricted to the complement of
 *     Q = [v_1 .. v_{j-1} u_k] (Section 4.3);
 *   - the PCG preconditioner P_k = (I-QQ^T) Phat_k (I-QQ^T), with Phat_0 =
 *     (L L^T)^{-1}, L = IC(lfil, tau_IC, A) (Section 2), updated by the
 *     simplified BFGS formula eq. "lastprec" (or, as an option, the full
 *     formula of Section 3) and applied by Algorithm 3.1 with at most k_max
 *     stored pairs (Section 4.4);
 *   - the initial guess of each eigenpair from DACG (Section 4.1);
 *   - driven by Algorithm 3.2.
 * The sign convention of the paper is r = A u - theta u, J_k s = -r, so the
 * BFGS scalars alpha_s = s_s^T r_s are negative.
 *
 * Conventions common to every call:
 *   - Status codes, never exceptions; nle_last_error() gives a message.
 *   - Matrices are CSR with int64 row pointers, int32 column indices sorted
 *     ascending within each row, FP64 values; the pattern and the values
 *     must be symmetric, every diagonal entry present and positive.
 *   - Vectors are FP64 in the natural (caller's) row order.  A block of
 *     p vectors of length n is stored vector after vector: element i of
 *     vector j is at [j*n + i].
 *   - "buffers_on_device" = 1 means the vector arguments of that call are
 *     CUDA device pointers; 0 means host pointers (the library copies them
 *     through its own pinned staging buffers).
 *   - The caller owns every buffer it passes; the library never frees or
 *     retains caller memory beyond the call.  The handle owns all device
 *     memory it allocates and frees it in nle_destroy.
 *   - All work is ordered on the handle's CUDA stream; every call returns
 *     after that work has completed (it synchronises the stream), so outputs
 *     are ready on return.
 *   - A handle is not thread safe; different handles may be used from
 *     different host threads.
 *   - Every device-side wait (grid barriers, triangular-solve dependencies)
 *     is bounded by nle_options.spin_timeout_s; when a wait runs out the
 *     kernel records NLE_ERR_TIMEOUT, finishes without further waiting, and
 *     the call returns that status with the CUDA context still usable.
 */
#ifndef NLE_H
#define NLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nle_ctx *nle_t;

typedef enum {
  NLE_OK = 0,
  NLE_ERR_ARG = 1,        /* invalid argument (size, pointer, p >= n, ...) */
  NLE_ERR_CSR = 2,        /* malformed CSR: unsorted, asymmetric, missing diagonal */
  NLE_ERR_NOT_SPD = 3,    /* non-positive diagonal or IC pivot */
  NLE_ERR_BREAKDOWN = 4,  /* reserved: PCG breakdowns are handled inside the solve */
  NLE_ERR_NOCONV = 5,     /* some eigenpair missed the tolerance; outputs still written */
  NLE_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  NLE_ERR_OOM = 7,        /* device or host allocation failed */
  NLE_ERR_TIMEOUT = 8,    /* a bounded device-side wait ran out */
  NLE_ERR_STATE = 9,      /* call out of order (e.g. nle_solve before nle_factor_ic) */
  NLE_ERR_NO_DEVICE = 10  /* no CUDA device */
} nle_status;

enum { NLE_FP64 = 0, NLE_MIXED = 1 };

/* Bits of nle_pcg_info.exit / per-solve exit counters. */
enum {
  NLE_EXIT_TOL = 0,        /* (i)   ||g_l|| <= tau_PCG ||g_0|| */
  NLE_EXIT_MAXIT = 1,      /* (ii)  l = IMAX_PCG */
  NLE_EXIT_EIGRES = 2,     /* (iii) eq. "residual": ||A x - rho x||/||x|| < tau rho */
  NLE_EXIT_STAGNATION = 3, /* (iv)  ||r_{k,l}|| decreases slower than ||g_l|| */
  NLE_EXIT_BREAKDOWN = 4   /* p^T J p <= 0: the iterate so far is returned */
};

#define NLE_MAX_P 64 /* largest p accepted by nle_solve */
#define NLE_MAX_KMAX 10

/* Solver options.  Defaults (nle_default_options) follow the paper's Table
 * "default" (Section 5) where it gives a value, and k_max = 5 (Section 5.2:
 * "5 outer iterations are enough", results do not change for k_max >= 5). */
typedef struct {
  int k_max;             /* stored BFGS pairs, 0..NLE_MAX_KMAX (default 5) */
  double tau_pcg;        /* inner relative tolerance (default 1e-2) */
  double tau_dacg;       /* DACG tolerance ||A x - q x|| <= tau_dacg q (default 1e-2) */
  int max_dacg;          /* DACG iteration cap (default 5000) */
  int precision;         /* NLE_FP64 (default) or NLE_MIXED (FP32 bulk, FP64 outer step) */
  int exit_eigres;       /* enable inner exit (iii) (default 1) */
  int exit_stagnation;   /* enable inner exit (iv) (default 1) */
  int dacg_recompute;    /* recompute A x in DACG every this many iterations (default 50) */
  double spin_timeout_s; /* bound on each device-side wait, seconds (default 2.0) */
  int grid_ctas;         /* persistent grid size; 0 = one CTA per SM (default 0) */
  int trsv_warps;        /* warps per CTA in the triangular solves, 1..16 (default 16) */
  int ordering;          /* NLE_ORDER_NATURAL (default) or a multicolour ordering, see
                            nle_multicolor_order; applied before the IC factor */
  int bfgs_update;       /* NLE_BFGS_SIMPLIFIED (default) or NLE_BFGS_FULL */
  int trsv_schedule;     /* NLE_SCHED_AUTO (default), NLE_SCHED_LEVEL or NLE_SCHED_CHAIN */
  int trsv_poll_ns;      /* pause (ns, 0..10000) a warp of the triangular solves takes between
                            two polls of inputs that are not ready (default 0: none) */
  int trsv_rows;         /* level schedule: rows a warp takes at a time, 4 (8 lanes per row)
                            or 2 (16 lanes, for factors with wide rows); 0 (default): chosen
                            by the autotuner under NLE_SCHED_AUTO, 4 otherwise */
  int ic_device;         /* where nle_factor_ic computes the numeric factor: NLE_IC_AUTO
                            (default), NLE_IC_HOST or NLE_IC_DEVICE, see below */
} nle_options;

/* Where nle_factor_ic computes the numeric IC factor.  Both compute the
 * same factor bit for bit (same algorithm, same operation order, correctly
 * rounded operations).
 *   NLE_IC_HOST    on the host, one column after the other;
 *   NLE_IC_DEVICE  on the device: one warp per column, columns running
 *                  concurrently, each waiting (time-bounded) for the
 *                  earlier columns it depends on; needs lfil <= 31, and a
 *                  column whose working set outgrows the kernel's per-warp
 *                  tables (256 candidate rows and columns, 128 entries
 *                  after the drop test) returns NLE_ERR_ARG;
 *   NLE_IC_AUTO    the device when lfil <= 31, the host otherwise or when
 *                  a column outgrows the device tables.
 * nle_stats reports which ran and how long it took. */
#define NLE_IC_AUTO 0
#define NLE_IC_HOST 1
#define NLE_IC_DEVICE 2

/* Schedule of the triangular solves of Phat_0 = (L L^T)^{-1} (Section 2).
 * Both give the same solution (up to rounding order); they differ in how
 * the rows are dealt to the GPU's warps:
 *   NLE_SCHED_LEVEL  rows of each CTA's slab sorted by level of L, groups
 *                    of 4 rows per warp step, every row polling its own
 *                    inputs (no barrier between levels);
 *   NLE_SCHED_CHAIN  the factored matrix's own row order; runs of rows in
 *                    which each row depends on its predecessor (the grid
 *                    lines of a stencil matrix in natural order) stay on one
 *                    warp, which resolves that dependency in registers;
 *                    needs the natural ordering;
 *   NLE_SCHED_AUTO   nle_factor_ic times one application of (L L^T)^{-1}
 *                    on the device with the level schedule at 4 and at 2
 *                    rows per warp step (nle_options.trsv_rows) and with
 *                    the chain schedule (natural ordering only), and keeps
 *                    the fastest.
 * The choice and the timings are reported in nle_stats. */
#define NLE_SCHED_AUTO 0
#define NLE_SCHED_LEVEL 1
#define NLE_SCHED_CHAIN 2

/* BFGS update of the preconditioner (Section 3).  The full update uses
 * y_k = r_{k+1} - r_k; the paper's simplified update (eq. "lastprec", the
 * one its experiments use) replaces y_k by -r_k.  Either way Algorithm 3.1
 * runs on the stored pairs (s_k, w_k), w_k = -y_k, and a pair is kept only
 * when s_k^T w_k < 0 (Theorem 3.2).  The full update needs k_max <=
 * NLE_MAX_KMAX - 1 (one slot stages the newest pair until r_{k+1} is known). */
#define NLE_BFGS_SIMPLIFIED 0
#define NLE_BFGS_FULL 1

/* Symmetric orderings applied by nle_factor_ic before the IC factor.  The
 * paper factors A as given; a multicolour ordering factors P A P^T instead
 * (a different IC preconditioner of the same eigenproblem) with far fewer
 * levels in its triangular solves.  Inputs and outputs of every call stay
 * in the caller's numbering. */
#define NLE_ORDER_NATURAL 0
#define NLE_ORDER_MULTICOLOR1 1 /* greedy colouring of the graph of A */
#define NLE_ORDER_MULTICOLOR2 2 /* greedy colouring of the graph of A^2 (distance 2) */

/* Per-solve statistics, mirroring the columns of the paper's tables
 * (DACG its, outer its, MVP, CPU) plus device timings. */
typedef struct {
  int p;
  int dacg_its[NLE_MAX_P];
  int outer_its[NLE_MAX_P];
  int pcg_its[NLE_MAX_P];       /* inner iterations summed over the outer steps */
  int converged[NLE_MAX_P];
  double final_res[NLE_MAX_P];  /* ||A v - lambda v|| / lambda, FP64 */
  int64_t mvp_dacg;             /* products with A in DACG */
  int64_t mvp_newton;           /* products with A in the Newton phase */
  int exit_count[5];            /* inner exits by reason (NLE_EXIT_*) */
  double ms_dacg;               /* device time of the DACG phase */
  double ms_newton;             /* device time of the Newton phase */
  double ms_pcg_inner;          /* part of ms_newton spent in inner PCG iterations */
  int64_t pcg_iterations;       /* total inner iterations (for GB/s accounting) */
  int64_t pcg_sum_m;            /* sum over inner iterations of the columns of Q */
  int64_t pcg_sum_k;            /* sum over inner iterations of the stored pairs */
  int64_t dacg_iterations;      /* total DACG iterations */
  int64_t dacg_sum_m;           /* sum over DACG iterations of the deflated columns */
  int64_t kernel_launches;      /* CUDA kernels this call launched */
  double ms_phase[8];           /* device time by pass: SpMV, vector update, forward solve,
                                   backward solve, dot products, direction, outer FP64 step,
                                   other (Gram matrices) */
  int ascending;                /* 1 when eigenvalues came out strictly ascending */
  double ms_batch;              /* device time of the batched launch that solved this
                                   problem (nle_batch_solve; 0 after nle_solve) */
  int trsv_schedule;            /* NLE_SCHED_LEVEL or NLE_SCHED_CHAIN: the schedule in use */
  double tune_ms_level;         /* autotuner: device ms of one (L L^T)^{-1} application with */
  double tune_ms_chain;         /*   each candidate (0 when not timed): level schedule with 4 */
  double tune_ms_level2;        /*   rows per warp step, chain schedule, level with 2 rows */
  int64_t strands;              /* chain schedule: strands of L (runs of dependent rows) */
  int trsv_rows;                /* level schedule: rows per warp step in use */
  int ic_on_device;             /* 1 when the IC factor in use was computed on the device */
  double ms_ic_factor;          /* wall time of the numeric factor (device: with the copies) */
  double ms_ic_kernel;          /* device time of the factor kernel (0 on the host) */
  double ms_ic_setup;           /* wall time of the whole nle_factor_ic (factor, levels,
                                   layouts, autotuner) */
} nle_stats;

/* Parameters and outcome of one inner solve (nle_pcg). */
typedef struct {
  int its;     /* iterations performed (products with A) */
  int exit;    /* NLE_EXIT_* */
  double gnorm0, gnorm; /* ||g_0||, ||g_its|| */
  double eigres;        /* exit (iii) estimate at the last iteration */
} nle_pcg_info;

/* Fill *opt with the defaults above. */
void nle_default_options(nle_options *opt);

/* Create a handle for the n x n SPD matrix A (Section 1).
 *   rowptr[n+1], col[nnz], val[nnz]: CSR as described above; on_device
 *   says whether they are device (1) or host (0) pointers.  The handle
 *   copies them, so the caller may free them after the call.
 *   stream: cudaStream_t the handle orders its work on (NULL = legacy
 *   default stream).  opt may be NULL (defaults).
 * Errors: NLE_ERR_ARG (n < 2, nnz < n, NULL pointers), NLE_ERR_CSR (pattern
 * checks), NLE_ERR_NOT_SPD (non-positive diagonal), NLE_ERR_NO_DEVICE,
 * NLE_ERR_OOM, NLE_ERR_CUDA.  *out is NULL on error. */
nle_status nle_create(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col, const double *val,
                      int on_device, void *stream, const nle_options *opt, nle_t *out);

/* IC(lfil, tau_IC) factor of A (Section 2: Phat_0 = (L L^T)^{-1}) and the
 * level sets of L and L^T that schedule the triangular solves.
 * The factor is computed in FP64 (on the device or the host, see
 * nle_options.ic_device: the same factor bit for bit) by a left-looking
 * column algorithm with a fixed operation order: column j starts from the lower
 * part of column j of A; for every k < j with L(j,k) != 0, in ascending k,
 * every row i >= j of column k is updated w[i] -= L(i,k) L(j,k); the pivot
 * w[j] must be positive; L(j,j) = sqrt(w[j]), L(i,j) = w[i]/L(j,j); an
 * off-diagonal is dropped when |L(i,j)| < tau_IC ||A(:,j)||_2; of the rest
 * the lfil largest in modulus are kept (ties to the smaller row).
 * The factor and its levels are uploaded once; the device then works in a
 * slab-major, level-minor order of the unknowns (one slab of consecutive
 * rows per CTA, sorted by level of L inside the slab: a relabelling, the
 * method is unchanged).  With nle_options.ordering the factor is that of
 * P A P^T for the multicolour permutation P.  Errors: NLE_ERR_ARG (lfil < 0, tau_IC < 0;
 * NLE_IC_DEVICE with lfil > 31 or a column beyond the device tables),
 * NLE_ERR_NOT_SPD (non-positive pivot), NLE_ERR_TIMEOUT (a wait of the device
 * factor ran past spin_timeout_s), NLE_ERR_OOM, NLE_ERR_CUDA.
 * Calling it again refactors with the new parameters. */
nle_status nle_factor_ic(nle_t h, int lfil, double tau_ic);

/* Leftmost p eigenpairs by Algorithm 3.2 (DACG-Newton).
 *   tol: outer tolerance tau, ||A u - theta u|| <= tau theta.
 *   max_newton: ITMAX; max_pcg: IMAX_PCG.
 *   X0 [p*n]: start vector x_0 of every eigenpair (projected and
 *   normalised by the library); NULL draws a fixed pseudo-random start.
 *   lambda [p] and V [p*n] receive the eigenvalues in the order found
 *   (ascending when the method finds the leftmost pairs in order) and unit
 *   eigenvectors whose entry of largest modulus is positive.
 *   stats may be NULL.
 * Returns NLE_ERR_NOCONV when an eigenpair stopped at max_newton (outputs
 * and stats still written), NLE_ERR_STATE before nle_factor_ic,
 * NLE_ERR_ARG for p < 1, p >= n, p > NLE_MAX_P, tol <= 0. */
nle_status nle_solve(nle_t h, int p, double tol, int max_newton, int max_pcg, const double *X0, double *lambda,
                     double *V, nle_stats *stats, int buffers_on_device);

/* Adjoint of the last nle_solve (not in the paper).  For the loss L(lambda, V)
 * with gradients gbar_lambda [p] and gbar_V [p*n] (either may be NULL),
 * accumulates grad_val[e] += dL/dA_ab for every stored entry e = (a,b) of
 * A, treating A_ab and A_ba as independent:
 *   dlambda_j/dA_ab = v_ja v_jb;
 *   for the eigenvectors xi_j = -sum_{i<=p,i!=j} v_i (v_i^T gbar_vj)/(lambda_i-lambda_j) - y_j,
 *   y_j perp V solving (I-VV^T)(A-lambda_j I)(I-VV^T) y = (I-VV^T) gbar_vj by
 *   the same projected PCG, and dL/dA_ab += xi_ja v_jb.
 * The projected solves use FP64 residuals with iterative refinement so
 * that the result is accurate to ~1e-10 relative on both precisions.
 * Errors: NLE_ERR_STATE without a prior successful nle_solve, NLE_ERR_ARG
 * for a repeated eigenvalue. */
nle_status nle_backward(nle_t h, const double *gbar_lambda, const double *gbar_V, double *grad_val,
                        int buffers_on_device);

/* Solve `count` independent problems (each handle factored) in ONE
 * persistent launch: groups of G CTAs take problems from a device work
 * queue, largest n first, and each group runs the whole of Algorithm 3.2
 * (DACG and Newton for every eigenpair) for its problem, then takes the next.
 * G = 4, or 8 when some handle was factored for more than 4 CTAs.
 * Requirements: every handle was factored for at most 8 CTAs (create it with
 * nle_options.grid_ctas = 4 or 8, or small enough n), all handles share the
 * precision, the device and the schedule of the triangular solves (factor
 * them with the same explicit nle_options.trsv_schedule; NLE_SCHED_AUTO may
 * choose differently per matrix); the options of hs[0] apply and the work
 * runs on hs[0]'s stream.  p, tol, max_newton, max_pcg as in nle_solve.
 * lambdas[b] [p] and Vs[b] [p*n_b] are device pointers; X0s may be NULL or
 * an array of device pointers (entries may be NULL: fixed pseudo-random
 * starts).  per_problem[b] (nullable) receives each problem's status; the
 * return value is the worst of them.  Each handle then holds its solution
 * for nle_backward. */
nle_status nle_batch_solve(int count, nle_t *hs, int p, double tol, int max_newton, int max_pcg,
                           const double *const *X0s, double *const *lambdas, double *const *Vs,
                           nle_status *per_problem);

/* Statistics of the handle's last solve, by nle_solve or as one problem of
 * nle_batch_solve (there the device times of the phases are 0 and ms_batch
 * is the time of the whole batched launch).  The set-up fields (schedule of
 * the triangular solves, autotuner timings, IC factor) describe the
 * handle's current factor and are filled after nle_factor_ic alone (the
 * solve fields are then 0).  NLE_ERR_STATE before nle_factor_ic. */
nle_status nle_get_stats(nle_t h, nle_stats *stats);

/* ---- Building blocks of the hot path, exposed for verification ---------- */

/* y = (A - theta I) x in the handle's working precision (the product with
 * the Jacobian before projection, Section 4.3).  x, y: n, FP64. */
nle_status nle_apply_shifted(nle_t h, double theta, const double *x, double *y, int buffers_on_device);

/* c = P g by Algorithm 3.1 with k stored pairs (S, R: k*n, oldest first,
 * alpha[s] = s_s^T r_s < 0 recomputed by the library from the rounded
 * vectors) and the final Gram-Schmidt step against the m columns of Q
 * (m*n, orthonormal; m = 0 skips it).  Working precision of the handle. */
nle_status nle_apply_prec(nle_t h, int k, const double *S, const double *R, int m, const double *Q,
                          const double *g, double *c, int buffers_on_device);

/* One inner solve J_k s = -r, s perp Q (Section 4.3) with theta, the current
 * iterate u (= last column of Q), the residual r, Q (m*n), the k stored
 * pairs (S, R as in nle_apply_prec), and the options of the handle for the
 * exits; tol is the outer tau used by exit (iii).  s: n output. */
nle_status nle_pcg(nle_t h, double theta, double tol, int max_pcg, const double *r, int m, const double *Q, int k,
                   const double *S, const double *R, double *s, nle_pcg_info *info, int buffers_on_device);

/* Copy the IC factor out (host arrays).  Pass NULL for any output to only
 * query sizes.  L is CSR lower triangular with the diagonal last in each
 * row (nnzL entries, Lrowptr n+1); levL/levU: level of every row of L and
 * of U = L^T; *nlevL, *nlevU: number of levels.  With a multicolour
 * ordering the factor is that of P A P^T, in its numbering (row k of the
 * factor is row perm[k] of A, perm from nle_multicolor_order). */
nle_status nle_get_factor(nle_t h, int64_t *nnzL, int64_t *Lrowptr, int32_t *Lcol, double *Lval, int32_t *levL,
                          int32_t *levU, int64_t *nlevL, int64_t *nlevU);

/* Greedy multicolour ordering of a symmetric sparsity pattern (host only,
 * no device, no handle).  Not in the paper: it serves the optional
 * reordering of nle_options.ordering.  Rows are coloured in natural order,
 * each with the smallest colour not used by an already coloured row of its
 * neighbourhood: {j != i : A_ij != 0} for distance 1, and additionally the
 * neighbours of those rows for distance 2.  perm[k] (n entries, caller
 * owned) lists the rows by colour, ascending row inside a colour, so
 * P A P^T has row k = row perm[k] of A; *ncolors receives the number of
 * colours.  NLE_ERR_ARG for distance not 1 or 2 or NULL pointers,
 * NLE_ERR_CSR for a malformed pattern. */
nle_status nle_multicolor_order(int64_t n, const int64_t *rowptr, const int32_t *col, int distance, int32_t *perm,
                                int32_t *ncolors);

/* ---- Allocation-free preconditioner application --------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need the preconditioner: code
 * running inside another framework's memory pool, real-time loops in which
 * cudaMalloc's implicit device synchronisation and latency are not
 * acceptable, or programs that must finish all allocation at start-up.
 *
 * c = (L L^T)^{-1} g, the incomplete-Cholesky part of the preconditioner,
 * in FP64, with L given by the caller:
 *   Lrp[n+1], Lcol, Lval: the strictly lower part of L in CSR (int32 row
 *     pointers), rows in natural order;
 *   Urp[n+1], Ucol, Uval: the strictly upper part of U = L^T in CSR;
 *   diag[n]: the diagonal of L;  g[n]: input;  c[n]: output, which must
 *     not overlap g (NLE_ERR_ARG otherwise: no in-place application).
 * Every pointer is a device pointer owned by the caller; stream is the
 * cudaStream_t the work is ordered on (NULL = legacy default stream).  The
 * call reads its error word back on that stream and waits for the stream
 * before it returns.  It clears the runtime's pending launch error (if an
 * earlier launch of the caller left one) before its own launches.
 *
 * It allocates nothing: its only temporary storage is one fixed array of
 * NLE_NOALLOC_MAX_N + 32 doubles (about 2 MB) compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * Consequences for the caller:
 *   - n must be 1..NLE_NOALLOC_MAX_N; larger n returns NLE_ERR_ARG with a
 *     message in nle_last_error(NULL) and touches no memory;
 *   - the first call on a device looks up the array's device address once
 *     for that device (cudaGetSymbolAddress, with that device current);
 *   - it cannot be called while its stream is being captured into a CUDA
 *     graph: it reads its error word back and waits for the stream;
 *   - all calls share the array and it keeps the last call's contents (the
 *     call resets what must start fresh), so calls that overlap on the GPU,
 *     on any streams or threads, race: serialise them;
 *   - entries that are not strictly triangular are skipped and reported
 *     (NLE_ERR_CSR); a wait that runs out reports NLE_ERR_TIMEOUT.
 */
#define NLE_NOALLOC_MAX_N 262144
nle_status nle_ic_apply_noalloc(int64_t n, const int32_t *Lrp, const int32_t *Lcol, const double *Lval,
                                const int32_t *Urp, const int32_t *Ucol, const double *Uval, const double *diag,
                                const double *g, double *c, void *stream);

/* Message of the last failed call on h (or of the last nle_create failure
 * when h is NULL).  Valid until the next call on h. */
const char *nle_last_error(nle_t h);

/* Release the handle and all device memory it owns.  NULL is ignored. */
void nle_destroy(nle_t h);

#ifdef __cplusplus
}
#endif

#endif /* NLE_H */
