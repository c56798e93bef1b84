/*
 * ddlr.h -- C ABI of the GB300 (sm_103a) DDLR preconditioner library.
 *
 * DDLR (Li & Saad, "Low-rank correction methods for algebraic domain
 * decomposition preconditioners") splits a sparse SPD matrix, reordered with
 * all interior unknowns first and all interface unknowns last (Sec. 2.2,
 * eq. Bmat), as A = A0 - E E^T with E = [a^-1 Ehat ; -a I] and
 * A0 = blkdiag(B_{1,a}, ..., B_{p,a}, C_a) (Sec. 3.1, eq. EF and eq. split),
 * and preconditions CG with the Sherman-Morrison-Woodbury based
 *   DDLR-1: M^-1 = A0^-1 + (A0^-1 E) G_{k,theta}^-1 (E^T A0^-1)
 *           (Sec. 3.2, eq. Mprec with prop. gkt, applied by Algorithm 1), or
 *   DDLR-2: M^-1 = A0^-1 + U_k H_k U_k^T   (Sec. 3.3, eq. Form2a),
 * where the rank-k data come from Lanczos with full reorthogonalisation
 * (Sec. 4.4).
 *
 * Conventions for every call:
 *  - Matrices are passed as full symmetric CSR (both triangles), int32 row
 *    pointers and column indices, strictly ascending columns in each row,
 *    float64 values, in the caller's ORIGINAL ordering.  The library copies what
 *    it needs; the caller keeps ownership of every array it passes.
 *  - Vectors are float64, original ordering, column-major n x nrhs with leading
 *    dimension ld >= n.  A vector pointer may be device memory (then the call is
 *    asynchronous on the handle's stream, except where noted) or host memory
 *    (pageable or pinned; detected with cudaPointerGetAttributes, staged through
 *    device buffers, and the call returns when the result is in host memory).
 *  - The handle owns all of its device memory until ddlr_destroy.  A handle is
 *    not thread-safe: use one handle per thread or serving slot.
 *  - No C++ exception crosses the ABI.  Every call returns a ddlr_status; the
 *    text of the last error is available from ddlr_last_error.
 */
#ifndef DDLR_H
#define DDLR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddlr_ctx *ddlr_handle;

typedef enum {
  DDLR_OK = 0,
  DDLR_ERR_INVALID = 1,    /* bad argument, malformed or non-symmetric CSR   */
  DDLR_ERR_OOM = 2,        /* device or host allocation failed                */
  DDLR_ERR_BREAKDOWN = 3,  /* non-positive pivot in a local factorisation     */
  DDLR_ERR_NOT_SPD = 4,    /* prop. spd-1 / spd-2 check failed (Sec. 5)       */
  DDLR_ERR_NOCONV = 5,     /* PCG did not reach tol within maxit ('F', Sec. 5) */
  DDLR_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up              */
  DDLR_ERR_NAN = 7,        /* NaN or Inf met in a residual or a Lanczos step  */
  DDLR_ERR_CUDA = 8        /* a CUDA runtime call failed                      */
} ddlr_status;

typedef struct {
  int variant;             /* 1 = DDLR-1 (Sec. 3.2), 2 = DDLR-2 (Sec. 3.3)         */
  int rank_k;              /* k >= 1, k <= s (k = s gives M^-1 = A^-1 with exact
                              local factors, eq. split3)                          */
  double alpha;            /* splitting parameter a of eq. EF; default 1 (Sec. 5) */
  int theta_mode;          /* DDLR-1: 1 = theta = lambda_{k+1} (default, Sec. 5),
                              0 = theta = 0 (eq. Lambda-1)                         */
  int factor;              /* local solver: 0 = IC(0) on the block pattern,
                              1 = exact Cholesky (IC on the symbolic fill pattern),
                              2 = incomplete L D L^T on the block pattern, 3 =
                              exact L D L^T (symbolic fill pattern); 2 and 3 do
                              not pivot (a zero pivot is BREAKDOWN), serve
                              indefinite blocks (Sec. 5), and need precision 0,
                              c_solver 0 and lowrank_method 0 or 2; their
                              right-hand sides are solved one at a time        */
  int c_order;             /* elimination order of C_a: 0 = ascending original
                              index, 1 = multicolour (the two colour classes of a
                              bipartite graph, else greedy colouring)              */
  int b_order;             /* elimination order inside the interior blocks B_{i,a}:
                              0 = ascending original index, 1 = multicolour as for
                              c_order                                              */
  int precision;           /* 0 = FP64 throughout; 1 = mixed: FP32 factors and
                              triangular solves, FP32/BF16 U_k, inside an FP64
                              flexible CG                                          */
  int uk_bf16;             /* precision 1 only: 1 = U_k stored in BF16            */
  int scale_diag;          /* 1 = build DDLR on D^-1/2 A D^-1/2, D = diag(A)      */
  int lanczos_max;         /* maximum Lanczos steps; 0 = 5k (Sec. 5)              */
  int lanczos_check;       /* convergence check period; default 10 (Sec. 5)       */
  double lanczos_eps;      /* tolerance of eq. converge; default 1e-4 (Sec. 5)    */
  unsigned long long seed; /* SplitMix64 stream of the Lanczos start vector       */
  int max_nrhs;            /* largest nrhs used with this handle (workspace)      */
  int c_solver;            /* solve with C_a (Sec. 4.3): 0 = factored like a local
                              block (c_order, factor); 1 = preconditioned Chebyshev
                              iterations with the block Jacobi preconditioner D_a
                              (the couplings of C_a inside one subdomain, factored
                              like a local block) on a spectrum interval estimated
                              by Lanczos on (C_a, D_a); 2 = product with the
                              symmetric part of an approximate inverse X of C_a
                              from self-preconditioned MR iterations with
                              dual-threshold dropping (Algorithm 2)               */
  int cheb_steps;          /* c_solver 1: Chebyshev steps per solve (default 5,
                              Sec. 5)                                               */
  int cheb_lanczos;        /* c_solver 1: Lanczos steps of the spectrum estimate
                              (default 20)                                          */
  int lowrank_method;      /* 0 = Lanczos (Sec. 4.4, default); 1 = randomized
                              subspace iteration (the faster technique the
                              conclusion names): ell = rank_k + rand_oversample
                              columns (at most 64, at most s), rand_power power
                              steps, Rayleigh-Ritz on the ell-dimensional basis;
                              2 = Lanczos bidiagonalisation of A0^-1 E (DDLR-2
                              only, Sec. 4.4): U_k and V_k together, the same
                              step limit and eq. converge test as Lanczos        */
  int rand_oversample;     /* lowrank_method 1: oversampling p (default 10)      */
  int rand_power;          /* lowrank_method 1: power steps q (default 2)         */
  int mr_iters;            /* c_solver 2: MR iterations (default 3)              */
  int mr_lfil;             /* c_solver 2: entries kept per column of Z (default 8;
                              1 + mr_iters * mr_lfil <= 32)                        */
  double mr_droptol;       /* c_solver 2: drop tolerance relative to the column
                              norm of Z (default 1e-3)                             */
  int indefinite;          /* 1 = accept a preconditioner that is not SPD, for
                              ddlr_gmres (Sec. 5: indefinite problems and
                              preconditioners found not SPD).  DDLR-1 keeps Ritz
                              values >= 1 and needs only 1 - lambda_i and
                              1 - theta away from zero; DDLR-2 inverts I - K by
                              Gauss-Jordan elimination with partial pivoting.  A
                              singular G_{k,theta} or I - K gives BREAKDOWN.  The
                              local factors stay IC(0) / Cholesky, so A0 must be
                              positive definite (else BREAKDOWN).  Default 0.   */
  int fill_level;          /* incomplete factors (factor 0 and 2): the level of
                              fill of their pattern -- A0's entries have level
                              0, eliminating pivot t gives entry (i, j) of two
                              later neighbours of t the level lev(i,t) +
                              lev(j,t) + 1, and entries up to this level are
                              kept.  Default 0 (the pattern of A0); 0..64;
                              INVALID with factor 1 or 3.                      */
  int lanczos_reorth;      /* full reorthogonalisation of each Lanczos vector
                              against all earlier ones (Sec. 4.4 Lanczos with
                              reorthogonalisation): 0 (default) = one classical
                              Gram-Schmidt pass, and a second one when the
                              first left less than half of ||w||^2 (the DGKS
                              criterion); 1 = two passes every step.  A restart
                              vector always takes two.                        */
  double wait_limit_s;     /* limit of every bounded device wait, seconds (grid
                              barriers of the persistent kernels, ready flags of
                              the synchronisation-free solve; the TMA solve waits
                              at least 1 s for its copies): when it runs out the
                              kernel records it and returns, and the call gives
                              DDLR_ERR_TIMEOUT.  Default 2; (0, 3600].          */
} ddlr_options;

typedef struct {
  int n, p, s, m, k, variant, precision;
  int lanczos_steps;       /* m of Sec. 4.4 (steps actually taken); with
                              lowrank_method 1 the basis size ell                  */
  int ncolors;             /* colours of C_a (c_order 1), else 0                  */
  int levels_interior;     /* max dependency levels of an interior block factor   */
  int levels_c;            /* dependency levels of the C_a factor                 */
  double theta;            /* theta used in G_{k,theta}^-1 (DDLR-1)               */
  double lambda_max;       /* largest Ritz value (DDLR-1; must be < 1)            */
  long long nnz_a;         /* nnz(A)                                              */
  long long nnz_factor;    /* stored factor entries incl. diagonals, all blocks   */
  long long nnz_ehat;      /* nnz(Ehat)                                           */
  double fill_ratio;       /* nnz(preconditioner)/nnz(A) as in Sec. 5             */
  long long device_bytes;  /* device memory held by the handle                    */
  double setup_ms;         /* wall time of the last (re)setup                     */
  int batch_block_chunks;  /* rows per pass picked by the autotuner for the batched
                              level solve (0 before the first batched call)       */
  int batch_block_elem;    /* block size picked for the batched row kernels      */
  double plan_ms;          /* host analysis (orderings, levels, layouts) of setup */
  int persistent;          /* bit 0: PCG, bit 1: Lanczos run as one cooperative launch */
  double cheb_lo, cheb_hi; /* c_solver 1: spectrum interval of D_a^-1 C_a in use  */
  int cheb_lanczos_steps;  /* c_solver 1: Lanczos steps the estimate took         */
  int reorth_passes;       /* Gram-Schmidt passes of the Lanczos steps of the last
                              build (lowrank_method 0; restart vectors excluded) */
  int reorth_fp32;         /* of the corrections w -= Q c of those passes (and of
                              restart vectors), the ones the persistent Lanczos
                              kernel formed in FP32 from an FP32 copy of Q: only
                              where their error bound is below FP64 rounding of w */
} ddlr_info;

typedef struct {
  int its;                 /* iterations (x updates)                              */
  double relres;           /* true relative residual ||b - A x|| / ||b||          */
  int status;              /* DDLR_OK, DDLR_ERR_NOCONV or DDLR_ERR_NAN            */
} ddlr_solve_info;

/* Fills *opt with the defaults named above (variant 1, k 16, alpha 1,
 * theta_mode 1, IC(0), c_order 0, b_order 0, FP64, lanczos 5k/10/1e-4, seed 0,
 * max_nrhs 1, c_solver 0, cheb_steps 5, cheb_lanczos 20, lowrank_method 0,
 * rand_oversample 10, rand_power 2, mr_iters 3, mr_lfil 8, mr_droptol 1e-3).
 * Returns DDLR_ERR_INVALID for a NULL pointer. */
ddlr_status ddlr_options_default(ddlr_options *opt);

/* Build the preconditioner (Sec. 4.1): classify nodes (Sec. 2.1), reorder
 * (eq. Bmat), form B_{i,a} = B_i + a^-2 E_i E_i^T and C_a = C + a^2 I
 * (eq. split), factor all p+1 blocks on the GPU, run Lanczos on the GPU
 * (Sec. 4.4) and form the low-rank data.
 *   n, rowptr[n+1], colind[nnz], val[nnz]: A, host memory, original order.
 *   part[n]: subdomain of each node, values in [0, p), host memory.
 *   opt: options (NULL = defaults).  cuda_stream: cudaStream_t or NULL for the
 *   legacy default stream.  *out receives the handle (NULL on failure).
 * Synchronous.  Errors: INVALID (malformed input, k > s, no interface nodes),
 * OOM, BREAKDOWN, NOT_SPD, NAN, CUDA. */
ddlr_status ddlr_setup(int n, const int *rowptr, const int *colind,
                       const double *val, const int *part, int p,
                       const ddlr_options *opt, void *cuda_stream,
                       ddlr_handle *out);

/* Numeric re-setup with the same sparsity pattern and partition: optional new
 * values val[nnz] (host or device memory, original CSR order; NULL keeps the
 * resident values), then the device-side part of ddlr_setup (scaling, block
 * forming, factorisation, Lanczos, low-rank data).  Synchronous. */
ddlr_status ddlr_refactor(ddlr_handle h, const double *val);

/* Improve the preconditioner by raising the rank k without discarding the
 * Lanczos vectors already computed (Sec. 3.4, "Improving a given
 * preconditioner"): the Lanczos process continues from its last step, with
 * the step limit (lanczos_max, else 5 k_new) and the convergence test of
 * eq. converge taken for k_new, then U_k and Lambda_k / H_k are rebuilt for
 * k_new.  When neither run is stopped by the convergence test, the result is
 * the one ddlr_setup with rank k_new would give.  The arrays of the old rank
 * stay allocated until ddlr_destroy.  Synchronous.  Errors: INVALID (k_new <=
 * rank_k, k_new > s or > 256, lowrank_method 1), NAN, NOT_SPD, CUDA. */
ddlr_status ddlr_increase_rank(ddlr_handle h, int k_new);

/* y = M^-1 x (Algorithm 1 for DDLR-1, eq. Form2a for DDLR-2) for nrhs vectors.
 * With nrhs > 1 the vectors are processed in batches of up to 64 in one set of
 * launches (row-major blocks, one lane per vector); a column's result does not
 * depend on the other columns of its batch.  x and y must not overlap.
 * Errors: INVALID (nrhs < 1, ld < n, NULL). */
ddlr_status ddlr_apply(ddlr_handle h, const double *x, double *y, int nrhs,
                       int ld);

/* y = A0^-1 x: the p local solves with B_{i,a} and the solve with C_a that
 * Algorithm 1 performs twice per application (Sec. 4.2). */
ddlr_status ddlr_a0_solve(ddlr_handle h, const double *x, double *y, int nrhs,
                          int ld);

/* y = A0^-1 x as ddlr_a0_solve computes it, for callers that must not
 * allocate device memory: applications whose device memory is all owned by
 * their own allocator or pool (where a cudaMalloc could fail or fragment it),
 * or code that runs inside such an allocator.  A call never calls cudaMalloc,
 * cudaFree or an allocating library routine: it reads the handle's factors
 * (allocated by ddlr_setup) and keeps its temporaries in static device memory.
 * The paper has no counterpart: it is a property of the library, not of the
 * method.
 * The two temporary vectors live in one file-scope device array of
 * 2 x 1,048,576 doubles (16 MiB), present on every GPU that loads the library
 * until the process exits, so n must be at most 1,048,576.  The first call on
 * each device does a one-time set-up (it looks up that array's device address
 * with cudaGetSymbolAddress); make that first call before any stream capture.
 * x and y: device memory, n doubles each, original order, not overlapping.
 * Asynchronous on the handle's stream.  Nothing needs to start at zero: every
 * entry of the array is written before it is read.  All calls in the process
 * share the array, so calls whose work overlaps on the GPU (other streams,
 * other handles, other threads) race: order them (one stream, or events).
 * The device current at the call must be the one the handle was set up on.
 * Errors: INVALID for n > 1,048,576, a precision-1 handle, NULL or host
 * pointers, another current device; CUDA if the set-up fails. */
ddlr_status ddlr_a0_solve_noalloc(ddlr_handle h, const double *x, double *y);

/* Preconditioned CG from x0 = 0 (Sec. 5) for each of nrhs right-hand sides,
 * stopping when ||r|| <= tol ||b|| and the true residual confirms it (else r is
 * replaced by b - A x and CG restarts), or after maxit iterations (maxit <= 0:
 * 500, Sec. 5).  With precision 1 the outer loop is flexible CG in FP64 around
 * the FP32 preconditioner.  With nrhs > 1 the right-hand sides are solved
 * together (batches of up to 64, one CUDA-graph iteration for the batch, a
 * converged column is frozen while the others continue); a column's iterates
 * do not depend on which other columns share its batch.  info[nrhs] (host memory, may be NULL) receives the
 * per-RHS result.  Synchronous.  Returns DDLR_OK when every RHS converged,
 * else DDLR_ERR_NOCONV or DDLR_ERR_NAN. */
ddlr_status ddlr_pcg(ddlr_handle h, const double *b, double *x, int nrhs,
                     int ld, double tol, int maxit, ddlr_solve_info *info);

/* Restarted GMRES(restart) from x0 = 0 (Sec. 5: GMRES(40) for the indefinite
 * problems and for preconditioners found not SPD), right-preconditioned by
 * M^-1: Arnoldi on A M^-1 with two classical Gram-Schmidt passes and Givens
 * rotations.  The preconditioned vectors Z = M^-1 V are kept (n x restart
 * doubles of workspace, allocated on first use), so the update x += Z y needs
 * no further apply, and an FP32 M^-1 (precision 1) is used as in flexible
 * GMRES.  A cycle ends when the rotated residual norm is <= tol ||b||, after
 * restart steps, at maxit steps in total, or when the new Arnoldi vector is
 * zero; the true residual b - A x then decides convergence and starts the
 * next cycle.  b, x: n doubles, host or device memory, original order, one
 * right-hand side.  maxit <= 0: 500; restart <= 0: 40; restart <= 512.  info
 * (host memory, may be NULL): its = Arnoldi steps (products with A), relres =
 * true relative residual.  Synchronous.  Returns DDLR_OK, DDLR_ERR_NOCONV or
 * DDLR_ERR_NAN; INVALID for NULL vectors, tol <= 0 or restart > 512. */
ddlr_status ddlr_gmres(ddlr_handle h, const double *b, double *x, double tol,
                       int maxit, int restart, ddlr_solve_info *info);

/* Sizes, counts and scalars of the handle (host struct). */
ddlr_status ddlr_get_info(ddlr_handle h, ddlr_info *info);

/* The Lanczos Ritz values (all m of T_m, descending) into out[cap] (host);
 * *count receives m. */
ddlr_status ddlr_get_ritz(ddlr_handle h, double *out, int cap, int *count);

/* The local factor entries (lower triangle incl. diagonal, every block) as
 * (row, col, value) in ORIGINAL indices.  With rows == NULL only *nnz is set.
 * Host arrays of length *nnz.  Synchronous. */
ddlr_status ddlr_get_factor_coo(ddlr_handle h, long long *nnz, int *rows,
                                int *cols, double *vals);

/* Low-rank data, host memory.  U is urows x k row-major with rows in ascending
 * original index of the nodes it covers (the s interface nodes for DDLR-1, all
 * n nodes for DDLR-2); lam[k] = Lambda_k (DDLR-1), theta (DDLR-1), Hk[k*k]
 * (DDLR-2).  Any output pointer may be NULL.  Synchronous. */
ddlr_status ddlr_get_lowrank(ddlr_handle h, double *U, double *lam,
                             double *theta, double *Hk);

/* Replace the low-rank data (same layout as ddlr_get_lowrank, host memory):
 * checkpoint restore, or injection of reference data for parity checks.
 * lam/theta are used by DDLR-1, Hk by DDLR-2.  Synchronous. */
ddlr_status ddlr_set_lowrank(ddlr_handle h, const double *U, const double *lam,
                             double theta, const double *Hk);

/* Replace the spectrum interval [lo, hi] of D_a^-1 C_a on which the Chebyshev
 * solve with C_a runs (c_solver 1, Sec. 4.3): a caller that knows bounds of
 * the spectrum, or injection of reference data for parity checks.  The
 * iteration's coefficients are recomputed on the device; the low-rank data
 * are kept (they were built with the previous interval).  Synchronous.
 * Errors: INVALID (c_solver 0, or not 0 < lo <= hi). */
ddlr_status ddlr_set_cheb_bounds(ddlr_handle h, double lo, double hi);

/* Kernel accounting: number of library kernel launches since the last reset,
 * and per-family device time accumulated with CUDA events recorded on the
 * launching stream while timing is enabled (ddlr_set_timing).  names receives
 * a comma-separated list of families (cap bytes), ms[cap_f] and launches[cap_f]
 * their totals.  Host memory. */
ddlr_status ddlr_set_timing(ddlr_handle h, int enable);
ddlr_status ddlr_get_counters(ddlr_handle h, long long *launches, char *names,
                              int cap, double *ms, long long *family_launches,
                              int cap_f, int *nfamilies);
ddlr_status ddlr_reset_counters(ddlr_handle h);

/* Algorithmic bytes (single RHS, int32 indices, each factor value and index
 * read once per sweep, vectors read and written once, gathered vector reads
 * counted as cache hits) of one M^-1 apply and of one A0 solve, and, per kernel
 * family of ddlr_get_counters (same order, cap_f entries), the bytes one launch
 * of that family moves on average (0 where not accounted).  Host memory. */
ddlr_status ddlr_get_traffic(ddlr_handle h, double *apply_bytes,
                             double *a0_solve_bytes, double *family_bytes,
                             int cap_f);

/* Use another stream (cudaStream_t) for later calls. */
ddlr_status ddlr_set_stream(ddlr_handle h, void *cuda_stream);

/* Change the limit of the handle's bounded device waits (ddlr_options
 * wait_limit_s) to `seconds` in (0, 3600].  Synchronises the handle's stream;
 * captured CUDA graphs are rebuilt at their next use.  A wait that runs out
 * sets a device flag, every CTA of the kernel returns, and the call that
 * launched it returns DDLR_ERR_TIMEOUT (its results are invalid); the flag is
 * cleared then, so the handle stays usable.  Errors: INVALID. */
ddlr_status ddlr_set_wait_limit(ddlr_handle h, double seconds);

/* Self-test of the library's binary64 <-> binary32 conversions written on the
 * bit patterns (IEEE 754-2008 Sec. 5.4.2 formatOf conversions: rounding to
 * nearest, ties to even; widening exact), which the batched mixed-precision
 * casts use, against the device's own conversion instructions.  in: n
 * doubles in DEVICE memory (not modified).  dir 0: each value narrowed to
 * binary32; dir 1: the low 32 bits of each value read as a binary32 and
 * widened.  *mismatches = the number of results whose bits differ (NaNs of
 * either kind count as equal when widening).  Synchronous, on the legacy
 * stream; allocates n doubles of device scratch.  Errors: INVALID (NULL or
 * host pointer, n < 0, bad dir), CUDA. */
ddlr_status ddlr_selftest_conversions(const double *in, long long n, int dir, long long *mismatches);

/* Text of the last error on this handle; with h == NULL, of the last failed
 * ddlr_setup on this thread.  Never NULL. */
const char *ddlr_last_error(ddlr_handle h);

/* Frees every device and host resource of the handle (NULL is a no-op). */
ddlr_status ddlr_destroy(ddlr_handle h);

/* ------------------------------------------------------------- serving
 * A solve service on one GPU (no counterpart in the paper; it serves many
 * solves with resident preconditioners, the amortisation the paper's
 * conclusion points to).  Every model (a matrix with its DDLR setup) stays
 * resident and has a worker thread with its own CUDA stream.  Requests are
 * queued per model.  A worker runs a block PCG whose columns are slots
 * (continuous batching): every few iterations it hands back the columns that
 * have converged and admits queued requests of its model into the free slots,
 * so a request waits for a free slot, never for a whole batch; with every slot
 * busy and requests waiting, the block is widened (up to max_batch columns)
 * without disturbing the running columns.  At most max_concurrent models hold
 * a block on the GPU at once, overlapping across models; while another model
 * waits for a place, a block admits nothing more and gives its place back
 * once it drains.  A block is opened or
 * widened only as far as its workspace fits in memory_fraction of the free
 * device memory.  A request's result does not depend on when it was admitted
 * or on the other requests of its block. */
typedef struct ddlr_server_ctx *ddlr_server;

typedef struct {
  int max_concurrent;      /* models with a block on the GPU at once (default 8) */
  int max_batch;           /* columns (slots) of a model's block, 1..64 (16)    */
  double tol;              /* relative residual target (1e-8)                   */
  int maxit;               /* iteration cap (500)                               */
  double memory_fraction;  /* share of free device memory usable (0.9)          */
} ddlr_server_options;

ddlr_status ddlr_server_options_default(ddlr_server_options *opt);

/* Creates a server on the current device.  Errors: INVALID (bad options). */
ddlr_status ddlr_server_create(const ddlr_server_options *opt, ddlr_server *out);

/* Sets up and keeps resident the preconditioner of one matrix (arguments as
 * ddlr_setup); *model receives its index.  Synchronous.  OOM if its estimated
 * footprint does not fit in the memory the server may use. */
ddlr_status ddlr_server_add_model(ddlr_server s, int n, const int *rowptr,
                                  const int *colind, const double *val,
                                  const int *part, int p,
                                  const ddlr_options *opt, int *model);

/* Queues the solve A x = b for a model; b (host, original order, n values) is
 * copied.  *request receives the request id.  Returns at once. */
ddlr_status ddlr_server_submit(ddlr_server s, int model, const double *b,
                               long long *request);

/* Waits for a request (timeout_s <= 0: no limit; TIMEOUT when it expires),
 * copies x (host, n values; may be NULL), its solve info (relres: the true
 * residual of the check that ended the solve; for NOCONV the recursive one),
 * the latency from submit to completion in seconds and the width of the block
 * when it finished, then forgets the request.  Returns the request's solve
 * status. */
ddlr_status ddlr_server_wait(ddlr_server s, long long request, double timeout_s,
                             double *x, ddlr_solve_info *info,
                             double *latency_s, int *batch);

/* Completed requests, most occupied slots of one block and most blocks on
 * the GPU seen, models, and the requests admitted into a block in which other
 * requests were running (continuous batching at work). */
ddlr_status ddlr_server_stats(ddlr_server s, long long *completed,
                              int *max_batch_seen, int *max_inflight_seen,
                              int *nmodels, long long *admitted_running);

/* Text of the server's last error (never NULL). */
const char *ddlr_server_last_error(ddlr_server s);

/* Stops the workers (queued requests are dropped) and frees every model. */
ddlr_status ddlr_server_destroy(ddlr_server s);

#ifdef __cplusplus
}
#endif
#endif /* DDLR_H */
