/*
 * ddlr_oracle.c -- plain, slow, FP64 CPU oracle of the DDLR preconditioner
 * (Li & Saad, "Low-rank correction methods for algebraic domain decomposition
 * preconditioners").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the product path never does.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every routine follows the paper's statement of the method step by step, in
 * the paper's notation, with no blocking, fusion or reordering:
 *   - Sec. 2.1-2.2 (eq. locsys2, Bmat): interior / interface classification and
 *     the global reordering (all interiors by subdomain, then all interfaces);
 *   - Sec. 3.1 (eq. EF, split): E = [a^-1 Ehat ; -a I],
 *     A0 = blkdiag(B + a^-2 Ehat Ehat^T, C + a^2 I), A = A0 - E E^T;
 *   - Sec. 4.1, 5: local solvers = incomplete Cholesky IC(0) on the pattern
 *     (or on the level-of-fill pattern of a given level, or exact Cholesky,
 *     dense), or for indefinite blocks incomplete LDL^T on the same patterns
 *     (or exact LDL^T, dense, no pivoting), one factor per
 *     B_{i,a} and one for C_a, each in its elimination order (ascending
 *     index, or multicolour);
 *   - Sec. 4.4 (eq. converge): Lanczos on H = E^T A0^-1 E (DDLR-1) or on
 *     E^T A0^-2 E (DDLR-2), with full reorthogonalisation (two classical
 *     Gram-Schmidt passes), convergence checked every `check` steps;
 *   - Sec. 3.2 (prop. gkt, Algorithm 1): DDLR-1 apply with
 *     G_{k,theta}^-1 = (1-theta)^-1 I + U_k [(I-L_k)^-1 - (1-theta)^-1 I] U_k^T;
 *   - Sec. 3.3 (eq. Form2a, lemma 1): DDLR-2 apply A0^-1 + U_k H_k U_k^T with
 *     U_k = A0^-1 E V_k and H_k = (I - U_k^T E V_k)^-1;
 *   - Sec. 4.3: the solve with C_a by a factorisation (c_solver 0) or by
 *     preconditioned Chebyshev iterations (c_solver 1) with the block Jacobi
 *     preconditioner D_a (the diagonal blocks of C_a that couple interface
 *     nodes of one subdomain), the spectrum of the pair (C_a, D_a) estimated
 *     by a few Lanczos steps with residual-norm safeguards, or by the
 *     approximate inverse of self-preconditioned MR iterations with
 *     dual-threshold dropping (c_solver 2, Algorithm 2);
 *   - Sec. 5: preconditioned CG from x0 = 0; for indefinite problems (or a
 *     preconditioner that is not SPD) restarted GMRES(m), right-preconditioned,
 *     from x0 = 0, with the setup accepting Ritz values >= 1 (DDLR-1) and an
 *     indefinite I - K (DDLR-2, inverted by Gaussian elimination with partial
 *     pivoting).
 *
 * Readings where the paper is silent are the same as the CUDA library's and are
 * listed with the design notes: natural (ascending original index) elimination
 * order inside interior blocks (b_order 0) or multicolour (b_order 1: the two
 * colour classes of a bipartite block graph, else a greedy colouring);
 * C_a factored like a local block, in ascending original index (c_order 0) or
 * multicolour order (c_order 1); Lanczos
 * start vector from SplitMix64; breakdown restarts; theta = Ritz_{k+1}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_NOMEM = 2, OR_BREAKDOWN = 3,
       OR_NOT_SPD = 4, OR_NOCONV = 5 };

/* ---------------------------------------------------------------- sparse */
typedef struct {
  int nr;       /* rows */
  int *rp;      /* nr+1 */
  int *ci;      /* column indices, ascending in each row */
  double *va;
} sp;

static void sp_free(sp *a) {
  free(a->rp); free(a->ci); free(a->va);
  a->rp = NULL; a->ci = NULL; a->va = NULL; a->nr = 0;
}

/* coordinate entry used to assemble matrices; duplicates are summed */
typedef struct { int r, c; double v; } trip;

static int trip_cmp(const void *a, const void *b) {
  const trip *x = (const trip *)a, *y = (const trip *)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

/* builds CSR from triplets (sorted, duplicates summed) */
static int sp_from_trips(sp *out, int nr, trip *t, long nt) {
  qsort(t, (size_t)nt, sizeof(trip), trip_cmp);
  long nu = 0;
  for (long q = 0; q < nt; q++) {
    if (nu > 0 && t[nu - 1].r == t[q].r && t[nu - 1].c == t[q].c)
      t[nu - 1].v += t[q].v;
    else
      t[nu++] = t[q];
  }
  out->nr = nr;
  out->rp = (int *)calloc((size_t)nr + 1, sizeof(int));
  out->ci = (int *)malloc(sizeof(int) * (size_t)(nu > 0 ? nu : 1));
  out->va = (double *)malloc(sizeof(double) * (size_t)(nu > 0 ? nu : 1));
  if (!out->rp || !out->ci || !out->va) return OR_NOMEM;
  for (long q = 0; q < nu; q++) out->rp[t[q].r + 1]++;
  for (int i = 0; i < nr; i++) out->rp[i + 1] += out->rp[i];
  for (long q = 0; q < nu; q++) { out->ci[q] = t[q].c; out->va[q] = t[q].v; }
  return OR_OK;
}

/* y = M x for an nr-row CSR */
static void sp_mv(const sp *M, const double *x, double *y) {
  for (int i = 0; i < M->nr; i++) {
    double acc = 0.0;
    for (int q = M->rp[i]; q < M->rp[i + 1]; q++) acc += M->va[q] * x[M->ci[q]];
    y[i] = acc;
  }
}

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* ---------------------------------------------------- SplitMix64 (Steele et
 * al. 2014): output i of stream `seed` is mix(seed + (i+1)*gamma). */
static uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double sm64_pm1(uint64_t seed, uint64_t i) {
  return 2.0 * ((double)(sm64(seed, i) >> 11) * 0x1.0p-53) - 1.0;
}

/* ------------------------------------------------------------ block factor */
typedef struct {
  int nb;        /* block size */
  int *ord;      /* ord[e] = block-local row (eq. Bmat order) eliminated e-th */
  int exact;     /* 1: dense factor, 0: incomplete on the pattern */
  int ldl;       /* 1: L D L^T with unit L, d_i stored in the diagonal slot */
  sp L;          /* incomplete: rows in elimination order, lower part incl. diagonal */
  double *D;     /* exact: dense nb x nb lower factor, row-major */
} blockfac;

/* IC(0) of the symmetric matrix S (elimination-ordered, full storage):
 *   l_ij = (s_ij - sum_{t<j, t in P_i and P_j} l_it l_jt) / l_jj   (j < i)
 *   l_ii = sqrt(s_ii - sum_{t<i} l_it^2)
 * over the lower pattern P_i of S; a pivot <= 0 is a breakdown. */
static int ic0_pattern(const sp *S, sp *L);

static int ic0(const sp *S, sp *L) {
  int st = ic0_pattern(S, L);
  if (st != OR_OK) return st;
  int n = S->nr;
  for (int i = 0; i < n; i++) {
    int b = L->rp[i], e = L->rp[i + 1];   /* diagonal is the last entry */
    for (int q = b; q < e - 1; q++) {
      int j = L->ci[q];
      double s = L->va[q];
      /* merge row i (entries before q) with row j (entries before its diag) */
      int qa = b, qb = L->rp[j], eb = L->rp[j + 1] - 1;
      while (qa < q && qb < eb) {
        if (L->ci[qa] == L->ci[qb]) { s -= L->va[qa] * L->va[qb]; qa++; qb++; }
        else if (L->ci[qa] < L->ci[qb]) qa++;
        else qb++;
      }
      L->va[q] = s / L->va[L->rp[j + 1] - 1];
    }
    double d = L->va[e - 1];
    for (int q = b; q < e - 1; q++) d -= L->va[q] * L->va[q];
    if (!(d > 0.0)) return OR_BREAKDOWN;
    L->va[e - 1] = sqrt(d);
  }
  return OR_OK;
}

/* the lower part of S (incl. diagonal) copied into L, rows in order */
static int ic0_pattern(const sp *S, sp *L) {
  int n = S->nr;
  long nnz = 0;
  for (int i = 0; i < n; i++)
    for (int q = S->rp[i]; q < S->rp[i + 1]; q++)
      if (S->ci[q] <= i) nnz++;
  L->nr = n;
  L->rp = (int *)calloc((size_t)n + 1, sizeof(int));
  L->ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  L->va = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!L->rp || !L->ci || !L->va) return OR_NOMEM;
  long w = 0;
  for (int i = 0; i < n; i++) {
    int has_diag = 0;
    for (int q = S->rp[i]; q < S->rp[i + 1]; q++)
      if (S->ci[q] <= i) {
        L->ci[w] = S->ci[q]; L->va[w] = S->va[q]; w++;
        if (S->ci[q] == i) has_diag = 1;
      }
    if (!has_diag) return OR_BREAKDOWN;
    L->rp[i + 1] = (int)w;
  }
  return OR_OK;
}

/* dense Cholesky S = L L^T (row-major lower); pivot <= 0 is a breakdown */
static int chol_dense(int n, double *a) {
  for (int j = 0; j < n; j++) {
    double d = a[(size_t)j * n + j];
    for (int t = 0; t < j; t++) d -= a[(size_t)j * n + t] * a[(size_t)j * n + t];
    if (!(d > 0.0)) return OR_BREAKDOWN;
    d = sqrt(d);
    a[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double s = a[(size_t)i * n + j];
      for (int t = 0; t < j; t++) s -= a[(size_t)i * n + t] * a[(size_t)j * n + t];
      a[(size_t)i * n + j] = s / d;
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) a[(size_t)i * n + j] = 0.0;
  return OR_OK;
}

/* The pattern of an incomplete factor with level of fill kf (the symmetric
 * form of the level-of-fill rule): entries of S have level 0; entry (i, j),
 * j < i, of the up-looking factor receives level lev(i,t) + lev(j,t) + 1 for
 * every t < j with (i, t) and (j, t) in the pattern, the smallest one
 * counting, and is kept when that level is <= kf.  Rows are built in order,
 * columns ascending, every row scanning all earlier columns: slow and plain.
 * out = S plus an explicit zero at every kept fill position (lower part). */
static int fill_pattern(const sp *S, int kf, sp *out) {
  int n = S->nr;
  const int INF = 1 << 29;
  int **kc = (int **)calloc((size_t)n + 1, sizeof(int *));   /* kept columns of each row, ascending */
  int **kl = (int **)calloc((size_t)n + 1, sizeof(int *));   /* and their levels */
  int *kn = (int *)calloc((size_t)n + 1, sizeof(int));
  int *lev = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  long nfill = 0;
  for (int i = 0; i < n; i++) {
    for (int c = 0; c < i; c++) lev[c] = INF;
    for (int q = S->rp[i]; q < S->rp[i + 1]; q++)
      if (S->ci[q] < i) lev[S->ci[q]] = 0;
    int cnt = 0;
    for (int j = 0; j < i; j++) {
      /* row j's kept entries (j, t), t < j, against row i's kept (i, t) */
      for (int a = 0; a < kn[j]; a++) {
        int t = kc[j][a];
        if (lev[t] <= kf && lev[t] + kl[j][a] + 1 < lev[j]) lev[j] = lev[t] + kl[j][a] + 1;
      }
      if (lev[j] <= kf) cnt++;
    }
    kc[i] = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    kl[i] = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    for (int j = 0; j < i; j++)
      if (lev[j] <= kf) {
        kc[i][kn[i]] = j; kl[i][kn[i]] = lev[j]; kn[i]++;
        if (lev[j] > 0) nfill++;
      }
  }
  long nt = S->rp[n] + nfill;
  trip *t = (trip *)malloc(sizeof(trip) * (size_t)(nt > 0 ? nt : 1));
  long w = 0;
  for (int i = 0; i < n; i++) {
    for (int q = S->rp[i]; q < S->rp[i + 1]; q++) { t[w].r = i; t[w].c = S->ci[q]; t[w].v = S->va[q]; w++; }
    for (int a = 0; a < kn[i]; a++)
      if (kl[i][a] > 0) { t[w].r = i; t[w].c = kc[i][a]; t[w].v = 0.0; w++; }
  }
  memset(out, 0, sizeof *out);
  int st = sp_from_trips(out, n, t, w);
  for (int i = 0; i < n; i++) { free(kc[i]); free(kl[i]); }
  free(kc); free(kl); free(kn); free(lev); free(t);
  return st;
}

/* incomplete LDL^T of S on its lower pattern P (same storage as ic0, d_i in
 * the diagonal slot, L unit lower):
 *   l_ij = (s_ij - sum_{t<j, t in P_i and P_j} l_it d_t l_jt) / d_j   (j < i)
 *   d_i  = s_ii - sum_{t<i} l_it^2 d_t
 * for symmetric indefinite blocks (Sec. 5: "incomplete Cholesky or LDL");
 * no pivoting, a zero (or non-finite) pivot is a breakdown. */
static int ildl0(const sp *S, sp *L) {
  int st = ic0_pattern(S, L);
  if (st != OR_OK) return st;
  int n = S->nr;
  for (int i = 0; i < n; i++) {
    int b = L->rp[i], e = L->rp[i + 1];
    for (int q = b; q < e - 1; q++) {
      int j = L->ci[q];
      double s = L->va[q];
      int qa = b, qb = L->rp[j], eb = L->rp[j + 1] - 1;
      while (qa < q && qb < eb) {
        if (L->ci[qa] == L->ci[qb]) {
          s -= L->va[qa] * L->va[L->rp[L->ci[qa] + 1] - 1] * L->va[qb];
          qa++; qb++;
        } else if (L->ci[qa] < L->ci[qb]) qa++;
        else qb++;
      }
      L->va[q] = s / L->va[eb];
    }
    double d = L->va[e - 1];
    for (int q = b; q < e - 1; q++) d -= L->va[q] * L->va[q] * L->va[L->rp[L->ci[q] + 1] - 1];
    if (!(d != 0.0) || !isfinite(d)) return OR_BREAKDOWN;
    L->va[e - 1] = d;
  }
  return OR_OK;
}

/* dense S = L D L^T without pivoting (row-major; unit L below the diagonal,
 * d_j on it); a zero or non-finite pivot is a breakdown */
static int ldl_dense(int n, double *a) {
  for (int j = 0; j < n; j++) {
    double d = a[(size_t)j * n + j];
    for (int t = 0; t < j; t++) d -= a[(size_t)j * n + t] * a[(size_t)j * n + t] * a[(size_t)t * n + t];
    if (!(d != 0.0) || !isfinite(d)) return OR_BREAKDOWN;
    a[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; i++) {
      double s = a[(size_t)i * n + j];
      for (int t = 0; t < j; t++) s -= a[(size_t)i * n + t] * a[(size_t)t * n + t] * a[(size_t)j * n + t];
      a[(size_t)i * n + j] = s / d;
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) a[(size_t)i * n + j] = 0.0;
  return OR_OK;
}

/* inverse of a dense n x n matrix (row-major, destroyed) by Gauss-Jordan
 * elimination with partial pivoting; a pivot of magnitude <= 1e-14 times the
 * largest entry of the matrix means singular (BREAKDOWN) */
static int gauss_jordan_inverse(int n, double *a, double *inv) {
  double amax = 0.0;
  for (int i = 0; i < n * n; i++) amax = fmax(amax, fabs(a[i]));
  for (int r = 0; r < n; r++)
    for (int c = 0; c < n; c++) inv[r * n + c] = (r == c) ? 1.0 : 0.0;
  for (int j = 0; j < n; j++) {
    int piv = j;
    for (int r = j + 1; r < n; r++)
      if (fabs(a[r * n + j]) > fabs(a[piv * n + j])) piv = r;
    if (!(fabs(a[piv * n + j]) > 1e-14 * amax)) return OR_BREAKDOWN;
    if (piv != j)
      for (int c = 0; c < n; c++) {
        double t = a[j * n + c]; a[j * n + c] = a[piv * n + c]; a[piv * n + c] = t;
        t = inv[j * n + c]; inv[j * n + c] = inv[piv * n + c]; inv[piv * n + c] = t;
      }
    double d = a[j * n + j];
    for (int c = 0; c < n; c++) { a[j * n + c] /= d; inv[j * n + c] /= d; }
    for (int r = 0; r < n; r++) {
      if (r == j) continue;
      double f = a[r * n + j];
      if (f == 0.0) continue;
      for (int c = 0; c < n; c++) { a[r * n + c] -= f * a[j * n + c]; inv[r * n + c] -= f * inv[j * n + c]; }
    }
  }
  return OR_OK;
}

/* solve (L L^T) x = b, or (L D L^T) x = b, in place, b in elimination order */
static void fac_solve(const blockfac *f, double *b) {
  int n = f->nb;
  if (f->ldl && f->exact) {
    const double *D = f->D;
    for (int i = 0; i < n; i++) {
      double s = b[i];
      for (int t = 0; t < i; t++) s -= D[(size_t)i * n + t] * b[t];
      b[i] = s;
    }
    for (int i = 0; i < n; i++) b[i] /= D[(size_t)i * n + i];
    for (int i = n - 1; i >= 0; i--) {
      double s = b[i];
      for (int t = i + 1; t < n; t++) s -= D[(size_t)t * n + i] * b[t];
      b[i] = s;
    }
  } else if (f->ldl) {
    const sp *L = &f->L;
    for (int i = 0; i < n; i++) {          /* L y = b, unit diagonal */
      double s = b[i];
      int e = L->rp[i + 1] - 1;
      for (int q = L->rp[i]; q < e; q++) s -= L->va[q] * b[L->ci[q]];
      b[i] = s;
    }
    for (int i = 0; i < n; i++) b[i] /= L->va[L->rp[i + 1] - 1];
    for (int i = n - 1; i >= 0; i--) {     /* L^T x = D^-1 y (column form) */
      int e = L->rp[i + 1] - 1;
      for (int q = L->rp[i]; q < e; q++) b[L->ci[q]] -= L->va[q] * b[i];
    }
  } else if (f->exact) {
    const double *D = f->D;
    for (int i = 0; i < n; i++) {
      double s = b[i];
      for (int t = 0; t < i; t++) s -= D[(size_t)i * n + t] * b[t];
      b[i] = s / D[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = b[i];
      for (int t = i + 1; t < n; t++) s -= D[(size_t)t * n + i] * b[t];
      b[i] = s / D[(size_t)i * n + i];
    }
  } else {
    const sp *L = &f->L;
    for (int i = 0; i < n; i++) {          /* forward: L y = b */
      double s = b[i];
      int e = L->rp[i + 1] - 1;
      for (int q = L->rp[i]; q < e; q++) s -= L->va[q] * b[L->ci[q]];
      b[i] = s / L->va[e];
    }
    for (int i = n - 1; i >= 0; i--) {     /* backward: L^T x = y (column form) */
      int e = L->rp[i + 1] - 1;
      b[i] = b[i] / L->va[e];
      for (int q = L->rp[i]; q < e; q++) b[L->ci[q]] -= L->va[q] * b[i];
    }
  }
}

/* ------------------------------------------------------------------ oracle */
typedef struct {
  int n, p, s, m;
  int variant, k, theta_mode, factor, c_order, scale_diag;
  double alpha;
  int *perm;       /* new index (eq. Bmat order) -> original index */
  int *iperm;      /* original -> new */
  int *boff;       /* p+2 offsets; block p (interface) = [m, n) */
  double *dsc;     /* D^-1/2 by original index (scale_diag), else NULL */
  sp A;            /* original A (unscaled), for PCG */
  sp Ap;           /* (scaled) A in new order */
  sp Eh;           /* Ehat: m rows, columns 0..s-1 (= new index - m) */
  sp EhT;          /* Ehat^T: s rows, columns 0..m-1 */
  blockfac *bf;    /* p+1 local factors of A0 */
  int urows;       /* s (DDLR-1) or n (DDLR-2) */
  double *U;       /* urows x k, row-major, new order */
  double *lam;     /* k Ritz values (DDLR-1) */
  double theta;
  double *Hk;      /* k x k (DDLR-2) */
  int msteps;      /* Lanczos steps */
  int reorth2;     /* 1: two Gram-Schmidt passes every Lanczos step; 0: the
                      second pass only on cancellation (cgs_reorth) */
  long reorth_passes;  /* Gram-Schmidt passes of the Lanczos steps (not the
                          restart vectors, which always take two) */
  double *ritz;    /* all Ritz values of T_m, descending */
  int ncolors;     /* colours of C_a (c_order 1) */
  double *work;    /* n scratch */
  double *work2;   /* n scratch */
  /* Sec. 4.3, c_solver 1: bf[p] factors D_a; Ca is the whole C_a */
  int c_solver, cheb_t, cheb_m;
  int mr_iters, mr_lfil;        /* c_solver 2 */
  double mr_droptol;
  int *xcnt, **xrow;            /* X ~ C_a^-1 by columns: rows ascending */
  double **xval;
  sp Ca;           /* s x s, interface indices (new index - m) */
  double cheb_lo, cheb_hi;
} oracle;

void or_free(oracle *o);

/* z = F^-1 x for block b's factor F (x, z in the block's eq. Bmat order) */
static void block_solve(oracle *o, int b, const double *x, double *z) {
  blockfac *f = &o->bf[b];
  double *t = o->work2;
  for (int e = 0; e < f->nb; e++) t[e] = x[f->ord[e]];
  fac_solve(f, t);
  for (int e = 0; e < f->nb; e++) z[f->ord[e]] = t[e];
}

/* Chebyshev iteration for C_a x = y from x_0 = 0 with the preconditioner D_a
 * (factored as block p), for the eigenvalues of D_a^-1 C_a taken in
 * [lo, hi]: centre c = (hi+lo)/2, half-width d = (hi-lo)/2.  The error after
 * t steps is T_t((c - L)/d) / T_t(c/d) applied to the initial error, L the
 * operator D_a^-1 C_a.  The recurrence follows from the three-term recurrence
 * of the Chebyshev polynomials T_j, with r_j = T_j(c/d) / T_{j+1}(c/d):
 *   r_0 = d/c,   r_{j+1} = d / (2c - d r_j),
 *   x_1 = x_0 + s_0,  s_0 = (1/c) D^-1 y,
 *   s_j = r_j r_{j-1} s_{j-1} + 2/(2c - d r_{j-1}) D^-1 (y - C_a x_j),
 *   x_{j+1} = x_j + s_j,
 * written with d only in numerators, so d = 0 (a one-point spectrum) gives
 * plain Richardson steps with step 1/c. */
static void cheb_solve(oracle *o, const double *y, double *x) {
  int s = o->s, t = o->cheb_t;
  double c = 0.5 * (o->cheb_hi + o->cheb_lo), d = 0.5 * (o->cheb_hi - o->cheb_lo);
  double *r = (double *)malloc(sizeof(double) * (size_t)s);
  double *z = (double *)malloc(sizeof(double) * (size_t)s);
  double *sd = (double *)malloc(sizeof(double) * (size_t)s);
  double *cs = (double *)malloc(sizeof(double) * (size_t)s);
  block_solve(o, o->p, y, z);
  for (int i = 0; i < s; i++) { sd[i] = z[i] / c; x[i] = sd[i]; r[i] = y[i]; }
  double rho = d / c;
  for (int j = 1; j < t; j++) {
    sp_mv(&o->Ca, sd, cs);                       /* r_j = r_{j-1} - C_a s_{j-1} */
    for (int i = 0; i < s; i++) r[i] -= cs[i];
    block_solve(o, o->p, r, z);
    double den = 2.0 * c - d * rho;
    double rho_n = d / den;
    for (int i = 0; i < s; i++) sd[i] = rho_n * rho * sd[i] + (2.0 / den) * z[i];
    for (int i = 0; i < s; i++) x[i] += sd[i];
    rho = rho_n;
  }
  free(r); free(z); free(sd); free(cs);
}

/* solve with C_a by the approximate inverse: z = X y, X by columns */
static void mr_apply(oracle *o, const double *y, double *z) {
  for (int i = 0; i < o->s; i++) z[i] = 0.0;
  for (int j = 0; j < o->s; j++)
    for (int t = 0; t < o->xcnt[j]; t++) z[o->xrow[j][t]] += o->xval[j][t] * y[j];
}

/* A0 solve in new order: p local solves with B_{i,a} and one with C_a */
static void a0_solve(oracle *o, const double *x, double *z) {
  for (int b = 0; b < o->p; b++) block_solve(o, b, x + o->boff[b], z + o->boff[b]);
  if (o->c_solver == 1) cheb_solve(o, x + o->m, z + o->m);
  else if (o->c_solver == 2) mr_apply(o, x + o->m, z + o->m);
  else block_solve(o, o->p, x + o->m, z + o->m);
}

/* Self-preconditioned global MR iterations with dual-threshold dropping
 * (Sec. 4.3, Algorithm 2) for X ~ C_a^-1, column by column:
 *   X_0 = diag(C_a)^-1;  for each of mr_iters iterations:
 *   R = I - C_a X,  Z = X R,  drop in Z,  beta = tr(R^T C_a Z) / ||C_a Z||_F^2,
 *   X = X + beta Z.
 * Dropping in column z_j: entries with |z_ij| <= mr_droptol ||z_j||_2 go,
 * then only the mr_lfil largest in magnitude stay (ties: lower row first).
 * tr(R^T C_a Z) = sum_j r_j . (C_a z_j) and ||C_a Z||_F^2 = sum_j ||C_a z_j||^2.
 * A zero ||C_a Z|| (R = 0 after dropping) ends the iterations. */
typedef struct { int i; double v; } ent;
static int ent_mag_cmp(const void *a, const void *b) {
  const ent *x = (const ent *)a, *y = (const ent *)b;
  double ax = fabs(x->v), ay = fabs(y->v);
  if (ax > ay) return -1;
  if (ax < ay) return 1;
  return (x->i > y->i) - (x->i < y->i);
}
static int ent_row_cmp(const void *a, const void *b) {
  const ent *x = (const ent *)a, *y = (const ent *)b;
  return (x->i > y->i) - (x->i < y->i);
}

static int mr_build(oracle *o) {
  int s = o->s;
  const sp *C = &o->Ca;
  o->xcnt = (int *)calloc((size_t)s, sizeof(int));
  o->xrow = (int **)calloc((size_t)s, sizeof(int *));
  o->xval = (double **)calloc((size_t)s, sizeof(double *));
  int *zcnt = (int *)calloc((size_t)s, sizeof(int));
  ent **zc = (ent **)calloc((size_t)s, sizeof(ent *));
  double *r = (double *)calloc((size_t)s, sizeof(double));
  double *z = (double *)calloc((size_t)s, sizeof(double));
  double *w = (double *)calloc((size_t)s, sizeof(double));
  ent *cand = (ent *)malloc(sizeof(ent) * (size_t)s);
  if (!o->xcnt || !o->xrow || !o->xval || !zcnt || !zc || !r || !z || !w || !cand) return OR_NOMEM;
  for (int j = 0; j < s; j++) {
    double cjj = 0.0;
    for (int q = C->rp[j]; q < C->rp[j + 1]; q++) if (C->ci[q] == j) cjj = C->va[q];
    o->xcnt[j] = 1;
    o->xrow[j] = (int *)malloc(sizeof(int));
    o->xval[j] = (double *)malloc(sizeof(double));
    o->xrow[j][0] = j;
    o->xval[j][0] = 1.0 / cjj;
  }
  for (int it = 0; it < o->mr_iters; it++) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j < s; j++) {
      /* r_j = e_j - C_a x_j */
      for (int i = 0; i < s; i++) { r[i] = 0.0; z[i] = 0.0; w[i] = 0.0; }
      r[j] = 1.0;
      for (int t = 0; t < o->xcnt[j]; t++) {
        int i = o->xrow[j][t];
        for (int q = C->rp[i]; q < C->rp[i + 1]; q++) r[C->ci[q]] -= C->va[q] * o->xval[j][t];
      }
      /* z_j = X r_j (self-preconditioned residual) */
      for (int l = 0; l < s; l++)
        if (r[l] != 0.0)
          for (int t = 0; t < o->xcnt[l]; t++) z[o->xrow[l][t]] += o->xval[l][t] * r[l];
      /* dual-threshold dropping */
      double nz2 = 0.0;
      for (int i = 0; i < s; i++) nz2 += z[i] * z[i];
      double thr = o->mr_droptol * sqrt(nz2);
      int nc = 0;
      for (int i = 0; i < s; i++)
        if (z[i] != 0.0 && fabs(z[i]) > thr) { cand[nc].i = i; cand[nc].v = z[i]; nc++; }
      qsort(cand, (size_t)nc, sizeof(ent), ent_mag_cmp);
      if (nc > o->mr_lfil) nc = o->mr_lfil;
      qsort(cand, (size_t)nc, sizeof(ent), ent_row_cmp);
      zcnt[j] = nc;
      zc[j] = (ent *)malloc(sizeof(ent) * (size_t)(nc > 0 ? nc : 1));
      memcpy(zc[j], cand, sizeof(ent) * (size_t)nc);
      /* w_j = C_a z_j; the trace and norm terms */
      for (int t = 0; t < nc; t++) {
        int i = cand[t].i;
        for (int q = C->rp[i]; q < C->rp[i + 1]; q++) w[C->ci[q]] += C->va[q] * cand[t].v;
      }
      for (int i = 0; i < s; i++) { num += r[i] * w[i]; den += w[i] * w[i]; }
    }
    if (!(den > 0.0)) {
      for (int j = 0; j < s; j++) free(zc[j]);
      break;
    }
    double beta = num / den;
    /* X = X + beta Z, column by column (rows stay ascending) */
    for (int j = 0; j < s; j++) {
      int na = o->xcnt[j], nb = zcnt[j], a = 0, b = 0, t = 0;
      int *ri = (int *)malloc(sizeof(int) * (size_t)(na + nb));
      double *rv = (double *)malloc(sizeof(double) * (size_t)(na + nb));
      while (a < na || b < nb) {
        if (b >= nb || (a < na && o->xrow[j][a] < zc[j][b].i)) { ri[t] = o->xrow[j][a]; rv[t] = o->xval[j][a]; a++; }
        else if (a >= na || zc[j][b].i < o->xrow[j][a]) { ri[t] = zc[j][b].i; rv[t] = beta * zc[j][b].v; b++; }
        else { ri[t] = o->xrow[j][a]; rv[t] = o->xval[j][a] + beta * zc[j][b].v; a++; b++; }
        t++;
      }
      free(o->xrow[j]); free(o->xval[j]); free(zc[j]);
      o->xrow[j] = ri; o->xval[j] = rv; o->xcnt[j] = t;
    }
  }
  free(zcnt); free(zc); free(r); free(z); free(w); free(cand);
  /* CG needs a symmetric preconditioner: the solve applies the symmetric
   * part (X + X^T) / 2 (dropping makes X itself unsymmetric) */
  long nt = 0;
  for (int j = 0; j < s; j++) nt += 2 * o->xcnt[j];
  trip *t = (trip *)malloc(sizeof(trip) * (size_t)(nt > 0 ? nt : 1));
  long w2 = 0;
  for (int j = 0; j < s; j++)
    for (int q = 0; q < o->xcnt[j]; q++) {
      int i = o->xrow[j][q];
      double v = 0.5 * o->xval[j][q];
      t[w2].r = j; t[w2].c = i; t[w2].v = v; w2++;   /* column j, row i */
      t[w2].r = i; t[w2].c = j; t[w2].v = v; w2++;   /* column i, row j */
    }
  sp S;
  memset(&S, 0, sizeof S);
  int st = sp_from_trips(&S, s, t, w2);
  free(t);
  if (st != OR_OK) return st;
  for (int j = 0; j < s; j++) {
    int cnt = S.rp[j + 1] - S.rp[j];
    free(o->xrow[j]); free(o->xval[j]);
    o->xrow[j] = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    o->xval[j] = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
    o->xcnt[j] = cnt;
    for (int q = 0; q < cnt; q++) { o->xrow[j][q] = S.ci[S.rp[j] + q]; o->xval[j][q] = S.va[S.rp[j] + q]; }
  }
  sp_free(&S);
  return OR_OK;
}

/* v = E w = [a^-1 Ehat w ; -a w]  (eq. EF), w of length s, v of length n */
static void e_mult(oracle *o, const double *w, double *v) {
  sp_mv(&o->Eh, w, v);
  for (int i = 0; i < o->m; i++) v[i] /= o->alpha;
  for (int j = 0; j < o->s; j++) v[o->m + j] = -o->alpha * w[j];
}

/* y = E^T z = a^-1 Ehat^T z_B - a z_C */
static void et_mult(oracle *o, const double *z, double *y) {
  sp_mv(&o->EhT, z, y);
  for (int j = 0; j < o->s; j++) y[j] = y[j] / o->alpha - o->alpha * z[o->m + j];
}

/* Lanczos operator: DDLR-1 H q = E^T A0^-1 E q; DDLR-2 E^T A0^-2 E q */
static void lanczos_op(oracle *o, const double *q, double *w) {
  double *v = (double *)malloc(sizeof(double) * (size_t)o->n);
  double *z = (double *)malloc(sizeof(double) * (size_t)o->n);
  e_mult(o, q, v);
  a0_solve(o, v, z);
  if (o->variant == 2) { a0_solve(o, z, v); memcpy(z, v, sizeof(double) * (size_t)o->n); }
  et_mult(o, z, w);
  free(v); free(z);
}

/* cyclic-by-row Jacobi eigen-decomposition of the dense symmetric m x m T:
 * on return diag(T) holds eigenvalues and the columns of V the vectors. */
static void jacobi_eig(int m, double *T, double *V) {
  for (int i = 0; i < m * m; i++) V[i] = 0.0;
  for (int i = 0; i < m; i++) V[i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double fro = 0.0;
    for (int i = 0; i < m * m; i++) fro += T[i] * T[i];
    fro = sqrt(fro);
    int rotated = 0;
    for (int p = 0; p < m - 1; p++)
      for (int q = p + 1; q < m; q++) {
        double apq = T[p * m + q];
        /* an entry below 1e-18 ||T||_F is already zero in double precision */
        if (fabs(apq) <= 1e-18 * fro) continue;
        rotated = 1;
        /* rotation zeroing T[p][q]: tau = (a_qq - a_pp)/(2 a_pq) */
        double tau = (T[q * m + q] - T[p * m + p]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < m; r++) {          /* T <- T J */
          double tp = T[r * m + p], tq = T[r * m + q];
          T[r * m + p] = c * tp - s * tq;
          T[r * m + q] = s * tp + c * tq;
        }
        for (int r = 0; r < m; r++) {          /* T <- J^T T */
          double tp = T[p * m + r], tq = T[q * m + r];
          T[p * m + r] = c * tp - s * tq;
          T[q * m + r] = s * tp + c * tq;
        }
        for (int r = 0; r < m; r++) {          /* V <- V J */
          double vp = V[r * m + p], vq = V[r * m + q];
          V[r * m + p] = c * vp - s * vq;
          V[r * m + q] = s * vp + c * vq;
        }
        T[p * m + q] = 0.0;   /* annihilated by construction */
        T[q * m + p] = 0.0;
      }
    if (!rotated) break;
  }
}

/* eigen-pairs of the tridiagonal T_m (alpha_1..m, beta_1..m-1), sorted
 * descending; ties keep the eigensolver's index order. vals[m], vecs m x m
 * (column c = c-th largest) when vecs != NULL. */
static void tri_eig(int m, const double *al, const double *be, double *vals, double *vecs) {
  double *T = (double *)calloc((size_t)m * m, sizeof(double));
  double *V = (double *)calloc((size_t)m * m, sizeof(double));
  int *idx = (int *)malloc(sizeof(int) * (size_t)m);
  for (int i = 0; i < m; i++) {
    T[i * m + i] = al[i];
    if (i + 1 < m) { T[i * m + i + 1] = be[i]; T[(i + 1) * m + i] = be[i]; }
  }
  jacobi_eig(m, T, V);
  for (int i = 0; i < m; i++) idx[i] = i;
  for (int i = 1; i < m; i++) {          /* stable insertion sort, descending */
    int v = idx[i], j = i - 1;
    while (j >= 0 && T[idx[j] * m + idx[j]] < T[v * m + v]) { idx[j + 1] = idx[j]; j--; }
    idx[j + 1] = v;
  }
  for (int c = 0; c < m; c++) {
    vals[c] = T[idx[c] * m + idx[c]];
    if (vecs)
      for (int r = 0; r < m; r++) vecs[r * m + c] = V[r * m + idx[c]];
  }
  free(T); free(V); free(idx);
}

static double topk_sum(int m, const double *al, const double *be, int k) {
  double *v = (double *)malloc(sizeof(double) * (size_t)m);
  tri_eig(m, al, be, v, NULL);
  double s = 0.0;
  for (int i = 0; i < k && i < m; i++) s += v[i];
  free(v);
  return s;
}

/* one classical Gram-Schmidt pass: w -= Q_j (Q_j^T w) */
static void cgs_pass(int s, int j, const double *Q, double *w, double *c) {
  for (int i = 0; i < j; i++) c[i] = dot(s, Q + (size_t)i * s, w);
  for (int i = 0; i < j; i++)
    for (int r = 0; r < s; r++) w[r] -= c[i] * Q[(size_t)i * s + r];
}

/* w -= Q_j (Q_j^T w), twice (classical Gram-Schmidt, two passes) */
static void cgs2(int s, int j, const double *Q, double *w, double *c) {
  cgs_pass(s, j, Q, w, c);
  cgs_pass(s, j, Q, w, c);
}

/* Full reorthogonalisation of the Lanczos vector w against Q_j.  always2:
 * two classical Gram-Schmidt passes.  Otherwise the second pass runs only
 * when the first one shrank w below 1/sqrt(2) of its norm, i.e.
 * ||w'||^2 < ||w||^2 / 2 (the criterion of Daniel, Gragg, Kaufman and
 * Stewart, 1976): without that much cancellation one pass already leaves w
 * orthogonal to Q_j to working precision.  Returns the number of passes. */
static int cgs_reorth(int s, int j, const double *Q, double *w, double *c, int always2) {
  double w0 = dot(s, w, w);
  cgs_pass(s, j, Q, w, c);
  if (!always2) {
    double w1 = dot(s, w, w);
    if (!(w1 < 0.5 * w0)) return 1;
  }
  cgs_pass(s, j, Q, w, c);
  return 2;
}

/* Lanczos with full reorthogonalisation (Sec. 4.4).  Q is s x mmax, column-
 * major.  Returns the number of steps m and the tridiagonal (al, be). */
static int lanczos(oracle *o, int k, int mmax, int check, double eps, uint64_t seed,
                   double *Q, double *al, double *be) {
  const int always2 = o->reorth2;
  int s = o->s;
  double *w = (double *)malloc(sizeof(double) * (size_t)s);
  double *c = (double *)malloc(sizeof(double) * (size_t)(mmax + 1));
  uint64_t restart = 0;
  for (int r = 0; r < s; r++) Q[r] = sm64_pm1(seed + restart, (uint64_t)r);
  double nq = sqrt(dot(s, Q, Q));
  for (int r = 0; r < s; r++) Q[r] /= nq;
  double scale = 0.0;
  int m = 0;
  double sig_prev = 0.0;
  int have_prev = 0;
  for (int j = 0; j < mmax; j++) {       /* step j+1 in the paper's 1-based count */
    double *q = Q + (size_t)j * s;
    lanczos_op(o, q, w);
    al[j] = dot(s, q, w);
    for (int r = 0; r < s; r++) w[r] -= al[j] * q[r];
    if (j > 0)
      for (int r = 0; r < s; r++) w[r] -= be[j - 1] * Q[(size_t)(j - 1) * s + r];
    o->reorth_passes += cgs_reorth(s, j + 1, Q, w, c, always2);
    double b = sqrt(dot(s, w, w));
    if (fabs(al[j]) > scale) scale = fabs(al[j]);
    m = j + 1;
    /* convergence test of eq. (converge) every `check` steps once m > k */
    if (check > 0 && m % check == 0 && m >= k + 1) {
      double sig = topk_sum(m, al, be, k);
      double sp_ = topk_sum(m - 1, al, be, k);
      (void)have_prev; (void)sig_prev;
      if (fabs(sig - sp_) < eps * fabs(sp_)) { be[j] = b; break; }
    }
    if (m == mmax) { be[j] = b; break; }
    if (b <= 1e-12 * (scale > 0 ? scale : 1.0)) {
      /* breakdown: invariant subspace found; continue from a fresh random
       * vector orthogonalised against Q_j, with beta_j = 0 */
      be[j] = 0.0;
      restart++;
      for (int r = 0; r < s; r++) w[r] = sm64_pm1(seed + restart, (uint64_t)r);
      cgs2(s, j + 1, Q, w, c);
      b = sqrt(dot(s, w, w));
      double *qn = Q + (size_t)(j + 1) * s;
      for (int r = 0; r < s; r++) qn[r] = w[r] / b;
    } else {
      be[j] = b;
      if (b > scale) scale = b;
      double *qn = Q + (size_t)(j + 1) * s;
      for (int r = 0; r < s; r++) qn[r] = w[r] / b;
    }
  }
  free(w); free(c);
  return m;
}

/* Spectrum estimate of D_a^-1 C_a (Sec. 4.3): Lanczos on the pair (C_a, D_a),
 * i.e. symmetric Lanczos in the D_a inner product, for cheb_m steps (fewer at
 * an invariant subspace), from the SplitMix64 stream seed + 2^32 taken in
 * ascending original index of the interface nodes.  With p_j = D_a q_j:
 *   w = C_a q_j - beta_{j-1} p_{j-1},  alpha_j = q_j^T w,  w -= alpha_j p_j,
 *   z = D_a^-1 w,  beta_j = sqrt(w^T z),  q_{j+1} = z / beta_j,
 *   p_{j+1} = w / beta_j.
 * Ritz values of T_m are estimates, not bounds; each Ritz value lies within
 * beta_m |e_m^T y| of an eigenvalue (y its unit eigenvector of T_m), so the
 * interval is widened by that residual norm at both ends.  A lower end that
 * the widening takes to zero or below falls back to the smallest Ritz value. */
static int cheb_estimate(oracle *o, uint64_t seed) {
  int s = o->s, mmax = o->cheb_m;
  double *r = (double *)malloc(sizeof(double) * (size_t)s);
  double *z = (double *)malloc(sizeof(double) * (size_t)s);
  double *q = (double *)malloc(sizeof(double) * (size_t)s);
  double *pv = (double *)malloc(sizeof(double) * (size_t)s);
  double *pp = (double *)calloc((size_t)s, sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (size_t)s);
  double *al = (double *)calloc((size_t)mmax + 1, sizeof(double));
  double *be = (double *)calloc((size_t)mmax + 1, sizeof(double));
  if (!r || !z || !q || !pv || !pp || !w || !al || !be) return OR_NOMEM;
  /* start vector in ascending original index: the interface part of the new
   * order is already ascending */
  for (int j = 0; j < s; j++) r[j] = sm64_pm1(seed + 0x100000000ULL, (uint64_t)j);
  block_solve(o, o->p, r, z);
  double beta = sqrt(dot(s, r, z)), scale = 0.0;
  int m = 0;
  for (int j = 0; j < mmax; j++) {
    for (int i = 0; i < s; i++) { q[i] = z[i] / beta; pv[i] = r[i] / beta; }
    sp_mv(&o->Ca, q, w);
    if (j > 0) for (int i = 0; i < s; i++) w[i] -= be[j - 1] * pp[i];
    al[j] = dot(s, q, w);
    for (int i = 0; i < s; i++) w[i] -= al[j] * pv[i];
    block_solve(o, o->p, w, z);
    double ww = dot(s, w, z);
    be[j] = ww > 0.0 ? sqrt(ww) : 0.0;
    m = j + 1;
    if (fabs(al[j]) > scale) scale = fabs(al[j]);
    if (be[j] <= 1e-14 * scale) break;      /* invariant subspace: T_m is exact */
    memcpy(pp, pv, sizeof(double) * (size_t)s);
    memcpy(r, w, sizeof(double) * (size_t)s);
    beta = be[j];
  }
  double *vals = (double *)malloc(sizeof(double) * (size_t)m);
  double *vecs = (double *)malloc(sizeof(double) * (size_t)m * m);
  tri_eig(m, al, be, vals, vecs);
  double bm = be[m - 1];
  o->cheb_hi = vals[0] + bm * fabs(vecs[(size_t)(m - 1) * m + 0]);
  o->cheb_lo = vals[m - 1] - bm * fabs(vecs[(size_t)(m - 1) * m + (m - 1)]);
  if (!(o->cheb_lo > 0.0)) o->cheb_lo = vals[m - 1];
  free(r); free(z); free(q); free(pv); free(pp); free(w); free(al); free(be); free(vals); free(vecs);
  return (o->cheb_lo > 0.0 && o->cheb_hi >= o->cheb_lo) ? OR_OK : OR_NOT_SPD;
}

/* Randomized subspace iteration for the low-rank part (the randomized
 * techniques the conclusion names as a faster alternative to Lanczos; the
 * method of Halko, Martinsson and Tropp): with the operator Op of the
 * Lanczos process (H = E^T A0^-1 E, or E^T A0^-2 E for DDLR-2),
 *   Omega = s x ell test matrix, column c = SplitMix64 stream seed + 2^33 + c
 *           over the interface nodes in ascending original index;
 *   Q = orth(Op Omega); q times: Q = orth(Op Q);
 *   B = Q^T (Op Q), symmetrised; B = Y diag(theta) Y^T, theta descending.
 * orth = the QR factor with positive diagonal R (classical Gram-Schmidt,
 * two passes, column by column).  Q is s x ell column-major, Y ell x ell
 * row-major (Y[j * ell + c] = component j of vector c), as tri_eig gives. */
static void orth_cols(int s, int ell, double *Q) {
  double *c = (double *)malloc(sizeof(double) * (size_t)(ell + 1));
  for (int j = 0; j < ell; j++) {
    double *w = Q + (size_t)j * s;
    cgs2(s, j, Q, w, c);
    double nw = sqrt(dot(s, w, w));
    for (int r = 0; r < s; r++) w[r] /= nw;
  }
  free(c);
}

/* Lanczos (Golub-Kahan) bidiagonalisation of K = A0^-1 E (n x s) for DDLR-2
 * (Sec. 4.4, the alternative that yields U_k and V_k together):
 *   v_1 = the Lanczos start vector;  for j = 1, 2, ...:
 *   u = K v_j - beta_{j-1} u_{j-1},  alpha_j = ||u||,  u_j = u / alpha_j;
 *   v = K^T u_j - alpha_j v_j,       beta_j = ||v||,   v_{j+1} = v / beta_j;
 * with both sequences fully reorthogonalised (two classical Gram-Schmidt
 * passes).  K V_m = U_m B_m with B_m upper bidiagonal (alpha on the diagonal,
 * beta above it), so B_m^T B_m (diagonal alpha_j^2 + beta_{j-1}^2, off-
 * diagonal alpha_j beta_j) is the tridiagonal matrix Lanczos on
 * K^T K = E^T A0^-2 E would give from the same start.  The convergence test
 * of eq. converge runs on its eigenvalues; a beta_j or alpha_j at or below
 * 1e-12 of the largest seen ends the process (invariant subspace).  V is
 * s x (mmax+1) and U n x mmax, column-major; td / te receive B_m^T B_m. */
static int lbd(oracle *o, int k, int mmax, int check, double eps, uint64_t seed, double *V, double *U,
               double *td, double *te) {
  int s = o->s, n = o->n;
  double *al = (double *)calloc((size_t)mmax + 1, sizeof(double));
  double *be = (double *)calloc((size_t)mmax + 1, sizeof(double));
  double *u = (double *)malloc(sizeof(double) * (size_t)n);
  double *t = (double *)malloc(sizeof(double) * (size_t)n);
  double *v = (double *)malloc(sizeof(double) * (size_t)s);
  double *c = (double *)malloc(sizeof(double) * (size_t)(mmax + 2));
  for (int r = 0; r < s; r++) V[r] = sm64_pm1(seed, (uint64_t)r);
  double nv = sqrt(dot(s, V, V));
  for (int r = 0; r < s; r++) V[r] /= nv;
  double scale = 0.0;
  int m = 0;
  for (int j = 0; j < mmax; j++) {
    double *vj = V + (size_t)j * s;
    e_mult(o, vj, t);                         /* u = K v_j - beta_{j-1} u_{j-1} */
    a0_solve(o, t, u);
    if (j > 0) for (int r = 0; r < n; r++) u[r] -= be[j - 1] * U[(size_t)(j - 1) * n + r];
    cgs2(n, j, U, u, c);
    al[j] = sqrt(dot(n, u, u));
    if (al[j] > scale) scale = al[j];
    m = j + 1;
    if (!(al[j] > 1e-12 * scale)) { m = j; break; }
    for (int r = 0; r < n; r++) U[(size_t)j * n + r] = u[r] / al[j];
    a0_solve(o, U + (size_t)j * n, t);        /* v = K^T u_j - alpha_j v_j */
    et_mult(o, t, v);
    for (int r = 0; r < s; r++) v[r] -= al[j] * vj[r];
    cgs2(s, j + 1, V, v, c);
    be[j] = sqrt(dot(s, v, v));
    if (be[j] > scale) scale = be[j];
    for (int i = 0; i < m; i++) {
      td[i] = al[i] * al[i] + (i > 0 ? be[i - 1] * be[i - 1] : 0.0);
      te[i] = al[i] * be[i];
    }
    if (check > 0 && m % check == 0 && m >= k + 1) {
      double sig = topk_sum(m, td, te, k);
      double spv = topk_sum(m - 1, td, te, k);
      if (fabs(sig - spv) < eps * fabs(spv)) break;
    }
    if (m == mmax || !(be[j] > 1e-12 * scale)) break;
    for (int r = 0; r < s; r++) V[(size_t)(j + 1) * s + r] = v[r] / be[j];
  }
  for (int i = 0; i < m; i++) {
    td[i] = al[i] * al[i] + (i > 0 ? be[i - 1] * be[i - 1] : 0.0);
    te[i] = al[i] * be[i];
  }
  /* B_m itself, for U_k = U_m (B_m Y_k): al and be kept behind td / te */
  for (int i = 0; i < m; i++) { td[mmax + 1 + i] = al[i]; te[mmax + 1 + i] = be[i]; }
  free(al); free(be); free(u); free(t); free(v); free(c);
  return m;
}

static void rand_subspace(oracle *o, int ell, int power, uint64_t seed, double *Q, double *vals, double *Y) {
  int s = o->s;
  double *W = (double *)malloc(sizeof(double) * (size_t)s * ell);
  for (int c = 0; c < ell; c++)
    for (int r = 0; r < s; r++) Q[(size_t)c * s + r] = sm64_pm1(seed + 0x200000000ULL + (uint64_t)c, (uint64_t)r);
  for (int c = 0; c < ell; c++) lanczos_op(o, Q + (size_t)c * s, W + (size_t)c * s);
  memcpy(Q, W, sizeof(double) * (size_t)s * ell);
  orth_cols(s, ell, Q);
  for (int it = 0; it < power; it++) {
    for (int c = 0; c < ell; c++) lanczos_op(o, Q + (size_t)c * s, W + (size_t)c * s);
    memcpy(Q, W, sizeof(double) * (size_t)s * ell);
    orth_cols(s, ell, Q);
  }
  for (int c = 0; c < ell; c++) lanczos_op(o, Q + (size_t)c * s, W + (size_t)c * s);
  double *B = (double *)malloc(sizeof(double) * (size_t)ell * ell);
  double *V = (double *)malloc(sizeof(double) * (size_t)ell * ell);
  for (int a = 0; a < ell; a++)
    for (int b = 0; b < ell; b++) B[a * ell + b] = dot(s, Q + (size_t)a * s, W + (size_t)b * s);
  for (int a = 0; a < ell; a++)
    for (int b = a + 1; b < ell; b++) {
      double v = 0.5 * (B[a * ell + b] + B[b * ell + a]);
      B[a * ell + b] = v; B[b * ell + a] = v;
    }
  jacobi_eig(ell, B, V);
  int *idx = (int *)malloc(sizeof(int) * (size_t)ell);
  for (int i = 0; i < ell; i++) idx[i] = i;
  for (int i = 1; i < ell; i++) {          /* stable insertion sort, descending */
    int v = idx[i], j = i - 1;
    while (j >= 0 && B[idx[j] * ell + idx[j]] < B[v * ell + v]) { idx[j + 1] = idx[j]; j--; }
    idx[j + 1] = v;
  }
  for (int c = 0; c < ell; c++) {
    vals[c] = B[idx[c] * ell + idx[c]];
    for (int r = 0; r < ell; r++) Y[r * ell + c] = V[r * ell + idx[c]];
  }
  free(W); free(B); free(V); free(idx);
}

/* ------------------------------------------------------------ public API */
int or_setup(int n, const int *rowptr, const int *colind, const double *val,
             const int *part, int p, int variant, int k, double alpha,
             int theta_mode, int factor, int c_order, int b_order, int scale_diag,
             int lanczos_max, int lanczos_check, double lanczos_eps,
             unsigned long long seed, int c_solver, int cheb_steps, int cheb_lanczos,
             int lowrank_method, int rand_oversample, int rand_power, int mr_iters, int mr_lfil,
             double mr_droptol, int indefinite, int fill_level, int lanczos_reorth, void **out) {
  *out = NULL;
  if (lanczos_reorth < 0 || lanczos_reorth > 1) return OR_INVALID;
  if (n <= 0 || p <= 0 || (variant != 1 && variant != 2) || k < 1 || !(alpha > 0))
    return OR_INVALID;
  if (c_solver < 0 || c_solver > 2 || (c_solver == 1 && (cheb_steps < 1 || cheb_lanczos < 1)) ||
      (c_solver == 2 && (mr_iters < 0 || mr_lfil < 1 || !(mr_droptol >= 0.0))))
    return OR_INVALID;
  if (lowrank_method < 0 || lowrank_method > 2 || rand_oversample < 0 || rand_power < 0) return OR_INVALID;
  if (lowrank_method == 2 && variant != 2) return OR_INVALID;   /* bidiagonalisation: DDLR-2 */
  if (factor < 0 || factor > 3 || fill_level < 0 || (fill_level > 0 && (factor == 1 || factor == 3)))
    return OR_INVALID;
  for (int i = 0; i < n; i++) {
    if (rowptr[i + 1] < rowptr[i]) return OR_INVALID;
    if (part[i] < 0 || part[i] >= p) return OR_INVALID;
    for (int q = rowptr[i]; q < rowptr[i + 1]; q++) {
      if (colind[q] < 0 || colind[q] >= n) return OR_INVALID;
      if (q > rowptr[i] && colind[q] <= colind[q - 1]) return OR_INVALID;
    }
  }
  /* symmetry of pattern and values */
  for (int i = 0; i < n; i++)
    for (int q = rowptr[i]; q < rowptr[i + 1]; q++) {
      int j = colind[q], found = 0;
      for (int t = rowptr[j]; t < rowptr[j + 1]; t++)
        if (colind[t] == i) { found = (val[t] == val[q]); break; }
      if (!found) return OR_INVALID;
    }
  oracle *o = (oracle *)calloc(1, sizeof(oracle));
  if (!o) return OR_NOMEM;
  o->n = n; o->p = p; o->variant = variant; o->k = k; o->alpha = alpha;
  o->theta_mode = theta_mode; o->factor = factor; o->c_order = c_order;
  o->scale_diag = scale_diag;
  o->c_solver = c_solver; o->cheb_t = cheb_steps; o->cheb_m = cheb_lanczos;
  o->mr_iters = mr_iters; o->mr_lfil = mr_lfil; o->mr_droptol = mr_droptol;
  o->reorth2 = lanczos_reorth;
  int st = OR_OK;
  long nnz = rowptr[n];

  /* original A (for PCG) */
  o->A.nr = n;
  o->A.rp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
  o->A.ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  o->A.va = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  memcpy(o->A.rp, rowptr, sizeof(int) * (size_t)(n + 1));
  memcpy(o->A.ci, colind, sizeof(int) * (size_t)nnz);
  memcpy(o->A.va, val, sizeof(double) * (size_t)nnz);

  /* optional symmetric diagonal scaling D^-1/2 A D^-1/2 */
  double *As = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  memcpy(As, val, sizeof(double) * (size_t)nnz);
  if (scale_diag) {
    o->dsc = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; i++) {
      double d = 0.0;
      for (int q = rowptr[i]; q < rowptr[i + 1]; q++) if (colind[q] == i) d = val[q];
      if (!(d > 0)) { free(As); or_free(o); return OR_INVALID; }
      o->dsc[i] = 1.0 / sqrt(d);
    }
    for (int i = 0; i < n; i++)
      for (int q = rowptr[i]; q < rowptr[i + 1]; q++)
        As[q] = val[q] * o->dsc[i] * o->dsc[colind[q]];
  }

  /* Sec. 2.1: node i is an interface node iff it couples to another part */
  int *iface = (int *)calloc((size_t)n, sizeof(int));
  for (int i = 0; i < n; i++)
    for (int q = rowptr[i]; q < rowptr[i + 1]; q++)
      if (part[colind[q]] != part[i]) iface[i] = 1;

  /* eq. (Bmat): interiors of subdomain 0..p-1 (ascending index), then all
   * interface nodes (ascending index) */
  o->perm = (int *)malloc(sizeof(int) * (size_t)n);
  o->iperm = (int *)malloc(sizeof(int) * (size_t)n);
  o->boff = (int *)malloc(sizeof(int) * (size_t)(p + 2));
  int w = 0;
  for (int b = 0; b < p; b++) {
    o->boff[b] = w;
    for (int i = 0; i < n; i++) if (part[i] == b && !iface[i]) o->perm[w++] = i;
  }
  o->boff[p] = w;
  o->m = w;
  for (int i = 0; i < n; i++) if (iface[i]) o->perm[w++] = i;
  o->boff[p + 1] = w;
  o->s = n - o->m;
  for (int g = 0; g < n; g++) o->iperm[o->perm[g]] = g;
  int m = o->m, s = o->s;
  if (s == 0) { free(As); free(iface); or_free(o); return OR_INVALID; }
  if (k > s) { free(As); free(iface); or_free(o); return OR_INVALID; }

  /* permuted (scaled) A */
  {
    trip *t = (trip *)malloc(sizeof(trip) * (size_t)(nnz > 0 ? nnz : 1));
    long nt = 0;
    for (int i = 0; i < n; i++)
      for (int q = rowptr[i]; q < rowptr[i + 1]; q++) {
        t[nt].r = o->iperm[i]; t[nt].c = o->iperm[colind[q]]; t[nt].v = As[q]; nt++;
      }
    sp_from_trips(&o->Ap, n, t, nt);
    free(t);
  }
  free(As);

  /* Ehat (m x s) and its transpose */
  {
    long ne = 0;
    for (int g = 0; g < m; g++)
      for (int q = o->Ap.rp[g]; q < o->Ap.rp[g + 1]; q++) if (o->Ap.ci[q] >= m) ne++;
    trip *t1 = (trip *)malloc(sizeof(trip) * (size_t)(ne > 0 ? ne : 1));
    trip *t2 = (trip *)malloc(sizeof(trip) * (size_t)(ne > 0 ? ne : 1));
    long nt = 0;
    for (int g = 0; g < m; g++)
      for (int q = o->Ap.rp[g]; q < o->Ap.rp[g + 1]; q++)
        if (o->Ap.ci[q] >= m) {
          t1[nt].r = g; t1[nt].c = o->Ap.ci[q] - m; t1[nt].v = o->Ap.va[q];
          t2[nt].r = o->Ap.ci[q] - m; t2[nt].c = g; t2[nt].v = o->Ap.va[q];
          nt++;
        }
    sp_from_trips(&o->Eh, m, t1, nt);
    sp_from_trips(&o->EhT, s, t2, nt);
    free(t1); free(t2);
  }

  /* local blocks of A0 (eq. split): B_{i,a} = B_i + a^-2 E_i E_i^T and
   * C_a = C + a^2 I.  Proposition (locality): Ehat Ehat^T has no coupling
   * between different subdomains; a violation is reported as INVALID. */
  o->bf = (blockfac *)calloc((size_t)(p + 1), sizeof(blockfac));
  o->work = (double *)malloc(sizeof(double) * (size_t)n);
  o->work2 = (double *)malloc(sizeof(double) * (size_t)n);
  int *blk = (int *)malloc(sizeof(int) * (size_t)n);
  for (int b = 0; b <= p; b++)
    for (int g = o->boff[b]; g < o->boff[b + 1]; g++) blk[g] = b;
  for (int b = 0; b <= p && st == OR_OK; b++) {
    int off = o->boff[b], nb = o->boff[b + 1] - off;
    blockfac *f = &o->bf[b];
    f->nb = nb;
    f->ord = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
    /* assemble the block in eq. Bmat (local) order */
    long cap = 16 + nb;
    for (int g = off; g < off + nb; g++) cap += o->Ap.rp[g + 1] - o->Ap.rp[g];
    if (b < p)
      for (int g = off; g < off + nb; g++)
        for (int q = o->Eh.rp[g]; q < o->Eh.rp[g + 1]; q++) {
          int j = o->Eh.ci[q];
          cap += o->EhT.rp[j + 1] - o->EhT.rp[j];
        }
    trip *t = (trip *)malloc(sizeof(trip) * (size_t)cap);
    long nt = 0;
    for (int g = off; g < off + nb; g++)
      for (int q = o->Ap.rp[g]; q < o->Ap.rp[g + 1]; q++) {
        int c = o->Ap.ci[q];
        if (c < off || c >= off + nb) continue;
        /* Chebyshev mode: block p is D_a, which keeps only the couplings
         * between interface nodes of the same subdomain */
        if (b == p && c_solver == 1 && part[o->perm[g]] != part[o->perm[c]]) continue;
        t[nt].r = g - off; t[nt].c = c - off; t[nt].v = o->Ap.va[q]; nt++;
      }
    if (b < p) {
      double ia2 = 1.0 / (alpha * alpha);
      for (int g = off; g < off + nb; g++)
        for (int q = o->Eh.rp[g]; q < o->Eh.rp[g + 1]; q++) {
          int j = o->Eh.ci[q];
          for (int t2 = o->EhT.rp[j]; t2 < o->EhT.rp[j + 1]; t2++) {
            int g2 = o->EhT.ci[t2];
            if (blk[g2] != b) { st = OR_INVALID; break; }
            t[nt].r = g - off; t[nt].c = g2 - off; t[nt].v = ia2 * o->Eh.va[q] * o->EhT.va[t2]; nt++;
          }
        }
    } else {
      for (int r = 0; r < nb; r++) { t[nt].r = r; t[nt].c = r; t[nt].v = alpha * alpha; nt++; }
    }
    sp B;
    memset(&B, 0, sizeof B);
    if (st == OR_OK) st = sp_from_trips(&B, nb, t, nt);
    free(t);
    if (st != OR_OK) { sp_free(&B); break; }

    /* elimination order: ascending index, or multicolour.  Multicolour: a
     * bipartite block graph is split into its two colour classes (each
     * connected component's lowest-index node in class 0); any other graph
     * is coloured greedily (ascending index, smallest colour no lower-indexed
     * neighbour has).  Nodes are then eliminated by colour, then index. */
    for (int e = 0; e < nb; e++) f->ord[e] = e;
    if ((b == p && c_order == 1) || (b < p && b_order == 1)) {
      int *col = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
      int *used = (int *)calloc((size_t)nb + 2, sizeof(int));
      int nc = 0;
      /* two-colouring: give every node the class its component's lowest node
       * forces, following edges from lower to higher visited nodes (a plain
       * depth-first walk with an explicit stack), and verify every edge */
      int *stack = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
      for (int r = 0; r < nb; r++) col[r] = -1;
      for (int r0 = 0; r0 < nb; r0++) {
        if (col[r0] >= 0) continue;
        int top = 0;
        col[r0] = 0;
        stack[top++] = r0;
        while (top > 0) {
          int u = stack[--top];
          for (int q = B.rp[u]; q < B.rp[u + 1]; q++) {
            int v = B.ci[q];
            if (v != u && col[v] < 0) { col[v] = 1 - col[u]; stack[top++] = v; }
          }
        }
      }
      int bip = 1;
      for (int r = 0; r < nb && bip; r++)
        for (int q = B.rp[r]; q < B.rp[r + 1]; q++)
          if (B.ci[q] != r && col[B.ci[q]] == col[r]) { bip = 0; break; }
      if (bip) {
        for (int r = 0; r < nb; r++) if (col[r] + 1 > nc) nc = col[r] + 1;
      } else {
        nc = 0;
        for (int r = 0; r < nb; r++) {
          for (int q = B.rp[r]; q < B.rp[r + 1]; q++)
            if (B.ci[q] < r) used[col[B.ci[q]]] = r + 1;
          int c = 0;
          while (used[c] == r + 1) c++;
          col[r] = c;
          if (c + 1 > nc) nc = c + 1;
        }
      }
      free(stack);
      if (b == p) o->ncolors = nc;
      int e = 0;
      for (int c = 0; c < nc; c++)
        for (int r = 0; r < nb; r++) if (col[r] == c) f->ord[e++] = r;
      free(col); free(used);
    }
    int *pos = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
    for (int e = 0; e < nb; e++) pos[f->ord[e]] = e;
    /* the block in elimination order */
    long bn = B.rp[nb];
    trip *t3 = (trip *)malloc(sizeof(trip) * (size_t)(bn > 0 ? bn : 1));
    long n3 = 0;
    for (int r = 0; r < nb; r++)
      for (int q = B.rp[r]; q < B.rp[r + 1]; q++) {
        t3[n3].r = pos[r]; t3[n3].c = pos[B.ci[q]]; t3[n3].v = B.va[q]; n3++;
      }
    sp S;
    memset(&S, 0, sizeof S);
    sp_from_trips(&S, nb, t3, n3);
    free(t3); free(pos); sp_free(&B);
    f->ldl = factor >= 2;
    if (factor == 1 || factor == 3) {
      f->exact = 1;
      f->D = (double *)calloc((size_t)nb * nb + 1, sizeof(double));
      if (!f->D) { st = OR_NOMEM; sp_free(&S); break; }
      for (int r = 0; r < nb; r++)
        for (int q = S.rp[r]; q < S.rp[r + 1]; q++) f->D[(size_t)r * nb + S.ci[q]] = S.va[q];
      st = factor == 3 ? ldl_dense(nb, f->D) : chol_dense(nb, f->D);
    } else if (fill_level > 0) {
      sp F;
      st = fill_pattern(&S, fill_level, &F);
      if (st == OR_OK) st = factor == 2 ? ildl0(&F, &f->L) : ic0(&F, &f->L);
      sp_free(&F);
    } else {
      st = factor == 2 ? ildl0(&S, &f->L) : ic0(&S, &f->L);
    }
    sp_free(&S);
  }
  free(blk);
  free(iface);
  if (st != OR_OK) { or_free(o); return st; }

  /* Sec. 4.3, c_solver 1: the whole C_a = C + a^2 I for the Chebyshev
   * iteration, and the spectrum estimate of (C_a, D_a) */
  if (c_solver >= 1) {
    long cap = s;
    for (int g = m; g < n; g++) cap += o->Ap.rp[g + 1] - o->Ap.rp[g];
    trip *t = (trip *)malloc(sizeof(trip) * (size_t)cap);
    long nt = 0;
    for (int g = m; g < n; g++) {
      for (int q = o->Ap.rp[g]; q < o->Ap.rp[g + 1]; q++)
        if (o->Ap.ci[q] >= m) { t[nt].r = g - m; t[nt].c = o->Ap.ci[q] - m; t[nt].v = o->Ap.va[q]; nt++; }
      t[nt].r = g - m; t[nt].c = g - m; t[nt].v = alpha * alpha; nt++;
    }
    st = sp_from_trips(&o->Ca, s, t, nt);
    free(t);
    if (st == OR_OK) st = c_solver == 1 ? cheb_estimate(o, (uint64_t)seed) : mr_build(o);
    if (st != OR_OK) { or_free(o); return st; }
  }

  /* low-rank part (Sec. 4.4): Lanczos, or the randomized subspace iteration */
  int mmax = lanczos_max > 0 ? lanczos_max : 5 * k;
  if (mmax > s) mmax = s;
  if (mmax < k) mmax = k;
  int ell = k + rand_oversample;
  if (ell > s) ell = s;
  if (lowrank_method == 1) mmax = ell;
  double *Q = (double *)malloc(sizeof(double) * (size_t)s * (size_t)(mmax + 1));
  double *al = (double *)calloc((size_t)mmax + 1, sizeof(double));
  double *be = (double *)calloc((size_t)mmax + 1, sizeof(double));
  if (!Q || !al || !be) { free(Q); free(al); free(be); or_free(o); return OR_NOMEM; }
  int mm;
  double *Y;
  double *Ub = NULL, *tdb = NULL, *teb = NULL;   /* bidiagonalisation: U_m and B_m */
  if (lowrank_method == 2) {
    Ub = (double *)malloc(sizeof(double) * (size_t)n * (size_t)mmax);
    tdb = (double *)calloc(2 * (size_t)mmax + 2, sizeof(double));
    teb = (double *)calloc(2 * (size_t)mmax + 2, sizeof(double));
    mm = lbd(o, k, mmax, lanczos_check, lanczos_eps, (uint64_t)seed, Q, Ub, tdb, teb);
    o->ritz = (double *)malloc(sizeof(double) * (size_t)mm);
    Y = (double *)malloc(sizeof(double) * (size_t)mm * mm);
    tri_eig(mm, tdb, teb, o->ritz, Y);
  } else if (lowrank_method == 1) {
    mm = ell;
    o->ritz = (double *)malloc(sizeof(double) * (size_t)mm);
    Y = (double *)malloc(sizeof(double) * (size_t)mm * mm);
    rand_subspace(o, ell, rand_power, (uint64_t)seed, Q, o->ritz, Y);
  } else {
    mm = lanczos(o, k, mmax, lanczos_check, lanczos_eps, (uint64_t)seed, Q, al, be);
    o->ritz = (double *)malloc(sizeof(double) * (size_t)mm);
    Y = (double *)malloc(sizeof(double) * (size_t)mm * mm);
    tri_eig(mm, al, be, o->ritz, Y);
  }
  o->msteps = mm;
  /* Ritz vectors: (Q_m Y)_k, s x k row-major */
  double *V = (double *)calloc((size_t)s * k, sizeof(double));
  for (int r = 0; r < s; r++)
    for (int c = 0; c < k; c++) {
      double acc = 0.0;
      for (int j = 0; j < mm; j++) acc += Q[(size_t)j * s + r] * Y[j * mm + c];
      V[(size_t)r * k + c] = acc;
    }
  free(Q); free(al); free(be);
  if (lowrank_method != 2) { free(Y); Y = NULL; }   /* the bidiagonal tail needs Y */

  if (variant == 1) {
    o->urows = s;
    o->U = V;
    o->lam = (double *)malloc(sizeof(double) * (size_t)k);
    for (int c = 0; c < k; c++) o->lam[c] = o->ritz[c];
    o->theta = (theta_mode == 1 && k < mm) ? o->ritz[k] : 0.0;
    if (!indefinite) {
      /* prop. spd-1: M is SPD when theta < 1 and every lambda_i < 1 */
      if (!(o->lam[0] < 1.0) || !(o->theta < 1.0)) { or_free(o); return OR_NOT_SPD; }
    } else {
      /* Ritz values above 1 are kept (A indefinite); G_{k,theta} must only be
       * invertible: 1 - lambda_i and 1 - theta away from zero */
      int sing = !(fabs(1.0 - o->theta) > 1e-12);
      for (int c = 0; c < k; c++) sing |= !(fabs(1.0 - o->lam[c]) > 1e-12);
      if (sing) { or_free(o); return OR_BREAKDOWN; }
    }
  } else {
    /* U_k = A0^-1 E V_k (n x k); K = U_k^T (E V_k); H_k = (I - K)^-1 */
    o->urows = n;
    o->U = (double *)calloc((size_t)n * k, sizeof(double));
    double *EV = (double *)calloc((size_t)n * k, sizeof(double));
    double *vc = (double *)malloc(sizeof(double) * (size_t)s);
    double *ev = (double *)malloc(sizeof(double) * (size_t)n);
    double *uc = (double *)malloc(sizeof(double) * (size_t)n);
    for (int c = 0; c < k; c++) {
      for (int r = 0; r < s; r++) vc[r] = V[(size_t)r * k + c];
      e_mult(o, vc, ev);
      if (lowrank_method == 2) {
        /* U_k = K V_k = U_m (B_m Y_k): no further solves with A0 */
        for (int r = 0; r < n; r++) uc[r] = 0.0;
        for (int i = 0; i < mm; i++) {
          double g = tdb[mmax + 1 + i] * Y[(size_t)i * mm + c];
          if (i + 1 < mm) g += teb[mmax + 1 + i] * Y[(size_t)(i + 1) * mm + c];
          for (int r = 0; r < n; r++) uc[r] += Ub[(size_t)i * n + r] * g;
        }
      } else {
        a0_solve(o, ev, uc);
      }
      for (int r = 0; r < n; r++) { EV[(size_t)r * k + c] = ev[r]; o->U[(size_t)r * k + c] = uc[r]; }
    }
    double *K = (double *)calloc((size_t)k * k, sizeof(double));
    for (int a = 0; a < k; a++)
      for (int b = 0; b < k; b++) {
        double acc = 0.0;
        for (int r = 0; r < n; r++) acc += o->U[(size_t)r * k + a] * EV[(size_t)r * k + b];
        K[a * k + b] = acc;
      }
    /* I - K, symmetrised, Cholesky (failure: not SPD, prop. spd-2), inverse;
     * indefinite: Gauss-Jordan elimination with partial pivoting */
    double *IK = (double *)calloc((size_t)k * k, sizeof(double));
    for (int a = 0; a < k; a++)
      for (int b = 0; b < k; b++)
        IK[a * k + b] = (a == b ? 1.0 : 0.0) - 0.5 * (K[a * k + b] + K[b * k + a]);
    int cst = indefinite ? OR_BREAKDOWN : chol_dense(k, IK);
    if (indefinite) {
      o->Hk = (double *)calloc((size_t)k * k, sizeof(double));
      if (gauss_jordan_inverse(k, IK, o->Hk) == OR_OK) cst = OR_OK;
    } else if (cst == OR_OK) {
      o->Hk = (double *)calloc((size_t)k * k, sizeof(double));
      double *e = (double *)malloc(sizeof(double) * (size_t)k);
      for (int c = 0; c < k; c++) {
        for (int r = 0; r < k; r++) e[r] = (r == c) ? 1.0 : 0.0;
        for (int i = 0; i < k; i++) {
          double sm = e[i];
          for (int t = 0; t < i; t++) sm -= IK[i * k + t] * e[t];
          e[i] = sm / IK[i * k + i];
        }
        for (int i = k - 1; i >= 0; i--) {
          double sm = e[i];
          for (int t = i + 1; t < k; t++) sm -= IK[t * k + i] * e[t];
          e[i] = sm / IK[i * k + i];
        }
        for (int r = 0; r < k; r++) o->Hk[r * k + c] = e[r];
      }
      free(e);
    }
    free(EV); free(vc); free(ev); free(uc); free(K); free(IK); free(V);
    free(Y); free(Ub); free(tdb); free(teb);
    if (cst != OR_OK) { or_free(o); return indefinite ? OR_BREAKDOWN : OR_NOT_SPD; }
  }
  *out = o;
  return OR_OK;
}

void or_free(oracle *o) {
  if (!o) return;
  free(o->perm); free(o->iperm); free(o->boff); free(o->dsc);
  sp_free(&o->A); sp_free(&o->Ap); sp_free(&o->Eh); sp_free(&o->EhT); sp_free(&o->Ca);
  if (o->xrow) for (int j = 0; j < o->s; j++) { free(o->xrow[j]); free(o->xval[j]); }
  free(o->xrow); free(o->xval); free(o->xcnt);
  if (o->bf) {
    for (int b = 0; b <= o->p; b++) {
      free(o->bf[b].ord); free(o->bf[b].D); sp_free(&o->bf[b].L);
    }
    free(o->bf);
  }
  free(o->U); free(o->lam); free(o->Hk); free(o->ritz);
  free(o->work); free(o->work2);
  free(o);
}

void or_destroy(void *h) { or_free((oracle *)h); }

/* M^-1 applied in new order (scaled system) */
static void apply_new(oracle *o, const double *x, double *u) {
  int n = o->n, s = o->s, k = o->k;
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *t = (double *)malloc(sizeof(double) * (size_t)k);
  if (o->variant == 1) {
    /* Algorithm 1 */
    double *y = (double *)malloc(sizeof(double) * (size_t)s);
    double *wv = (double *)malloc(sizeof(double) * (size_t)s);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    a0_solve(o, x, z);                                  /* A0 z = x */
    et_mult(o, z, y);                                   /* y = E^T z */
    double it = 1.0 / (1.0 - o->theta);                 /* w = G_{k,theta}^-1 y */
    for (int c = 0; c < k; c++) {
      double acc = 0.0;
      for (int r = 0; r < s; r++) acc += o->U[(size_t)r * k + c] * y[r];
      t[c] = acc * (1.0 / (1.0 - o->lam[c]) - it);
    }
    for (int r = 0; r < s; r++) {
      double acc = 0.0;
      for (int c = 0; c < k; c++) acc += o->U[(size_t)r * k + c] * t[c];
      wv[r] = it * y[r] + acc;
    }
    e_mult(o, wv, v);                                   /* v = E w */
    for (int i = 0; i < n; i++) v[i] += x[i];
    a0_solve(o, v, u);                                  /* A0 u = x + v */
    free(y); free(wv); free(v);
  } else {
    /* eq. (Form2a): u = A0^-1 x + U_k H_k U_k^T x */
    double *h = (double *)malloc(sizeof(double) * (size_t)k);
    a0_solve(o, x, u);
    for (int c = 0; c < k; c++) {
      double acc = 0.0;
      for (int r = 0; r < n; r++) acc += o->U[(size_t)r * k + c] * x[r];
      t[c] = acc;
    }
    for (int a = 0; a < k; a++) {
      double acc = 0.0;
      for (int b = 0; b < k; b++) acc += o->Hk[a * k + b] * t[b];
      h[a] = acc;
    }
    for (int r = 0; r < n; r++) {
      double acc = 0.0;
      for (int c = 0; c < k; c++) acc += o->U[(size_t)r * k + c] * h[c];
      u[r] += acc;
    }
    free(h);
  }
  free(z); free(t);
}

/* y = M^-1 x in the original ordering; with diagonal scaling
 * M^-1 = D^-1/2 Mhat^-1 D^-1/2 */
int or_apply(void *h, const double *x, double *y) {
  oracle *o = (oracle *)h;
  int n = o->n;
  double *xn = (double *)malloc(sizeof(double) * (size_t)n);
  double *yn = (double *)malloc(sizeof(double) * (size_t)n);
  for (int g = 0; g < n; g++) {
    int i = o->perm[g];
    xn[g] = o->dsc ? x[i] * o->dsc[i] : x[i];
  }
  apply_new(o, xn, yn);
  for (int g = 0; g < n; g++) {
    int i = o->perm[g];
    y[i] = o->dsc ? yn[g] * o->dsc[i] : yn[g];
  }
  free(xn); free(yn);
  return OR_OK;
}

/* z = A0^-1 x in the original ordering (scaled system when scale_diag) */
int or_a0_solve(void *h, const double *x, double *y) {
  oracle *o = (oracle *)h;
  int n = o->n;
  double *xn = (double *)malloc(sizeof(double) * (size_t)n);
  double *yn = (double *)malloc(sizeof(double) * (size_t)n);
  for (int g = 0; g < n; g++) xn[g] = x[o->perm[g]];
  a0_solve(o, xn, yn);
  for (int g = 0; g < n; g++) y[o->perm[g]] = yn[g];
  free(xn); free(yn);
  return OR_OK;
}

/* Preconditioned CG (Hestenes-Stiefel; flexible=1: Polak-Ribiere beta) from
 * x0 = 0.  Converged when ||r|| <= tol ||b||, confirmed on the true residual
 * b - A x; if that check fails, r is replaced by the true residual and CG
 * restarts from the current x.  its = number of x updates. */
int or_pcg(void *h, const double *b, double *x, double tol, int maxit, int flexible,
           int *its_out, double *relres_out) {
  oracle *o = (oracle *)h;
  int n = o->n;
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *zo = (double *)malloc(sizeof(double) * (size_t)n);
  double *p = (double *)malloc(sizeof(double) * (size_t)n);
  double *q = (double *)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
  double bn = sqrt(dot(n, b, b));
  int its = 0, st = OR_NOCONV;
  double rel = 0.0;
  if (bn == 0.0) { st = OR_OK; goto done; }
  or_apply(o, r, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = dot(n, r, z);
  while (its < maxit) {
    sp_mv(&o->A, p, q);
    double a = rz / dot(n, p, q);
    for (int i = 0; i < n; i++) { x[i] += a * p[i]; r[i] -= a * q[i]; }
    its++;
    if (sqrt(dot(n, r, r)) <= tol * bn) {
      sp_mv(&o->A, x, q);
      for (int i = 0; i < n; i++) q[i] = b[i] - q[i];
      if (sqrt(dot(n, q, q)) <= tol * bn) { st = OR_OK; break; }
      memcpy(r, q, sizeof(double) * (size_t)n);
      or_apply(o, r, z);
      memcpy(p, z, sizeof(double) * (size_t)n);
      rz = dot(n, r, z);
      continue;
    }
    memcpy(zo, z, sizeof(double) * (size_t)n);
    or_apply(o, r, z);
    double rzn = dot(n, r, z), beta;
    if (flexible) {
      double t = 0.0;
      for (int i = 0; i < n; i++) t += r[i] * (z[i] - zo[i]);
      beta = t / rz;
    } else {
      beta = rzn / rz;
    }
    rz = rzn;
    for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
  }
done:
  sp_mv(&o->A, x, q);
  for (int i = 0; i < n; i++) q[i] = b[i] - q[i];
  rel = bn > 0 ? sqrt(dot(n, q, q)) / bn : 0.0;
  *its_out = its;
  *relres_out = rel;
  free(r); free(z); free(zo); free(p); free(q);
  return st;
}

/* Restarted GMRES(m) (Saad and Schultz), right-preconditioned: the Krylov
 * space is that of A M^-1 from r0, and x = x0 + M^-1 V_j y.  Used in Sec. 5
 * for the indefinite problems with m = 40.  From x0 = 0; each cycle runs
 * Arnoldi with two classical Gram-Schmidt passes (the Hessenberg entry is
 * the sum of both passes' coefficients), keeps the least-squares problem
 * triangular with Givens rotations, so |g_{j+1}| is the residual norm of the
 * current iterate, and ends when that norm is <= tol ||b||, after m steps,
 * at maxit steps in total, or when the new Arnoldi vector is zero.  Then
 * y = R^-1 g, x += M^-1 (V y), and the true residual b - A x both decides
 * convergence and starts the next cycle.  its = Arnoldi steps. */
int or_gmres(void *h, const double *b, double *x, double tol, int maxit, int restart,
             int *its_out, double *relres_out) {
  oracle *o = (oracle *)h;
  int n = o->n, m = restart;
  if (m < 1 || maxit < 0) return OR_INVALID;
  double *V = (double *)malloc(sizeof(double) * (size_t)n * (m + 1));
  double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));   /* H[i + j (m+1)] */
  double *cs = (double *)malloc(sizeof(double) * (size_t)m);
  double *sn = (double *)malloc(sizeof(double) * (size_t)m);
  double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  double *y = (double *)malloc(sizeof(double) * (size_t)m);
  double *c = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
  double bn = sqrt(dot(n, b, b)), beta = bn;
  int its = 0, st = OR_NOCONV;
  while (1) {
    if (beta <= tol * bn) { st = OR_OK; break; }
    if (!(beta == beta)) { st = OR_BREAKDOWN; break; }
    if (its >= maxit) break;
    for (int i = 0; i < n; i++) V[i] = r[i] / beta;
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
    int j = 0;
    while (j < m && its < maxit) {
      double *hj = H + (size_t)j * (m + 1);
      or_apply(o, V + (size_t)j * n, z);          /* w = A M^-1 v_j */
      sp_mv(&o->A, z, w);
      for (int i = 0; i <= j; i++) hj[i] = 0.0;
      for (int pass = 0; pass < 2; pass++) {
        for (int i = 0; i <= j; i++) c[i] = dot(n, V + (size_t)i * n, w);
        for (int i = 0; i <= j; i++) {
          for (int q = 0; q < n; q++) w[q] -= c[i] * V[(size_t)i * n + q];
          hj[i] += c[i];
        }
      }
      double hn = sqrt(dot(n, w, w));
      hj[j + 1] = hn;
      if (hn > 0.0)
        for (int q = 0; q < n; q++) V[(size_t)(j + 1) * n + q] = w[q] / hn;
      for (int i = 0; i < j; i++) {              /* earlier rotations */
        double t = cs[i] * hj[i] + sn[i] * hj[i + 1];
        hj[i + 1] = -sn[i] * hj[i] + cs[i] * hj[i + 1];
        hj[i] = t;
      }
      double d = hypot(hj[j], hj[j + 1]);        /* the rotation that zeroes h_{j+1,j} */
      cs[j] = d > 0.0 ? hj[j] / d : 1.0;
      sn[j] = d > 0.0 ? hj[j + 1] / d : 0.0;
      hj[j] = d;
      hj[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      its++;
      j++;
      if (fabs(g[j]) <= tol * bn || !(hn > 0.0)) break;
    }
    for (int i = j - 1; i >= 0; i--) {           /* R y = g */
      double t = g[i];
      for (int l = i + 1; l < j; l++) t -= H[i + (size_t)l * (m + 1)] * y[l];
      y[i] = t / H[i + (size_t)i * (m + 1)];
    }
    for (int q = 0; q < n; q++) {
      double t = 0.0;
      for (int l = 0; l < j; l++) t += V[(size_t)l * n + q] * y[l];
      w[q] = t;
    }
    or_apply(o, w, z);
    for (int q = 0; q < n; q++) x[q] += z[q];
    sp_mv(&o->A, x, w);
    for (int q = 0; q < n; q++) r[q] = b[q] - w[q];
    beta = sqrt(dot(n, r, r));
  }
  *its_out = its;
  *relres_out = bn > 0 ? beta / bn : 0.0;
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(c); free(r); free(z); free(w);
  return st;
}

/* sizes and scalars: out[0..8] = n, p, s, m, k, msteps, ncolors, variant, urows */
void or_info(void *h, int *out, double *theta) {
  oracle *o = (oracle *)h;
  out[0] = o->n; out[1] = o->p; out[2] = o->s; out[3] = o->m; out[4] = o->k;
  out[5] = o->msteps; out[6] = o->ncolors; out[7] = o->variant; out[8] = o->urows;
  *theta = o->theta;
}

/* Gram-Schmidt passes taken by the Lanczos steps of the setup */
long or_reorth_passes(void *h) { return ((oracle *)h)->reorth_passes; }

void or_ritz(void *h, double *out) {
  oracle *o = (oracle *)h;
  memcpy(out, o->ritz, sizeof(double) * (size_t)o->msteps);
}

void or_perm(void *h, int *perm) {
  oracle *o = (oracle *)h;
  memcpy(perm, o->perm, sizeof(int) * (size_t)o->n);
}

/* low-rank data: U (urows x k, rows in new order), lam (k), Hk (k x k) */
void or_lowrank(void *h, double *U, double *lam, double *Hk) {
  oracle *o = (oracle *)h;
  memcpy(U, o->U, sizeof(double) * (size_t)o->urows * o->k);
  if (lam && o->lam) memcpy(lam, o->lam, sizeof(double) * (size_t)o->k);
  if (Hk && o->Hk) memcpy(Hk, o->Hk, sizeof(double) * (size_t)o->k * o->k);
}

/* number of stored factor entries (lower incl. diagonal) over all blocks */
long or_factor_nnz(void *h) {
  oracle *o = (oracle *)h;
  long t = 0;
  for (int b = 0; b <= o->p; b++) {
    blockfac *f = &o->bf[b];
    if (f->exact) {
      for (long i = 0; i < (long)f->nb * f->nb; i++) if (f->D[i] != 0.0) t++;
    } else {
      t += f->L.rp[f->nb];
    }
  }
  return t;
}

/* factor entries as (row, col, value) with ORIGINAL indices: entry L(e_i, e_j)
 * of a block's factor in its elimination order is reported at the original
 * indices of the rows eliminated at e_i and e_j. */
void or_factor_coo(void *h, int *ri, int *cj, double *v) {
  oracle *o = (oracle *)h;
  long w = 0;
  for (int b = 0; b <= o->p; b++) {
    blockfac *f = &o->bf[b];
    int off = o->boff[b];
    for (int i = 0; i < f->nb; i++) {
      if (f->exact) {
        for (int j = 0; j <= i; j++) {
          double d = f->D[(size_t)i * f->nb + j];
          if (d == 0.0) continue;
          ri[w] = o->perm[off + f->ord[i]]; cj[w] = o->perm[off + f->ord[j]]; v[w] = d; w++;
        }
      } else {
        for (int q = f->L.rp[i]; q < f->L.rp[i + 1]; q++) {
          ri[w] = o->perm[off + f->ord[i]];
          cj[w] = o->perm[off + f->ord[f->L.ci[q]]];
          v[w] = f->L.va[q]; w++;
        }
      }
    }
  }
}

/* SplitMix64 value in [-1, 1): exposed so the tests can pin the generator */
double or_sm64_pm1(unsigned long long seed, unsigned long long i) {
  return sm64_pm1((uint64_t)seed, (uint64_t)i);
}

/* Chebyshev data (c_solver 1): out = {lo, hi} of the spectrum interval used */
void or_cheb_bounds(void *h, double *out) {
  oracle *o = (oracle *)h;
  out[0] = o->cheb_lo; out[1] = o->cheb_hi;
}

/* replace the interval (tests: closed-form Chebyshev polynomials); the low-
 * rank data of the setup are kept */
void or_set_cheb_bounds(void *h, double lo, double hi) {
  oracle *o = (oracle *)h;
  o->cheb_lo = lo; o->cheb_hi = hi;
}
