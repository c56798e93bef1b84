// ddlr_rand.cuh -- randomized subspace iteration for the low-rank part
// (lowrank_method 1): the randomized technique the paper's conclusion names
// as a faster alternative to Lanczos (method of Halko, Martinsson, Tropp).
//
// With Op = E^T A0^-1 E (DDLR-1) or E^T A0^-2 E (DDLR-2) and ell = k + p:
//   Omega (s x ell): column c = SplitMix64 stream seed + 2^33 + c over the
//   interface nodes in ascending original index;
//   Q = orth(Op Omega); q times Q = orth(Op Q); B = Q^T Op Q (symmetrised);
//   B = Y diag(theta) Y^T, theta descending; U_k = Q Y_k (DDLR-1) or
//   V_k = Q Y_k (DDLR-2).
// orth is Cholesky QR applied twice (the QR factor with positive diagonal R,
// as the Gram-Schmidt of the oracle gives).  Op on a block uses the batched
// A0 solve; blocks are s x ell (or n x ell) row-major, ell <= 64.  B is
// reduced to tridiagonal form by Householder reflections in one CTA, its
// eigenpairs come from the tridiagonal eigensolver of the Lanczos path, and
// the reflections are applied back to the eigenvectors.
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

constexpr int kRandMaxL = 64;

// Omega: Y[r * L + c] = SplitMix64(seed + 2^33 + c)[rank[r]]
__global__ void k_rand_omega(int s, int L, const int *rank, unsigned long long seed, double *Y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)s * L) return;
  const int r = int(unsigned(e) / unsigned(L)), c = int(e - (long long)r * L);
  Y[e] = d_sm64_pm1(seed + 0x200000000ULL + (unsigned long long)c, (unsigned long long)rank[r]);
}

// V = E W = [a^-1 Ehat W ; -a W] for a block of L columns (W s x L, V n x L)
__global__ void k_e_block(int m, int s, int L, const int *eh_rp, const int *eh_ci, const double *eh, double ia,
                          double a, const double *W, double *V) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)(m + s) * L) return;
  const int r = int(unsigned(e) / unsigned(L)), c = int(e - (long long)r * L);
  double v;
  if (r < m) {
    double acc = 0;
    for (int q = eh_rp[r]; q < eh_rp[r + 1]; q++) acc += eh[q] * W[(long long)eh_ci[q] * L + c];
    v = ia * acc;
  } else {
    v = -a * W[(long long)(r - m) * L + c];
  }
  V[e] = v;
}

// partials[blk][a * L + b] = sum over this CTA's rows of X[r][a] Y[r][b]
// (rows in order; 32-row tiles staged in shared memory).  256 threads.
constexpr int kGramNT = 256, kGramTile = 32;
__global__ void __launch_bounds__(kGramNT)
k_gram_partial(long long s, int L, const double *X, const double *Y, double *partials) {
  __shared__ double xs[kGramTile * kRandMaxL], ys[kGramTile * kRandMaxL];
  constexpr int PER = kRandMaxL * kRandMaxL / kGramNT;   // pairs per thread (16)
  const int np = L * L;
  const long long chunk = (s + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * chunk, r1 = min(s, r0 + chunk);
  double acc[PER];
#pragma unroll
  for (int u = 0; u < PER; u++) acc[u] = 0.0;
  for (long long base = r0; base < r1; base += kGramTile) {
    const int nt = int(min((long long)kGramTile, r1 - base));
    __syncthreads();
    for (int t = threadIdx.x; t < nt * L; t += kGramNT) {
      xs[t] = X[base * L + t];
      ys[t] = Y[base * L + t];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; u++) {
      const int o = threadIdx.x + u * kGramNT;
      if (o < np) {
        const int a = o / L, b = o - a * L;
        double v = acc[u];
        for (int rr = 0; rr < nt; rr++) v += xs[rr * L + a] * ys[rr * L + b];
        acc[u] = v;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PER; u++) {
    const int o = threadIdx.x + u * kGramNT;
    if (o < np) partials[(long long)blockIdx.x * np + o] = acc[u];
  }
}

// out[o] = sum_g partials[g][o] in order (o < L*L)
__global__ void k_gram_reduce(int G, int np, const double *partials, double *out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= np) return;
  double v = 0;
  for (int g = 0; g < G; g++) v += partials[(long long)g * np + o];
  out[o] = v;
}

// Cholesky G = L L^T (G symmetrised first) and Linv = L^-1, one CTA of
// kRandMaxL threads; a pivot <= 0 or not finite sets *flag
__global__ void k_chol_inv(int L, const double *G, double *Linv, int *flag) {
  __shared__ double A[kRandMaxL * kRandMaxL];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int o = t; o < L * L; o += blockDim.x) {
    const int i = o / L, j = o - i * L;
    A[o] = 0.5 * (G[i * L + j] + G[j * L + i]);
  }
  __syncthreads();
  for (int j = 0; j < L; j++) {
    if (t == 0) {
      const double d = A[j * L + j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      A[j * L + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dj = A[j * L + j];
    for (int i = j + 1 + t; i < L; i += blockDim.x) A[i * L + j] /= dj;
    __syncthreads();
    for (int i = j + 1 + t; i < L; i += blockDim.x)
      for (int q = j + 1; q <= i; q++) A[i * L + q] -= A[i * L + j] * A[q * L + j];
    __syncthreads();
  }
  // column c of L^-1 (lower triangular), one thread per column
  for (int c = t; c < L; c += blockDim.x) {
    for (int i = 0; i < c; i++) Linv[i * L + c] = 0.0;
    Linv[c * L + c] = 1.0 / A[c * L + c];
    for (int i = c + 1; i < L; i++) {
      double acc = 0;
      for (int q = c; q < i; q++) acc += A[i * L + q] * Linv[q * L + c];
      Linv[i * L + c] = -acc / A[i * L + i];
    }
  }
  if (t == 0 && bad) *flag = 1;
}

// Q = Y L^-T row by row: Q[r][c] = sum_{j <= c} Y[r][j] Linv[c][j]
__global__ void k_apply_rinv(long long s, int L, const double *Y, const double *Linv, double *Q) {
  __shared__ double Li[kRandMaxL * kRandMaxL];
  for (int o = threadIdx.x; o < L * L; o += blockDim.x) Li[o] = Linv[o];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const double *y = Y + r * L;
  for (int c = 0; c < L; c++) {
    double acc = 0;
    for (int j = 0; j <= c; j++) acc += y[j] * Li[c * L + j];
    Q[r * L + c] = acc;
  }
}

// Householder tridiagonalisation of the symmetrised B (L x L), one CTA of
// kRandMaxL threads: d (diagonal), e (off-diagonal, e[i] couples i, i+1) and
// the unit reflection vectors Hv[j][*] (zero where the reflection is I)
__global__ void k_sym_tridiag(int L, const double *B, double *d, double *e, double *Hv) {
  __shared__ double A[kRandMaxL * kRandMaxL];
  __shared__ double v[kRandMaxL], p[kRandMaxL], w[kRandMaxL];
  __shared__ double sc[2];
  const int t = threadIdx.x;
  for (int o = t; o < L * L; o += blockDim.x) {
    const int i = o / L, j = o - i * L;
    A[o] = 0.5 * (B[i * L + j] + B[j * L + i]);
  }
  for (int o = t; o < L * L; o += blockDim.x) Hv[o] = 0.0;
  __syncthreads();
  for (int j = 0; j + 2 < L; j++) {
    // x = A[j+1.., j]; v = x - alpha e_1, alpha = -sign(x_0) ||x||
    if (t == 0) {
      double nx = 0;
      for (int i = j + 1; i < L; i++) nx += A[i * L + j] * A[i * L + j];
      nx = sqrt(nx);
      const double x0 = A[(j + 1) * L + j];
      const double alpha = x0 >= 0.0 ? -nx : nx;
      sc[0] = alpha;
      double nv = 0;
      for (int i = j + 1; i < L; i++) {
        const double vi = (i == j + 1) ? x0 - alpha : A[i * L + j];
        v[i] = vi;
        nv += vi * vi;
      }
      sc[1] = nv > 0.0 ? 1.0 / sqrt(nv) : 0.0;
    }
    __syncthreads();
    const double alpha = sc[0], inv = sc[1];
    if (inv == 0.0) continue;      // already tridiagonal in this column
    for (int i = j + 1 + t; i < L; i += blockDim.x) {
      v[i] *= inv;
      Hv[j * L + i] = v[i];
    }
    __syncthreads();
    // p = A_sub v (rows j+1..L-1)
    for (int i = j + 1 + t; i < L; i += blockDim.x) {
      double acc = 0;
      for (int q = j + 1; q < L; q++) acc += A[i * L + q] * v[q];
      p[i] = acc;
    }
    __syncthreads();
    if (t == 0) {
      double K = 0;
      for (int i = j + 1; i < L; i++) K += v[i] * p[i];
      sc[1] = K;
    }
    __syncthreads();
    const double K = sc[1];
    for (int i = j + 1 + t; i < L; i += blockDim.x) w[i] = 2.0 * (p[i] - K * v[i]);
    __syncthreads();
    // A_sub -= v w^T + w v^T; column j below the diagonal becomes alpha e_1
    for (int i = j + 1 + t; i < L; i += blockDim.x) {
      for (int q = j + 1; q < L; q++) A[i * L + q] -= v[i] * w[q] + w[i] * v[q];
      const double nval = (i == j + 1) ? alpha : 0.0;
      A[i * L + j] = nval;
      A[j * L + i] = nval;
    }
    __syncthreads();
  }
  for (int i = t; i < L; i += blockDim.x) {
    d[i] = A[i * L + i];
    e[i] = (i + 1 < L) ? A[(i + 1) * L + i] : 0.0;
  }
}

// eigenvectors of B from those of the tridiagonal form: Y (L x k column-
// major) <- P_0 P_1 ... P_{L-3} Y, one thread per vector
__global__ void k_back_transform(int L, int k, const double *Hv, double *Y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double *y = Y + (long long)c * L;
  for (int j = L - 3; j >= 0; j--) {
    const double *v = Hv + (long long)j * L;
    double dot = 0;
    for (int i = j + 1; i < L; i++) dot += v[i] * y[i];
    if (dot == 0.0) continue;
    for (int i = j + 1; i < L; i++) y[i] -= 2.0 * dot * v[i];
  }
}

// out (s x k row-major) = Q (s x L row-major) Y (L x k column-major)
__global__ void k_rm_gemm(long long s, int L, int k, const double *Q, const double *Y, double *out) {
  __shared__ double Ys[kRandMaxL * kRandMaxL];
  for (int o = threadIdx.x; o < L * k; o += blockDim.x) Ys[o] = Y[o];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const double *q = Q + r * L;
  for (int c = 0; c < k; c++) {
    double acc = 0;
    for (int j = 0; j < L; j++) acc += q[j] * Ys[c * L + j];
    out[r * k + c] = acc;
  }
}

}  // namespace ddlr
