// ddlr_gmres.cuh -- restarted GMRES(m), right-preconditioned (Sec. 5: the
// accelerator for the indefinite problems, GMRES(40)), and the inverse of an
// indefinite I - K for DDLR-2 in the indefinite mode.
//
// One Arnoldi step on A M^-1: z_j = M^-1 v_j (kept, so x += Z y needs no
// further apply), w = A z_j, two classical Gram-Schmidt passes against
// v_0..v_j (the Hessenberg column is the sum of both passes' coefficients:
// the generic CGS kernels of ddlr_lbd.cuh with k_gm_reduce_acc),
// h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}, then one Givens step.  H is
// column-major with leading dimension m + 1; all scalars stay on the device.
#pragma once
#include "ddlr_lbd.cuh"

namespace ddlr {

// c[col] = sum_g partials[g][col] (a warp per column, fixed order), and the
// Hessenberg column hcol[col] = c[col] (first pass) or += c[col]
__global__ void k_gm_reduce_acc(int G, int ncol, const double *partials, double *c, double *hcol, int first) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
  if (w >= ncol) return;
  double s = 0;
  for (int g = l; g < G; g += 32) s += partials[(long long)g * ncol + w];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) {
    c[w] = s;
    hcol[w] = first ? s : hcol[w] + s;
  }
}

// sqrt of the sum of G dot partials into *o1 and *o2 (a NaN stays a NaN)
__global__ void k_gm_norm(int G, const double *partials, double *o1, double *o2) {
  const double v = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    const double r = v >= 0.0 ? sqrt(v) : v;
    *o1 = r;
    *o2 = r;
  }
}

// g = (beta, 0, ..., 0), m + 1 entries
__global__ void k_gm_ginit(int m, const double *beta, double *g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= m) g[i] = i == 0 ? *beta : 0.0;
}

// Givens step j (one thread): the rotations 0..j-1 applied to column j of H,
// then the rotation that zeroes h_{j+1,j}; g updated; *res = |g_{j+1}|, the
// residual norm of the current iterate
__global__ void k_gm_givens(int j, double *hcol, double *cs, double *sn, double *g, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < j; i++) {
    const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
    hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
    hcol[i] = t;
  }
  const double d = hypot(hcol[j], hcol[j + 1]);
  cs[j] = d > 0.0 ? hcol[j] / d : 1.0;
  sn[j] = d > 0.0 ? hcol[j + 1] / d : 0.0;
  hcol[j] = d;
  hcol[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  *res = fabs(g[j + 1]);
}

// R y = g, R the leading j x j upper triangle of H (one thread)
__global__ void k_gm_backsolve(int j, const double *H, int ld, const double *g, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = j - 1; i >= 0; i--) {
    double t = g[i];
    for (int l = i + 1; l < j; l++) t -= H[i + (long long)l * ld] * y[l];
    y[i] = t / H[i + (long long)i * ld];
  }
}

// x += Z y (Z n x j column-major), a thread per row, y in shared memory
__global__ void k_gm_update(long long n, int j, const double *Z, const double *y, double *x) {
  extern __shared__ double ys[];
  for (int l = threadIdx.x; l < j; l += blockDim.x) ys[l] = y[l];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double t = 0;
  for (int l = 0; l < j; l++) t += Z[(long long)l * n + r] * ys[l];
  x[r] += t;
}

// r = b - q
__global__ void k_gm_resid(long long n, const double *b, const double *q, double *r) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - q[i];
}

// Indefinite mode, DDLR-2: H_k = (I - K)^-1 with K from the k_utv_partial
// partials, symmetrised as for the Cholesky path, inverted by Gauss-Jordan
// elimination with partial pivoting (one thread; work = k x k).  A pivot of
// magnitude <= 1e-14 times the largest entry sets *singular.  Hk row-major.
__global__ void k_hk_finalize_gj(int G, int k, const double *partials, double *work, double *Hk, int *singular) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *M = work;
  double amax = 0.0;
  for (int a = 0; a < k; a++)
    for (int b = 0; b < k; b++) {
      double s1 = 0, s2 = 0;
      for (int g = 0; g < G; g++) {
        s1 += partials[(long long)g * k * k + a * k + b];
        s2 += partials[(long long)g * k * k + b * k + a];
      }
      M[a * k + b] = (a == b ? 1.0 : 0.0) - 0.5 * (s1 + s2);
      amax = fmax(amax, fabs(M[a * k + b]));
      Hk[a * k + b] = a == b ? 1.0 : 0.0;
    }
  for (int j = 0; j < k; j++) {
    int piv = j;
    for (int r = j + 1; r < k; r++)
      if (fabs(M[r * k + j]) > fabs(M[piv * k + j])) piv = r;
    if (!(fabs(M[piv * k + j]) > 1e-14 * amax)) { *singular = 1; return; }
    if (piv != j)
      for (int c = 0; c < k; c++) {
        double t = M[j * k + c]; M[j * k + c] = M[piv * k + c]; M[piv * k + c] = t;
        t = Hk[j * k + c]; Hk[j * k + c] = Hk[piv * k + c]; Hk[piv * k + c] = t;
      }
    const double d = M[j * k + j];
    for (int c = 0; c < k; c++) { M[j * k + c] /= d; Hk[j * k + c] /= d; }
    for (int r = 0; r < k; r++) {
      if (r == j) continue;
      const double f = M[r * k + j];
      if (f == 0.0) continue;
      for (int c = 0; c < k; c++) { M[r * k + c] -= f * M[j * k + c]; Hk[r * k + c] -= f * Hk[j * k + c]; }
    }
  }
}

}  // namespace ddlr
