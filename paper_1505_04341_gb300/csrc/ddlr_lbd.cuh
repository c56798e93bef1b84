// ddlr_lbd.cuh -- Lanczos (Golub-Kahan) bidiagonalisation of K = A0^-1 E
// for DDLR-2 (lowrank_method 2; Sec. 4.4 names it as the way to compute U_k
// and V_k at the same time):
//   u = K v_j - beta_{j-1} u_{j-1},  alpha_j = ||u||,  u_j = u / alpha_j;
//   v = K^T u_j - alpha_j v_j,       beta_j = ||v||,   v_{j+1} = v / beta_j;
// both bases fully reorthogonalised (two classical Gram-Schmidt passes).
// K V_m = U_m B_m, B_m upper bidiagonal; B_m^T B_m is the tridiagonal matrix
// of Lanczos on K^T K = E^T A0^-2 E, whose eigenpairs (theta, Y) give
// V_k = V_m Y_k and U_k = K V_k = U_m (B_m Y_k) with no further A0 solves.
// Bases are column-major (ld = rows); scalars stay on the device.
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

// partials[blk * ncol + c] = sum over this CTA's rows of Q[c][r] w[r], a warp
// per column (fixed order: lanes stride the rows, then a shuffle tree)
template <int NT>
__global__ void __launch_bounds__(NT)
k_cgs_partial(long long nrows, int ncol, const double *Q, long long ld, const double *w, double *partials) {
  const int nw = NT / 32, wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  const long long chunk = (nrows + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
  for (int c = wi; c < ncol; c += nw) {
    const double *q = Q + (long long)c * ld;
    double acc = 0;
    for (long long r = r0 + l; r < r1; r += 32) acc += q[r] * w[r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (l == 0) partials[(long long)blockIdx.x * ncol + c] = acc;
  }
}

// c[col] = sum_g partials[g][col], a warp per column
__global__ void k_cgs_reduce(int G, int ncol, const double *partials, double *c) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
  if (w >= ncol) return;
  double s = 0;
  for (int g = l; g < G; g += 32) s += partials[(long long)g * ncol + w];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) c[w] = s;
}

// w -= Q c (Q rows x ncol column-major, c in shared memory)
__global__ void k_cgs_sub(long long nrows, int ncol, const double *Q, long long ld, const double *c, double *w) {
  extern __shared__ double cs[];
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) cs[j] = c[j];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  double acc = 0;
  for (int j = 0; j < ncol; j++) acc += Q[(long long)j * ld + r] * cs[j];
  w[r] -= acc;
}

// y -= (*coef) x
__global__ void k_lbd_axpy(long long n, const double *coef, const double *x, double *y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] -= *coef * x[i];
}

// out = x * (1 / *nrm)
__global__ void k_lbd_scale(long long n, const double *x, const double *nrm, double *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] * (1.0 / *nrm);
}

// B_m^T B_m for the first m steps: td[i] = alpha_i^2 + beta_{i-1}^2,
// te[i] = alpha_i beta_i
__global__ void k_lbd_tri(int m, const double *al, const double *be, double *td, double *te) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  td[i] = al[i] * al[i] + (i > 0 ? be[i - 1] * be[i - 1] : 0.0);
  te[i] = al[i] * be[i];
}

// G = B_m Y (m x k, column-major): G[i][c] = alpha_i Y[i][c] + beta_i Y[i+1][c]
__global__ void k_lbd_bmy(int m, int k, const double *al, const double *be, const double *Y, double *G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int c = e / m, i = e - c * m;
  double g = al[i] * Y[(long long)c * m + i];
  if (i + 1 < m) g += be[i] * Y[(long long)c * m + i + 1];
  G[e] = g;
}

}  // namespace ddlr
