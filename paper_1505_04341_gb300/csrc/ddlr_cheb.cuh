// ddlr_cheb.cuh -- the solve with C_a by preconditioned Chebyshev iterations
// (Sec. 4.3), for c_solver 1.
//
// D_a is the block Jacobi matrix of C_a: its couplings between interface nodes
// of one subdomain.  It is factored in place of C_a as block p of A0, so the
// level sweeps of A0 solve with D_a on the interface rows for free; what
// follows here turns that D_a^-1 x_C into t Chebyshev steps for C_a x = x_C
// from x_0 = 0 on the interval [lo, hi] of the spectrum of D_a^-1 C_a:
//   centre c = (hi + lo)/2, half-width d = (hi - lo)/2,
//   rho_0 = d/c,  rho_j = d / (2c - d rho_{j-1}),
//   s_0 = (1/c) D^-1 y,   x_1 = s_0,
//   r_j = r_{j-1} - C_a s_{j-1},   (r_0 = y)
//   s_j = rho_j rho_{j-1} s_{j-1} + 2/(2c - d rho_{j-1}) D^-1 r_j,
//   x_{j+1} = x_j + s_j,
// the three-term recurrence of the Chebyshev polynomials T_j, written with d
// only in numerators (d = 0 gives Richardson steps 1/c).  The coefficients
// depend on the interval only and sit in a device table, so a captured CUDA
// graph follows a change of interval:
//   tab[0] = lo, tab[1] = hi, tab[2] = 1/c,
//   tab[2 + j] = rho_j rho_{j-1},  tab[1 + t + j] = 2/(2c - d rho_{j-1}),
//   j = 1..t-1.
//
// One launch per step does the vector update of step j and the product with
// C_a that step j+1 needs: s_j at a neighbour column is formed where it is
// read from s_{j-1} and D^-1 r_j (same operands, same order, so the same
// bits as the stored value), and s_j is written to the other buffer of a
// pair.  Vectors are n x R row-major (R = 1 for one right-hand side); the
// interface rows are m..n-1 and C_a's columns are interface indices.
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

constexpr int kChebMaxSteps = 64;

__device__ __forceinline__ void cheb_table(double lo, double hi, int t, double *tab, float *tab32) {
  const double c = 0.5 * (hi + lo), d = 0.5 * (hi - lo);
  tab[0] = lo;
  tab[1] = hi;
  tab[2] = 1.0 / c;
  double rho = d / c;
  for (int j = 1; j < t; j++) {
    const double den = 2.0 * c - d * rho;
    const double rn = d / den;
    tab[2 + j] = rn * rho;
    tab[1 + t + j] = 2.0 / den;
    rho = rn;
  }
  if (tab32)
    for (int i = 0; i < 2 * t + 1; i++) tab32[i] = float(tab[i]);
}

// coefficients from a given interval
__global__ void k_cheb_coef(double lo, double hi, int t, double *tab, float *tab32) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cheb_table(lo, hi, t, tab, tab32);
}

// interval from the Lanczos estimate: Ritz values vals (descending, m of them)
// with unit eigenvectors Y (column-major m x m) of T_m; each end is widened by
// beta_m |e_m^T y| (the residual norm of its Ritz pair); a lower end taken to
// zero or below falls back to the smallest Ritz value
__global__ void k_cheb_bounds(int m, const double *vals, const double *Y, const double *be, int t,
                              double *tab, float *tab32) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bm = be[m - 1];
  const double hi = vals[0] + bm * fabs(Y[m - 1]);
  double lo = vals[m - 1] - bm * fabs(Y[(size_t)(m - 1) * m + (m - 1)]);
  if (!(lo > 0.0)) lo = vals[m - 1];
  cheb_table(lo, hi, t, tab, tab32);
}

// a^2 on the diagonal of C_a
__global__ void k_cc_add_diag(int s, const int *diag, double a2, double *val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) val[diag[i]] += a2;
}

// start vector of the estimate: SplitMix64 stream seed + 2^32, drawn in the
// order of rank[] (ascending original index of the interface nodes)
__global__ void k_cheb_start(int s, int m, const int *rank, unsigned long long seed, double *r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) r[m + i] = d_sm64_pm1(seed + 0x100000000ULL, (unsigned long long)rank[i]);
}

// q = z / beta, pv = r / beta (interface rows)
__global__ void k_cheb_lz_qp(int s, int m, const double *beta, const double *z, const double *r, double *q,
                             double *pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s) return;
  const double b = *beta;
  q[m + i] = z[m + i] / b;
  pv[m + i] = r[m + i] / b;
}

// w = C_a q - beta_prev pp   (beta_prev == nullptr: first step)
__global__ void k_cheb_lz_w(int s, int m, const int *rp, const int *ci, const double *val, const double *q,
                            const double *pp, const double *beta_prev, double *w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s) return;
  double acc = 0;
  for (int e = rp[i]; e < rp[i + 1]; e++) acc += val[e] * q[m + ci[e]];
  if (beta_prev) acc -= *beta_prev * pp[m + i];
  w[m + i] = acc;
}

// w -= alpha pv
__global__ void k_cheb_lz_sub(int s, int m, const double *alpha, const double *pv, double *w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s) w[m + i] -= *alpha * pv[m + i];
}

// *out = sqrt(max(sum of partials, 0)) (fixed order)
__global__ void k_cheb_reduce_norm(int G, const double *partials, double *out) {
  const double v = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) *out = v > 0.0 ? sqrt(v) : 0.0;
}

// first step.  z holds D^-1 y on the interface rows on entry; t == 1 scales
// it in place (x_1 = s_0), else s_0 -> d, x_1 -> xacc, r_1 = y - C_a s_0.
template <typename T>
__global__ void k_cheb_first(int s, int m, int R, const int *rp, const int *ci, const T *cv, const T *tab, int t,
                             const T *y, T *z, T *d, T *xacc, T *r, const int *gate) {
  if (gate && *gate) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)s * R) return;
  const int i = R == 1 ? int(e) : int(unsigned(e) / unsigned(R)), col = int(e - (long long)i * R);
  const long long g = (long long)(m + i) * R + col;
  const T c0 = tab[2];
  const T di = c0 * z[g];
  if (t == 1) { z[g] = di; return; }
  T acc = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) acc += cv[q] * (c0 * z[(long long)(m + ci[q]) * R + col]);
  d[g] = di;
  xacc[g] = di;
  r[g] = y[g] - acc;
}

// step j = 1..t-1: zt = D^-1 r_j; s_j from s_{j-1} (dold) and zt; the last
// step writes x_t into z, the others accumulate x, write s_j to dnew and form
// r_{j+1} = r_j - C_a s_j
template <typename T>
__global__ void k_cheb_step(int s, int m, int R, const int *rp, const int *ci, const T *cv, const T *tab, int t,
                            int j, const T *zt, const T *dold, T *dnew, T *xacc, T *r, T *z, const int *gate) {
  if (gate && *gate) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)s * R) return;
  const int i = R == 1 ? int(e) : int(unsigned(e) / unsigned(R)), col = int(e - (long long)i * R);
  const long long g = (long long)(m + i) * R + col;
  const T c1 = tab[2 + j], c2 = tab[1 + t + j];
  const T dn = c1 * dold[g] + c2 * zt[g];
  if (j == t - 1) { z[g] = xacc[g] + dn; return; }
  T acc = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    const long long h = (long long)(m + ci[q]) * R + col;
    acc += cv[q] * (c1 * dold[h] + c2 * zt[h]);
  }
  dnew[g] = dn;
  xacc[g] += dn;
  r[g] -= acc;
}

}  // namespace ddlr
