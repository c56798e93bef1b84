// ddlr_batch.cuh -- kernels of the batched (multi right-hand side) path.
//
// A block of R vectors is stored row-major in device order: X[r*R + q] is
// row r of right-hand side q, so the R values of one row are contiguous and a
// warp reads a row of 32 right-hand sides in one 128/256-byte transaction.
// Every per-column quantity is computed with the same arithmetic whatever R is
// and whichever other columns share the block: row-local work is identical,
// and every reduction splits the rows into the same kRedGrid contiguous ranges,
// sums each range in row order (eight interleaved partial sums combined in a
// fixed tree), then sums the ranges in order.  A solve therefore gives the same
// bits alone and inside a batch.
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

// (row, column) of element idx of a row-major n x R block.  32-bit unsigned
// division when idx fits (a 64-bit division is a long instruction sequence,
// a large share of these streaming kernels' work)
__device__ __forceinline__ long long row_of(long long idx, int R) {
  return idx < 0xffffffffLL ? (long long)(unsigned(idx) / unsigned(R)) : idx / R;
}
__device__ __forceinline__ int col_of(long long idx, long long row, int R) { return int(idx - row * R); }

constexpr int kMaxR = 64;   // right-hand sides per batched launch

// rows [r0, r1) of reduction range g out of G over nrows rows
__device__ __forceinline__ void red_range(long long nrows, int g, int G, long long &r0, long long &r1) {
  const long long chunk = (nrows + G - 1) / G;
  r0 = (long long)g * chunk;
  r1 = r0 + chunk < nrows ? r0 + chunk : nrows;
  if (r0 > nrows) r0 = nrows;
}

// Row arithmetic of the batched level solves with explicit rounding (no
// contraction left to the compiler), so the scalar and the vector kernels --
// a batch takes one or the other by its width -- give every element the same
// bits: z = x * d rounded, then acc - v z as one fused multiply-add.
__device__ __forceinline__ float mr_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mr_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mr_fms(float acc, float v, float z) { return fmaf(-v, z, acc); }
__device__ __forceinline__ double mr_fms(double acc, double v, double z) { return fma(-v, z, acc); }

// one dependency level of many blocks, R right-hand sides: CTA q solves chunk q;
// thread -> (row sub-index, column); mode as k_sptrsv_chunks (0-4)
template <typename T>
__global__ void k_sptrsv_chunks_mr(SolveLayout S, const int4 *chunks, int mode,
                                   const T *lval, const T *uval, const T *dinv,
                                   const T *X, T *Z, int R, const int *gate) {
  if (gate && *gate) return;
  const int4 ch = chunks[blockIdx.x];
  const int lvl = ch.x, r0 = S.lvl_row0[lvl], s0 = S.lvl_slice0[lvl];
  const int per = blockDim.x / R;
  const int q = threadIdx.x % R, sub = threadIdx.x / R;
  if (sub >= per) return;
  const bool bwd = mode == 1 || mode == 4;
  const bool from_x = mode == 3 || mode == 4 || mode == 5;   // first forward level formed where read
  const bool pre = mode == 5;                                 // values pre-scaled by 1 / L_cc
  const int *soff = bwd ? S.u_soff : S.l_soff;
  const int *sw = bwd ? S.u_sw : S.l_sw;
  const int *col = bwd ? S.u_col : S.l_col;
  const T *val = bwd ? uval : lval;
  for (int i = ch.y + sub; i < ch.y + ch.z; i += per) {
    const int r = r0 + i, sl = s0 + (i >> 5), ln = i & 31;
    const int off = soff[sl] + ln, w = sw[sl];
    const T d = dinv[r];
    T acc = mode == 4 ? X[(long long)r * R + q] * d : (bwd ? Z : X)[(long long)r * R + q];
    for (int kk = 0; kk < w; kk++) {
      const int c = col[off + kk * 32];
      const T zc = (from_x && !bwd) ? (pre ? X[(long long)c * R + q] : X[(long long)c * R + q] * dinv[c])
                                    : Z[(long long)c * R + q];
      acc -= val[off + kk * 32] * zc;
    }
    acc *= d;
    if (mode == 2 || mode == 3 || mode == 5) acc *= d;
    Z[(long long)r * R + q] = acc;
  }
}

// k_sptrsv_chunks_mr from the level-order descriptor list: CTA q solves rows
// [q P, (q+1) P) of the level's list (count rows), P = kMrRowsPerThread x the
// rows a pass of the CTA covers (blockDim / R).  A thread takes its
// kMrRowsPerThread rows together: the rows of a level depend only on rows of
// other levels, so their descriptor, operand and gathered loads are all in
// flight at once (a thread walking its rows one by one kept one dependent
// chain of loads in flight).  Each row's arithmetic is that of one row alone.
constexpr int kMrRowsPerThread = 4;
template <typename T>
__global__ void k_sptrsv_desc_mr(const int4 *desc, int count, int mode, const int *l_col, const int *u_col,
                                 const T *lval, const T *uval, const T *dinv, const T *X, T *Z, int R,
                                 const int *gate) {
  if (gate && *gate) return;
  constexpr int RR = kMrRowsPerThread;
  const int per = blockDim.x / R;
  const int q = threadIdx.x % R, sub = threadIdx.x / R;
  if (sub >= per) return;
  const bool bwd = mode == 1 || mode == 4;
  const bool from_x = mode == 3 || mode == 4 || mode == 5;
  const bool pre = mode == 5;
  const int *col = bwd ? u_col : l_col;
  const T *val = bwd ? uval : lval;
  const int i0 = blockIdx.x * per * RR;
  int r[RR], off[RR], w[RR];
  T acc[RR], d[RR];
  int wmax = 0;
#pragma unroll
  for (int u = 0; u < RR; u++) {
    const int i = i0 + sub + u * per;
    r[u] = -1; off[u] = 0; w[u] = 0;
    if (i < count) {
      const int4 dsc = desc[i];
      r[u] = dsc.x;
      off[u] = bwd ? dsc.z : dsc.y;
      w[u] = bwd ? int(unsigned(dsc.w) >> 16) : int(unsigned(dsc.w) & 0xffffu);
      wmax = max(wmax, w[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < RR; u++) {
    acc[u] = T(0);
    d[u] = T(0);
    if (r[u] >= 0) {
      d[u] = dinv[r[u]];
      const long long e = (long long)r[u] * R + q;
      acc[u] = mode == 4 ? mr_mul(X[e], d[u]) : (bwd ? Z : X)[e];
    }
  }
  for (int kk = 0; kk < wmax; kk++) {
    int c[RR];
    T v[RR], zc[RR];
#pragma unroll
    for (int u = 0; u < RR; u++) {
      if (kk < w[u]) {
        c[u] = col[off[u] + kk * 32];
        v[u] = val[off[u] + kk * 32];
      }
    }
#pragma unroll
    for (int u = 0; u < RR; u++) {
      if (kk < w[u]) {
        const long long e = (long long)c[u] * R + q;
        zc[u] = (from_x && !bwd) ? (pre ? X[e] : mr_mul(X[e], dinv[c[u]])) : Z[e];
      }
    }
#pragma unroll
    for (int u = 0; u < RR; u++)
      if (kk < w[u]) acc[u] = mr_fms(acc[u], v[u], zc[u]);
  }
#pragma unroll
  for (int u = 0; u < RR; u++) {
    if (r[u] < 0) continue;
    T a = mr_mul(acc[u], d[u]);
    if (mode == 2 || mode == 3 || mode == 5) a = mr_mul(a, d[u]);
    Z[(long long)r[u] * R + q] = a;
  }
}

// k_sptrsv_desc_mr with 16-byte vectors: a thread takes kV = 16 / sizeof(T)
// consecutive columns of a row (float4 / double2 loads and stores of X, Z and
// the gathered rows), so the row's descriptor, column indices, values and
// index arithmetic are shared by kV columns instead of being redone per
// column.  Needs R % kV == 0 (the blocks are 16-byte aligned); each element's
// arithmetic is that of the scalar kernel.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ static float get(const V &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
  __device__ static void set(V &v, int i, float x) {
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
  }
};
template <> struct Vec16<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ static double get(const V &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static void set(V &v, int i, double x) {
    if (i == 0) v.x = x; else v.y = x;
  }
};
template <typename T>
__global__ void k_sptrsv_desc_mr_v(const int4 *desc, int count, int mode, const int *l_col, const int *u_col,
                                   const T *lval, const T *uval, const T *dinv, const T *X, T *Z, int R,
                                   const int *gate) {
  if (gate && *gate) return;
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int kV = VT::n, RR = kMrRowsPerThread;
  const int tpr = R / kV;                       // threads per row
  const int per = blockDim.x / tpr;
  const int q0 = (threadIdx.x % tpr) * kV, sub = threadIdx.x / tpr;
  if (sub >= per) return;
  const bool bwd = mode == 1 || mode == 4;
  const bool from_x = mode == 3 || mode == 4 || mode == 5;
  const bool pre = mode == 5;
  const int *col = bwd ? u_col : l_col;
  const T *val = bwd ? uval : lval;
  const int i0 = blockIdx.x * per * RR;
  int r[RR], off[RR], w[RR];
  V acc[RR];
  T d[RR];
  int wmax = 0;
#pragma unroll
  for (int u = 0; u < RR; u++) {
    const int i = i0 + sub + u * per;
    r[u] = -1; off[u] = 0; w[u] = 0;
    if (i < count) {
      const int4 dsc = desc[i];
      r[u] = dsc.x;
      off[u] = bwd ? dsc.z : dsc.y;
      w[u] = bwd ? int(unsigned(dsc.w) >> 16) : int(unsigned(dsc.w) & 0xffffu);
      wmax = max(wmax, w[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < RR; u++) {
    d[u] = T(0);
    if (r[u] >= 0) {
      d[u] = dinv[r[u]];
      const V xv = *reinterpret_cast<const V *>((mode == 4 || !bwd ? X : Z) + (long long)r[u] * R + q0);
      if (mode == 4) {
#pragma unroll
        for (int e = 0; e < kV; e++) VT::set(acc[u], e, mr_mul(VT::get(xv, e), d[u]));
      } else {
        acc[u] = xv;
      }
    }
  }
  for (int kk = 0; kk < wmax; kk++) {
    int c[RR];
    T v[RR], dc[RR];
#pragma unroll
    for (int u = 0; u < RR; u++) {
      if (kk < w[u]) {
        c[u] = col[off[u] + kk * 32];
        v[u] = val[off[u] + kk * 32];
      }
    }
    V zc[RR];
#pragma unroll
    for (int u = 0; u < RR; u++) {
      if (kk < w[u]) {
        const bool fx = from_x && !bwd;
        zc[u] = *reinterpret_cast<const V *>((fx ? X : Z) + (long long)c[u] * R + q0);
        dc[u] = (fx && !pre) ? dinv[c[u]] : T(1);
      }
    }
#pragma unroll
    for (int u = 0; u < RR; u++) {
      if (kk < w[u]) {
        const bool scale = from_x && !bwd && !pre;
#pragma unroll
        for (int e = 0; e < kV; e++) {
          const T z = scale ? mr_mul(VT::get(zc[u], e), dc[u]) : VT::get(zc[u], e);
          VT::set(acc[u], e, mr_fms(VT::get(acc[u], e), v[u], z));
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < RR; u++) {
    if (r[u] < 0) continue;
    V o;
#pragma unroll
    for (int e = 0; e < kV; e++) {
      T a = mr_mul(VT::get(acc[u], e), d[u]);
      if (mode == 2 || mode == 3 || mode == 5) a = mr_mul(a, d[u]);
      VT::set(o, e, a);
    }
    *reinterpret_cast<V *>(Z + (long long)r[u] * R + q0) = o;
  }
}

// Y = E^T Z = a^-1 Ehat^T Z_B - a Z_C   (interface rows j, columns q)
template <typename T>
__global__ void k_et_mr(int s, int m, const int *eht_rp, const int *eht_ci,
                        const T *eht_val, T ia, T a, const T *Z, T *Y, int R,
                        const int *gate) {
  if (gate && *gate) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long j = row_of(idx, R);
  const int q = col_of(idx, j, R);
  if (j >= s) return;
  T acc = 0;
  for (int p = eht_rp[j]; p < eht_rp[j + 1]; p++) acc = mr_fms(acc, -eht_val[p], Z[(long long)eht_ci[p] * R + q]);
  Y[j * R + q] = mr_fms(mr_mul(ia, acc), a, Z[(m + j) * R + q]);
}

// RHS_B = X_B + a^-1 Ehat W   (interior rows)
template <typename T>
__global__ void k_e_interior_mr(int m, const int *eh_rp, const int *eh_ci,
                                const T *eh_val, T ia, const T *W, const T *X, T *RHS,
                                int R, const int *gate) {
  if (gate && *gate) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r = row_of(idx, R);
  const int q = col_of(idx, r, R);
  if (r >= m) return;
  T acc = 0;
  for (int p = eh_rp[r]; p < eh_rp[r + 1]; p++) acc = mr_fms(acc, -eh_val[p], W[(long long)eh_ci[p] * R + q]);
  RHS[r * R + q] = mr_fms(X[r * R + q], -ia, acc);
}

// k_et_mr and k_e_interior_mr with 16-byte vectors of kV columns per thread
// (R % kV == 0); per element the arithmetic of the scalar kernels (explicit
// rounding, so both forms give the same bits)
template <typename T>
__global__ void k_et_mr_v(int s, int m, const int *eht_rp, const int *eht_ci, const T *eht_val, T ia, T a,
                          const T *Z, T *Y, int R, const int *gate) {
  if (gate && *gate) return;
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int kV = VT::n;
  const int tpr = R / kV;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long j = t / tpr;
  if (j >= s) return;
  const int q0 = int(t - j * tpr) * kV;
  V acc;
#pragma unroll
  for (int e = 0; e < kV; e++) VT::set(acc, e, T(0));
  for (int p = eht_rp[j]; p < eht_rp[j + 1]; p++) {
    const T v = eht_val[p];
    const V z = *reinterpret_cast<const V *>(Z + (long long)eht_ci[p] * R + q0);
#pragma unroll
    for (int e = 0; e < kV; e++) VT::set(acc, e, mr_fms(VT::get(acc, e), -v, VT::get(z, e)));
  }
  const V zc = *reinterpret_cast<const V *>(Z + (long long)(m + j) * R + q0);
  V o;
#pragma unroll
  for (int e = 0; e < kV; e++) VT::set(o, e, mr_fms(mr_mul(ia, VT::get(acc, e)), a, VT::get(zc, e)));
  *reinterpret_cast<V *>(Y + j * R + q0) = o;
}

template <typename T>
__global__ void k_e_interior_mr_v(int m, const int *eh_rp, const int *eh_ci, const T *eh_val, T ia, const T *W,
                                  const T *X, T *RHS, int R, const int *gate) {
  if (gate && *gate) return;
  using VT = Vec16<T>;
  using V = typename VT::V;
  constexpr int kV = VT::n;
  const int tpr = R / kV;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r = t / tpr;
  if (r >= m) return;
  const int q0 = int(t - r * tpr) * kV;
  V acc;
#pragma unroll
  for (int e = 0; e < kV; e++) VT::set(acc, e, T(0));
  for (int p = eh_rp[r]; p < eh_rp[r + 1]; p++) {
    const T v = eh_val[p];
    const V w = *reinterpret_cast<const V *>(W + (long long)eh_ci[p] * R + q0);
#pragma unroll
    for (int e = 0; e < kV; e++) VT::set(acc, e, mr_fms(VT::get(acc, e), -v, VT::get(w, e)));
  }
  const V x = *reinterpret_cast<const V *>(X + r * R + q0);
  V o;
#pragma unroll
  for (int e = 0; e < kV; e++) VT::set(o, e, mr_fms(VT::get(x, e), -ia, VT::get(acc, e)));
  *reinterpret_cast<V *>(RHS + r * R + q0) = o;
}

// partials[g][c*R + q] = sum over rows of range g (in order) of U[row][c] Y[row][q]
// (stage 1 of U_k^T Y, k x R).  Needs k*R <= 4 * blockDim.
template <typename T, typename TU>
__global__ void __launch_bounds__(256)
k_utx_mr_partial(long long nrows, int k, const TU *U, const T *Y, int R, T *partials,
                 const int *gate) {
  if (gate && *gate) return;
  __shared__ T us[32 * 64];
  __shared__ T ys[32 * kMaxR];
  long long r0, r1;
  red_range(nrows, blockIdx.x, gridDim.x, r0, r1);
  const int no = k * R;
  T acc[4] = {0, 0, 0, 0};
  for (long long base = r0; base < r1; base += 32) {
    const int nt = int(min(32LL, r1 - base));
    for (int t = threadIdx.x; t < nt * k; t += blockDim.x)
      us[t] = T(to_acc(U[(base + t / k) * k + t % k]));
    for (int t = threadIdx.x; t < nt * R; t += blockDim.x) ys[t] = Y[base * R + t];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int o = threadIdx.x + u * blockDim.x;
      if (o < no) {
        const int c = o / R, q = o % R;
        T a = acc[u];
        for (int rr = 0; rr < nt; rr++) a += us[rr * k + c] * ys[rr * R + q];
        acc[u] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int o = threadIdx.x + u * blockDim.x;
    if (o < no) partials[(long long)blockIdx.x * no + o] = acc[u];
  }
}

// T[o] = coef[o / R] * sum_g partials[g][o] (o = c*R + q), fixed order; with H:
// T = H * (that k x R block).  One CTA; k*R <= 1024.
template <typename T>
__global__ void k_reduce_mr(int G, int k, int R, const T *partials, const T *coef,
                            const T *H, T *out, const int *gate) {
  if (gate && *gate) return;
  __shared__ T tmp[1024];
  const int no = k * R;
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    T s = 0;
    for (int g = 0; g < G; g++) s += partials[(long long)g * no + o];
    tmp[o] = coef ? coef[o / R] * s : s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    if (H) {
      const int c = o / R, q = o % R;
      T s = 0;
      for (int b = 0; b < k; b++) s += H[c * k + b] * tmp[b * R + q];
      out[o] = s;
    } else {
      out[o] = tmp[o];
    }
  }
}

// W = Y/(1-theta) + U_k Tm ; RHS_C = X_C - a W   (interface rows, DDLR-1)
template <typename T, typename TU>
__global__ void k_w_rhs_mr(int s, int m, int k, const TU *U, const T *Tm, const T *Y,
                           const T *inv1mt, T a, const T *X, T *W, T *RHS, int R,
                           const int *gate) {
  if (gate && *gate) return;
  __shared__ T ts[1024];
  for (int o = threadIdx.x; o < k * R; o += blockDim.x) ts[o] = Tm[o];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long j = row_of(idx, R);
  const int q = col_of(idx, j, R);
  if (j >= s) return;
  const TU *u = U + j * k;
  T acc = 0;
  for (int c = 0; c < k; c++) acc += T(to_acc(u[c])) * ts[c * R + q];
  const T wj = (*inv1mt) * Y[j * R + q] + acc;
  W[j * R + q] = wj;
  RHS[(m + j) * R + q] = X[(m + j) * R + q] - a * wj;
}

// Uo += U_k HT   (DDLR-2, all rows)
template <typename T, typename TU>
__global__ void k_u_add_mr(long long nrows, int k, const TU *U, const T *HT, T *Uo, int R,
                           const int *gate) {
  if (gate && *gate) return;
  __shared__ T ts[1024];
  for (int o = threadIdx.x; o < k * R; o += blockDim.x) ts[o] = HT[o];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r = row_of(idx, R);
  const int q = col_of(idx, r, R);
  if (r >= nrows) return;
  const TU *u = U + r * k;
  T acc = 0;
  for (int c = 0; c < k; c++) acc += T(to_acc(u[c])) * ts[c * R + q];
  Uo[r * R + q] += acc;
}

// --------------------------------------------- tensor-core U_k products
// The multi-RHS U_k products are dense GEMMs (s x k by k x R, reduced over the
// s rows for U_k^T Y), so with FP32 preconditioner vectors they run on the
// tensor cores: mma.sync m16n8k8 with TF32 operands and FP32 accumulation.
// An FP32 operand x is split into its TF32 rounding hi and the TF32 rounding
// of x - hi; the three products hi*hi + hi*lo + lo*hi keep about the accuracy
// of FP32 products (the dropped lo*lo term is 2^-22 relative).  A BF16 U_k is
// exact in TF32 (lo = 0): two products.  An output element depends only on
// its own row of one operand and column of the other, and the row ranges and
// their order are those of the scalar kernels, so a column's result does not
// depend on the other columns of its batch.
__device__ __forceinline__ unsigned tf32_of(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, unsigned &hi, unsigned &lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += a * b with both split: three products (two when a is exact in TF32)
template <bool kAExact>
__device__ __forceinline__ void mma_tf32x3(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4],
                                           const unsigned (&bh)[2], const unsigned (&bl)[2]) {
  if (!kAExact) mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}
template <typename TU> struct TcExact { static constexpr bool v = false; };
template <> struct TcExact<__nv_bfloat16> { static constexpr bool v = true; };

// partials[g][c*R + q] = sum over the rows of range g of U[row][c] Y[row][q]
// (stage 1 of U_k^T Y, as k_utx_mr_partial), on the tensor cores.  256
// threads; k <= 64, R <= 64.  The CTA streams its rows in stages of 32 rows
// (the U and Y tiles of a stage are contiguous in memory), zero-padded to
// 16-column (c) and 8-column (q) tiles; warp w owns output tiles w and w + 8.
constexpr int kTcRows = 32, kTcUS = 68, kTcYS = 72;   // smem strides: conflict-free fragment reads
template <typename TU>
__global__ void __launch_bounds__(256)
k_utx_mr_tc(long long nrows, int k, const TU *U, const float *Y, int R, float *partials, const int *gate) {
  if (gate && *gate) return;
  __shared__ float us[kTcRows * kTcUS];
  __shared__ float ys[kTcRows * kTcYS];
  constexpr bool kEx = TcExact<TU>::v;
  long long r0, r1;
  red_range(nrows, blockIdx.x, gridDim.x, r0, r1);
  const int MT = (k + 15) >> 4, NQ = (R + 7) >> 3, ntile = MT * NQ;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int i = threadIdx.x; i < kTcRows * kTcUS; i += blockDim.x) us[i] = 0.f;
  for (int i = threadIdx.x; i < kTcRows * kTcYS; i += blockDim.x) ys[i] = 0.f;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  __syncthreads();
  for (long long base = r0; base < r1; base += kTcRows) {
    const int nt = int(min((long long)kTcRows, r1 - base));
    const TU *ub = U + base * k;
    const float *yb = Y + base * R;
    for (int i = threadIdx.x; i < nt * k; i += blockDim.x) {
      const int rr = int(unsigned(i) / unsigned(k));
      us[rr * kTcUS + (i - rr * k)] = to_acc(ub[i]);
    }
    for (int i = threadIdx.x; i < nt * R; i += blockDim.x) {
      const int rr = int(unsigned(i) / unsigned(R));
      ys[rr * kTcYS + (i - rr * R)] = yb[i];
    }
    if (nt < kTcRows) {          // last stage of the range: zero the rows past its end
      for (int i = threadIdx.x; i < (kTcRows - nt) * 64; i += blockDim.x) {
        const int rr = nt + (i >> 6), c = i & 63;
        us[rr * kTcUS + c] = 0.f;
        ys[rr * kTcYS + c] = 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < 2; sl++) {
      const int tt = w + 8 * sl;
      if (tt < ntile) {
        const int c0 = (tt / NQ) << 4, q0 = (tt % NQ) << 3;
#pragma unroll
        for (int kk = 0; kk < kTcRows; kk += 8) {
          unsigned ah[4], al[4], bh[2], bl[2];
          tf32_split(us[(kk + t) * kTcUS + c0 + g], ah[0], al[0]);
          tf32_split(us[(kk + t) * kTcUS + c0 + g + 8], ah[1], al[1]);
          tf32_split(us[(kk + t + 4) * kTcUS + c0 + g], ah[2], al[2]);
          tf32_split(us[(kk + t + 4) * kTcUS + c0 + g + 8], ah[3], al[3]);
          tf32_split(ys[(kk + t) * kTcYS + q0 + g], bh[0], bl[0]);
          tf32_split(ys[(kk + t + 4) * kTcYS + q0 + g], bh[1], bl[1]);
          mma_tf32x3<kEx>(acc[sl], ah, al, bh, bl);
        }
      }
    }
    __syncthreads();
  }
  const int no = k * R;
#pragma unroll
  for (int sl = 0; sl < 2; sl++) {
    const int tt = w + 8 * sl;
    if (tt >= ntile) continue;
    const int c0 = (tt / NQ) << 4, q0 = (tt % NQ) << 3;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int c = c0 + g + ((e & 2) ? 8 : 0), q = q0 + 2 * t + (e & 1);
      if (c < k && q < R) partials[(long long)blockIdx.x * no + c * R + q] = acc[sl][e];
    }
  }
}

// out[o] = (coef ? coef[o / R] : 1) * sum over g < G of partials[g * no + o]
// (o < no = k R), in a fixed order: warp w of a CTA sums its eighth of the g
// range for 32 consecutive o (one per lane, coalesced), then the eight warp
// sums are added in order.  Grid: ceil(no / 32) CTAs of 256 threads.
template <typename T>
__global__ void __launch_bounds__(256)
k_reduce_cols_mr(int G, int no, int R, const T *partials, const T *coef, T *out, const int *gate) {
  if (gate && *gate) return;
  __shared__ T sm[8][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int o = blockIdx.x * 32 + l;
  const int per = (G + 7) / 8, g0 = w * per, g1 = min(G, g0 + per);
  T v = 0;
  if (o < no)
    for (int g = g0; g < g1; g++) v += partials[(long long)g * no + o];
  sm[w][l] = v;
  __syncthreads();
  if (w == 0 && o < no) {
    T t = 0;
    for (int ww = 0; ww < 8; ww++) t += sm[ww][l];
    out[o] = coef ? coef[o / R] * t : t;
  }
}

// Rows [j0, j0 + 16) of D = U_k Tm (U row-major nrows x k, Tm k x R) on the
// tensor cores for one warp: acc[nq] holds the 16 x 8 tile of columns
// [8 nq, 8 nq + 8).  ts: Tm in shared memory with row stride TS (floats).
template <typename TU>
__device__ __forceinline__ void tc_rows_times_small(long long nrows, int k, const TU *U, const float *ts, int TS,
                                                    int NQ, long long j0, float (&acc)[8][4]) {
  constexpr bool kEx = TcExact<TU>::v;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long ja = j0 + g, jb = j0 + g + 8;
  for (int c0 = 0; c0 < k; c0 += 8) {
    const int ca = c0 + t, cb = c0 + t + 4;
    auto uat = [&](long long j, int c) { return (j < nrows && c < k) ? to_acc(U[j * k + c]) : 0.f; };
    unsigned ah[4], al[4];
    tf32_split(uat(ja, ca), ah[0], al[0]);
    tf32_split(uat(jb, ca), ah[1], al[1]);
    tf32_split(uat(ja, cb), ah[2], al[2]);
    tf32_split(uat(jb, cb), ah[3], al[3]);
#pragma unroll
    for (int nq = 0; nq < 8; nq++) {
      if (nq < NQ) {
        unsigned bh[2], bl[2];
        tf32_split(ca < k ? ts[ca * TS + nq * 8 + g] : 0.f, bh[0], bl[0]);
        tf32_split(cb < k ? ts[cb * TS + nq * 8 + g] : 0.f, bh[1], bl[1]);
        mma_tf32x3<kEx>(acc[nq], ah, al, bh, bl);
      }
    }
  }
}

// shared-memory copy of the k x R block Tm with row stride TS (zero-padded to
// a multiple of 8 columns); returns TS.  ts holds k * TS floats.
__device__ __forceinline__ int tc_stage_small(const float *Tm, int k, int R, float *ts) {
  const int TS = ((R + 31) & ~31) + 8;      // = 8 (mod 32): conflict-free B fragment reads
  for (int o = threadIdx.x; o < k * TS; o += blockDim.x) {
    const int c = o / TS, q = o - c * TS;
    ts[o] = q < R ? Tm[c * R + q] : 0.f;
  }
  __syncthreads();
  return TS;
}

// k_w_rhs_mr on the tensor cores: W = Y/(1-theta) + U_k Tm ; RHS_C = X_C - a W.
// A warp computes 16 interface rows x all R columns.  256 threads.
template <typename TU>
__global__ void __launch_bounds__(256)
k_w_rhs_mr_tc(int s, int m, int k, const TU *U, const float *Tm, const float *Y, const float *inv1mt, float a,
              const float *X, float *W, float *RHS, int R, const int *gate) {
  if (gate && *gate) return;
  __shared__ float ts[64 * 72];
  const int TS = tc_stage_small(Tm, k, R, ts);
  const int NQ = (R + 7) >> 3;
  const long long j0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16;
  if (j0 >= s) return;
  float acc[8][4];
#pragma unroll
  for (int nq = 0; nq < 8; nq++) acc[nq][0] = acc[nq][1] = acc[nq][2] = acc[nq][3] = 0.f;
  tc_rows_times_small<TU>(s, k, U, ts, TS, NQ, j0, acc);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float i1 = *inv1mt;
#pragma unroll
  for (int nq = 0; nq < 8; nq++) {
    if (nq >= NQ) continue;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const long long j = j0 + g + ((e & 2) ? 8 : 0);
      const int q = nq * 8 + 2 * t + (e & 1);
      if (j < s && q < R) {
        const float wj = i1 * Y[j * R + q] + acc[nq][e];
        W[j * R + q] = wj;
        RHS[(m + j) * R + q] = X[(m + j) * R + q] - a * wj;
      }
    }
  }
}

// k_u_add_mr on the tensor cores: Uo += U_k HT (DDLR-2, all rows)
template <typename TU>
__global__ void __launch_bounds__(256)
k_u_add_mr_tc(long long nrows, int k, const TU *U, const float *HT, float *Uo, int R, const int *gate) {
  if (gate && *gate) return;
  __shared__ float ts[64 * 72];
  const int TS = tc_stage_small(HT, k, R, ts);
  const int NQ = (R + 7) >> 3;
  const long long j0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16;
  if (j0 >= nrows) return;
  float acc[8][4];
#pragma unroll
  for (int nq = 0; nq < 8; nq++) acc[nq][0] = acc[nq][1] = acc[nq][2] = acc[nq][3] = 0.f;
  tc_rows_times_small<TU>(nrows, k, U, ts, TS, NQ, j0, acc);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nq = 0; nq < 8; nq++) {
    if (nq >= NQ) continue;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const long long j = j0 + g + ((e & 2) ? 8 : 0);
      const int q = nq * 8 + 2 * t + (e & 1);
      if (j < nrows && q < R) Uo[j * R + q] += acc[nq][e];
    }
  }
}

// Q = A P (sliced ELL, device order), R columns
template <typename T>
__global__ void k_spmv_mr(int n, const int *soff, const int *sw, const int *col,
                          const T *val, const T *P, T *Q, int R, const int *gate) {
  if (gate && *gate) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r = row_of(idx, R);
  const int q = col_of(idx, r, R);
  if (r >= n) return;
  const int g = int(r >> 5), l = int(r & 31);
  const int off = soff[g] + l, w = sw[g];
  T acc = 0;
  for (int kk = 0; kk < w; kk++) acc += val[off + kk * 32] * P[(long long)col[off + kk * 32] * R + q];
  Q[r * R + q] = acc;
}

// partials[g][q] (and [g][R+q]) = column dot products of A.B (and A.C) over
// range g of the rows.  The range is cut into 8 equal sub-ranges, one warp
// each; a lane sums its column over the sub-range in row order with eight
// interleaved partial sums (fixed tree), and the 8 sub-range sums are added in
// order.  Launch with 256 threads; lanes q >= R idle.
__global__ void __launch_bounds__(256)
k_dot_mr_partial(long long n, int R, const double *A, const double *B,
                 const double *C, double *partials, const int *gate) {
  if (gate && *gate) return;
  __shared__ double red[8][2 * kMaxR];
  const int w = threadIdx.x >> 5, q = threadIdx.x & 31;
  long long g0, g1;
  red_range(n, blockIdx.x, gridDim.x, g0, g1);
  const long long sub = (g1 - g0 + 7) / 8;
  for (int qq = q; qq < R; qq += 32) {
    long long r0 = g0 + w * sub, r1 = r0 + sub;
    if (r0 > g1) r0 = g1;
    if (r1 > g1) r1 = g1;
    double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0}, t8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long r = r0;
    for (; r + 8 <= r1; r += 8) {
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const double a = A[(r + u) * R + qq];
        s8[u] = fma(a, B[(r + u) * R + qq], s8[u]);
        if (C) t8[u] = fma(a, C[(r + u) * R + qq], t8[u]);
      }
    }
    for (int u = 0; r < r1; r++, u++) {
      const double a = A[r * R + qq];
      s8[u] = fma(a, B[r * R + qq], s8[u]);
      if (C) t8[u] = fma(a, C[r * R + qq], t8[u]);
    }
    red[w][qq] = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
    red[w][R + qq] = ((t8[0] + t8[1]) + (t8[2] + t8[3])) + ((t8[4] + t8[5]) + (t8[6] + t8[7]));
  }
  __syncthreads();
  for (int o = threadIdx.x; o < (C ? 2 * R : R); o += blockDim.x) {
    double sm = 0;
    for (int ww = 0; ww < 8; ww++) sm += red[ww][o];
    partials[(long long)blockIdx.x * 2 * R + o] = sm;
  }
}

// ------------------------------------------------------- block PCG control
struct PcgStateMR {
  double rz[kMaxR], pq[kMaxR], alpha[kMaxR], beta[kMaxR], rr[kMaxR], bb[kMaxR];
  double tol2[kMaxR], rt2[kMaxR];
  int its[kMaxR], done[kMaxR], status[kMaxR], check[kMaxR], restart[kMaxR];
  int fresh[kMaxR];   // admitted into a running block: joins at the next preconditioner step
  int R, maxit, flexible, all_done, any_check;
  int no_check;   // 1 unless some column's true residual is to be checked this iteration
  int pad[2];
};

// ---- fused step kernels of the block PCG with their column dot products.
// Rows are taken in blocks of kFbRows = 64; in a block, row lane l (of 8)
// takes rows l, l + 8, ... of the block in order, a thread owns one (row
// lane, column) pair, and the 8 lane sums of a column are added in lane order
// into partials[block][q].  k_fused_partials_reduce then adds the blocks of each
// of the G = kRedGrid reduction ranges in order into the [g][2R] layout the
// scalar kernels read.  Nothing in this order depends on R, so a column's dot
// products are the same in every batch.  Launch: a CTA takes fb_groups(R)
// row blocks (8 R threads each, at least 256 threads a CTA for small R, so
// narrow blocks are not held to a few threads per SM by the CTA limit).
constexpr int kFbRows = 64, kFbLanes = 8, kFbCta = 256, kFbMaxRed = 512;
__host__ __device__ inline int fb_groups(int R) { return R * kFbLanes >= kFbCta ? 1 : kFbCta / (R * kFbLanes); }

// Q = A P (sliced ELL) and the column partials of P.Q.  Bound by the FP64
// pipe (one FMA per stored entry and column, one more for the dot product:
// 8 per row and column for the 7-point operators), so the products are not
// batched in wider predicated groups, whose idle lanes still take FP64 issue
// slots.
__global__ void k_spmv_pq_mr(int n, const int *__restrict__ soff, const int *__restrict__ sw,
                             const int *__restrict__ col, const double *__restrict__ val,
                             const double *__restrict__ P, double *__restrict__ Q, int R, double *bpart,
                             const int *gate) {
  if (gate && *gate) return;
  __shared__ double red[kFbMaxRed];
  const int gt = kFbLanes * R, gi = threadIdx.x / gt, tt = threadIdx.x % gt;
  const int q = tt % R, l = tt / R;
  const int nblk = (n + kFbRows - 1) / kFbRows;
  const int rb = blockIdx.x * fb_groups(R) + gi;
  double acc = 0.0;
  if (rb < nblk) {
    const int r0 = rb * kFbRows;
    for (int i = l; i < kFbRows; i += kFbLanes) {
      const int r = r0 + i;
      if (r >= n) break;
      const int g = r >> 5, ln = r & 31;
      const int off = soff[g] + ln, w = sw[g];
      double t = 0;
      for (int kk = 0; kk < w; kk++) t = fma(val[off + kk * 32], P[(long long)col[off + kk * 32] * R + q], t);
      const long long e = (long long)r * R + q;
      Q[e] = t;
      acc = fma(P[e], t, acc);
    }
  }
  red[(gi * kFbLanes + l) * R + q] = acc;
  __syncthreads();
  if (l == 0 && rb < nblk) {
    double v = 0.0;
    for (int j = 0; j < kFbLanes; j++) v += red[(gi * kFbLanes + j) * R + q];
    bpart[(long long)rb * R + q] = v;
  }
}

// X += alpha P; Rr -= alpha Q for the running columns, and the column
// partials of Rr.Rr (all columns)
__global__ void k_update_rr_mr(long long n, const PcgStateMR *st, const double *P, const double *Q, double *X,
                               double *Rr, double *bpart) {
  if (st->all_done) return;
  __shared__ double red[kFbMaxRed];
  const int R = st->R;
  const int gt = kFbLanes * R, gi = threadIdx.x / gt, tt = threadIdx.x % gt;
  const int q = tt % R, l = tt / R;
  const long long nblk = (n + kFbRows - 1) / kFbRows;
  const long long rb = (long long)blockIdx.x * fb_groups(R) + gi;
  const bool run = !st->done[q];
  const double a = st->alpha[q];
  double acc = 0.0;
  if (rb < nblk) {
    const long long r0 = rb * kFbRows;
    for (int i = l; i < kFbRows; i += kFbLanes) {
      const long long r = r0 + i;
      if (r >= n) break;
      const long long e = r * R + q;
      double rv = Rr[e];
      if (run) {
        X[e] += a * P[e];
        rv -= a * Q[e];
        Rr[e] = rv;
      }
      acc = fma(rv, rv, acc);
    }
  }
  red[(gi * kFbLanes + l) * R + q] = acc;
  __syncthreads();
  if (l == 0 && rb < nblk) {
    double v = 0.0;
    for (int j = 0; j < kFbLanes; j++) v += red[(gi * kFbLanes + j) * R + q];
    bpart[rb * R + q] = v;
  }
}

// partials[g][q] (stride 2R) = sum over the blocks of reduction range g, in
// order, of bpart[block][q]; grid kRedGrid, R threads
__global__ void k_fused_partials_reduce(int nblocks, int R, const double *bpart, double *partials,
                                        const int *gate) {
  if (gate && *gate) return;
  const int q = threadIdx.x;
  if (q >= R) return;
  long long b0, b1;
  red_range(nblocks, blockIdx.x, gridDim.x, b0, b1);
  double v = 0.0;
  for (long long b = b0; b < b1; b++) v += bpart[b * R + q];
  partials[(long long)blockIdx.x * 2 * R + q] = v;
}


// sums[o] = sum over the G partial rows of column o (o < no), a warp per
// column: lanes take every 32nd partial in order, then a shuffle tree (a
// serial sum of G = 304 FP64 values is ~20k cycles of add latency here).
// Every thread of the block must call it (it ends in a barrier).
constexpr int kScalarThreads = 1024;
__device__ __forceinline__ void col_sums(const double *partials, int G, int R, int no, double *sums) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int o = w; o < no; o += nw) {
    double v = 0;
    for (int g = l; g < G; g += 32) v += partials[(long long)g * 2 * R + o];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (l == 0) sums[o] = v;
  }
  __syncthreads();
}

__global__ void k_pcgmr_init(PcgStateMR *st, const double *partials, int G, int R,
                             double tol, int maxit, int flexible) {
  const int q = threadIdx.x;
  __shared__ double sm[kMaxR];
  col_sums(partials, G, R, R, sm);
  if (q == 0) {
    st->R = R; st->maxit = maxit; st->flexible = flexible; st->any_check = 0; st->no_check = 1;
  }
  if (q < R) {
    const double bb = sm[q];
    st->bb[q] = bb;
    st->tol2[q] = tol * tol * bb;
    st->its[q] = 0; st->status[q] = 0; st->check[q] = 0; st->restart[q] = 0; st->fresh[q] = 0;
    st->done[q] = (bb == 0.0) ? 1 : 0;
    st->rz[q] = 0;
  }
  __syncthreads();
  if (q == 0) {
    int all = 1;
    for (int c = 0; c < R; c++) all &= st->done[c];
    st->all_done = all;
  }
}

__global__ void k_pcgmr_rz0(PcgStateMR *st, const double *partials, int G) {
  if (st->all_done) return;
  const int q = threadIdx.x, R = st->R;
  __shared__ double sm[kMaxR];
  col_sums(partials, G, R, R, sm);
  if (q < R && !st->done[q]) {
    const double s = sm[q];
    st->rz[q] = s;
    if (!(s == s) || isinf(s)) { st->status[q] = 7; st->done[q] = 1; }
  }
}

__global__ void k_pcgmr_alpha(PcgStateMR *st, const double *partials, int G) {
  if (st->all_done) return;
  const int q = threadIdx.x, R = st->R;
  __shared__ double sm[kMaxR];
  col_sums(partials, G, R, R, sm);
  if (q < R) {
    double a = 0.0;
    if (!st->done[q] && !st->fresh[q]) {
      const double pq = sm[q];
      st->pq[q] = pq;
      a = st->rz[q] / pq;
      if (!(a == a) || isinf(a)) { st->status[q] = 7; st->done[q] = 1; a = 0.0; }
    }
    st->alpha[q] = a;
  }
}


__global__ void k_pcgmr_rr(PcgStateMR *st, const double *partials, int G) {
  if (st->all_done) return;
  const int q = threadIdx.x, R = st->R;
  __shared__ int anyc;
  __shared__ double sm[kMaxR];
  if (q == 0) anyc = 0;
  col_sums(partials, G, R, R, sm);
  if (q < R && !st->done[q] && !st->fresh[q]) {
    const double rr = sm[q];
    st->rr[q] = rr;
    st->its[q] += 1;
    if (!(rr == rr) || isinf(rr)) { st->status[q] = 7; st->done[q] = 1; }
    else {
      st->check[q] = (rr <= st->tol2[q]) ? 1 : 0;
      if (st->check[q]) atomicOr(&anyc, 1);
      else if (st->its[q] >= st->maxit) { st->status[q] = 5; st->done[q] = 1; }
    }
  }
  __syncthreads();
  if (q == 0) { st->any_check = anyc; st->no_check = anyc ? 0 : 1; }
}

// T = B - A X for the columns whose true residual is to be checked
__global__ void k_pcgmr_true_res(int n, const PcgStateMR *st, const int *soff, const int *sw,
                                 const int *col, const double *val, const double *B,
                                 const double *X, double *Tt) {
  if (st->all_done || !st->any_check) return;
  const int R = st->R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)n * R;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = row_of(idx, R);
    const int q = col_of(idx, r, R);
    if (!st->check[q]) continue;
    const int g = int(r >> 5), l = int(r & 31);
    const int off = soff[g] + l, w = sw[g];
    double ax = 0;
    for (int kk = 0; kk < w; kk++) ax += val[off + kk * 32] * X[(long long)col[off + kk * 32] * R + q];
    Tt[idx] = B[idx] - ax;
  }
}

__global__ void k_pcgmr_true_dec(PcgStateMR *st, const double *partials, int G) {
  const int q = threadIdx.x, R = st->R;
  if (q == 0) st->no_check = 1;   // the check of this iteration is consumed here
  if (st->all_done || !st->any_check) return;
  __shared__ double sm[kMaxR];
  col_sums(partials, G, R, R, sm);
  if (q < R && st->check[q] && !st->done[q]) {
    const double rt2 = sm[q];
    st->rt2[q] = rt2;
    if (rt2 <= st->tol2[q]) { st->status[q] = 0; st->done[q] = 1; }
    else {
      st->restart[q] = 1;
      if (st->its[q] >= st->maxit) { st->status[q] = 5; st->done[q] = 1; }
    }
  }
  if (q < R) st->check[q] = 0;
}

// (a restart is only ever set by a true-residual check of this iteration)
__global__ void k_pcgmr_copy_r(long long n, const PcgStateMR *st, const double *Tt, double *Rr) {
  if (st->all_done || !st->any_check) return;
  const int R = st->R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n * R;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = col_of(idx, row_of(idx, R), R);
    if (st->restart[q] && !st->done[q]) Rr[idx] = Tt[idx];
  }
}

__global__ void k_pcgmr_beta(PcgStateMR *st, const double *partials, int G) {
  if (st->all_done) return;
  const int q = threadIdx.x, R = st->R;
  __shared__ double sm[2 * kMaxR];
  col_sums(partials, G, R, 2 * R, sm);
  if (q < R && !st->done[q]) {
    const double rzn = sm[q];
    const double rzo = sm[R + q];
    double beta = st->flexible ? (rzn - rzo) / st->rz[q] : rzn / st->rz[q];
    if (st->restart[q] || st->fresh[q]) beta = 0.0;
    st->beta[q] = beta;
    st->rz[q] = rzn;
    st->restart[q] = 0;
    st->fresh[q] = 0;
    if (!(rzn == rzn) || isinf(rzn)) { st->status[q] = 7; st->done[q] = 1; }
  }
  __syncthreads();
  if (q == 0) {
    int all = 1;
    for (int c = 0; c < R; c++) all &= st->done[c];
    st->all_done = all;
  }
}

// P = Z + beta P (and Zold = Z) for the columns still running
__global__ void k_pcgmr_p(long long n, const PcgStateMR *st, const double *Z, double *P,
                          double *Zold) {
  const int R = st->R;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * R) return;
  const int q = col_of(idx, row_of(idx, R), R);
  if (st->done[q]) return;
  const double z = Z[idx];
  P[idx] = z + st->beta[q] * P[idx];
  if (Zold) Zold[idx] = z;
}

// ------------------------------------------------ continuous batching (serving)
// A column admitted into a running block starts as a fresh solve (x0 = 0,
// r = b, p = 0) marked `fresh`: in the next iteration the step and the
// residual test skip it (alpha = 0 against p = 0 and A p = 0 leaves x and r
// unchanged), the preconditioner gives z = M^-1 b, r.z becomes its rz and
// beta = 0 makes p = z -- the state a solve started alone has after its
// initial apply.  Every later iteration of the column is the same arithmetic
// as alone, so its result does not depend on when it was admitted or which
// other columns share the block.

// column q of a row-major n x R block <- a vector in original order
__global__ void k_col_in(int n, int R, int q, const int *perm, const double *in, double *out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[(long long)g * R + q] = in[perm[g]];
}
// a vector in original order <- column q of a row-major n x R block
__global__ void k_col_out(int n, int R, int q, const int *perm, const double *in, double *out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[perm[g]] = in[(long long)g * R + q];
}
// admitted columns (mask[q] != 0): X = 0, Rr = B, P = 0
__global__ void k_slot_reset(long long n, int R, const int *mask, const double *B, double *X, double *Rr,
                             double *P) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * R) return;
  const int q = col_of(idx, row_of(idx, R), R);
  if (!mask[q]) return;
  X[idx] = 0.0;
  Rr[idx] = B[idx];
  P[idx] = 0.0;
}
// the per-column state of the admitted columns (partials: column sums of B.B)
__global__ void k_slot_init(PcgStateMR *st, const double *partials, int G, const int *mask, int R, double tol,
                            int maxit, int flexible) {
  const int q = threadIdx.x;
  __shared__ double sm[kMaxR];
  col_sums(partials, G, R, R, sm);
  if (q == 0) { st->R = R; st->maxit = maxit; st->flexible = flexible; }
  if (q < R && mask[q]) {
    const double bb = sm[q];
    st->bb[q] = bb;
    st->tol2[q] = tol * tol * bb;
    st->rt2[q] = 0.0;
    st->rr[q] = bb;
    st->its[q] = 0; st->status[q] = 0; st->check[q] = 0;
    st->done[q] = (bb == 0.0) ? 1 : 0;
    st->fresh[q] = 1;       // beta = 0 at its first preconditioner step (and
    st->restart[q] = 0;     // no copy of a true residual: restart is the
    st->rz[q] = 0.0;        // mark of a failed check of this iteration)
  }
  __syncthreads();
  if (q == 0) {
    int all = 1;
    for (int c = 0; c < R; c++) all &= st->done[c];
    st->all_done = all;
    st->any_check = 0;
    st->no_check = 1;
  }
}
// a block of R0 columns laid out again as R1 columns: column q of the new
// block is column map[q] of the old one (map[q] < 0: a new, zero column)
__global__ void k_relayout(long long n, int R0, int R1, const int *map, const double *in, double *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * R1) return;
  const long long r = row_of(idx, R1);
  const int q = col_of(idx, r, R1);
  const int o = map[q];
  out[idx] = o >= 0 ? in[r * R0 + o] : 0.0;
}

// Tt = B - Q (all columns)
__global__ void k_sub_mr(long long cnt, const double *B, const double *Q, double *Tt) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < cnt) Tt[idx] = B[idx] - Q[idx];
}

// gather/scatter between caller layout (column-major, original order, ld) and
// the batch layout (row-major, device order); optional row scaling
__global__ void k_batch_in(int n, int R, const int *perm, const double *in, long long ld,
                           double *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * R) return;
  const long long g = row_of(idx, R);
  const int q = col_of(idx, g, R);
  out[idx] = in[q * ld + perm[g]];
}
__global__ void k_batch_out(int n, int R, const int *perm, const double *in, double *out,
                            long long ld) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * R) return;
  const long long g = row_of(idx, R);
  const int q = col_of(idx, g, R);
  out[q * ld + perm[g]] = in[idx];
}
// Binary64 <-> binary32 conversions written out on the bit patterns (IEEE 754:
// rounding to nearest, ties to even, for results in the normal binary32 range;
// widening is exact), in integer instructions.  On this part the hardware
// conversions issue to the FP64 pipe, which the scaling multiply already
// occupies; the streaming cast kernels were bound by that pipe.  Zeros,
// subnormal results, overflow, infinities and NaNs take the hardware
// conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = unsigned(b >> 32);
  const unsigned e = (hi >> 20) & 0x7ffu;            // binary64 biased exponent
  if (e >= 897u && e <= 1150u) {                      // binary32 biased exponent e - 896 in [1, 254]
    const unsigned long long m = b & 0x000fffffffffffffull;
    unsigned f = ((e - 896u) << 23) | unsigned(m >> 29);
    const unsigned rest = unsigned(m & 0x1fffffffull);   // the 29 bits dropped
    if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) f += 1u;   // a carry moves to the exponent
    return __uint_as_float(f | (hi & 0x80000000u));
  }
  return __double2float_rn(x);
}
__device__ __forceinline__ double f32_to_f64(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e != 0u && e != 255u) {
    const unsigned long long b = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                                 (static_cast<unsigned long long>(e + 896u) << 52) |
                                 (static_cast<unsigned long long>(u & 0x7fffffu) << 29);
    return __longlong_as_double(static_cast<long long>(b));
  }
  return double(v);
}
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ void from_f64(double x, float &o) { o = f64_to_f32_rn(x); }
__device__ __forceinline__ void from_f64(double x, double &o) { o = x; }

// tests: out[i] = the bit-pattern conversions of in[i] (dir 0: binary64 ->
// binary32 -> stored widened; dir 1: the binary32 reading of the low word
// widened), compared with the hardware conversions by the caller
__global__ void k_cvt_check(long long n, const double *in, double *out, int dir) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (dir == 0) {
    const float f = f64_to_f32_rn(in[i]);
    const float h = __double2float_rn(in[i]);
    out[i] = __float_as_uint(f) == __float_as_uint(h) ? 0.0 : 1.0;
  } else {
    const float v = __uint_as_float(unsigned(__double_as_longlong(in[i])));
    const double a = f32_to_f64(v), h = double(v);
    out[i] = (__double_as_longlong(a) == __double_as_longlong(h)) || (v != v && a != a) ? 0.0 : 1.0;
  }
}

// out = TO(in * d_row) (d == nullptr: no scaling): the diagonal scaling of the
// scaled system and the change of precision of the preconditioner in one pass.
// A thread takes four consecutive elements (one row index computed for them,
// the next by increment); launch with ceil(n R / 4) threads.
template <typename TO, typename TI>
__global__ void k_scale_cast_mr(long long n, int R, const double *d, const TI *in, TO *out, const int *gate) {
  if (gate && *gate) return;
  const long long nR = n * R;
  const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= nR) return;
  TI v[4];
#pragma unroll
  for (int u = 0; u < 4; u++) v[u] = i0 + u < nR ? in[i0 + u] : TI(0);
  long long r = d ? row_of(i0, R) : 0;
  int q = d ? col_of(i0, r, R) : 0;
#pragma unroll
  for (int u = 0; u < 4; u++) {
    if (i0 + u >= nR) break;
    double x = to_f64(v[u]);
    if (d) {
      x *= d[r];
      if (++q == R) { q = 0; r++; }
    }
    from_f64(x, out[i0 + u]);
  }
}

__global__ void k_scale_rows_mr(long long n, int R, const double *d, const double *in,
                                double *out, const int *gate) {
  if (gate && *gate) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * R) out[idx] = in[idx] * d[row_of(idx, R)];
}

}  // namespace ddlr
