// ddlr_mr.cuh -- the solve with C_a by an approximate inverse X ~ C_a^-1
// built with self-preconditioned global MR iterations and dual-threshold
// dropping (Sec. 4.3, Algorithm 2), for c_solver 2:
//   X_0 = diag(C_a)^-1; per iteration, column by column,
//   r_j = e_j - C_a x_j,  z_j = X r_j,  drop in z_j,  w_j = C_a z_j;
//   beta = sum_j r_j . w_j / sum_j ||w_j||^2;  x_j += beta z_j.
// Dropping in z_j: entries with |z_ij| <= droptol ||z_j||_2 go, then the
// lfil largest in magnitude stay (ties: lower row first).  The solve applies
// the symmetric part (X + X^T)/2 as a row-wise sparse product.
//
// One thread per column.  X columns are kept sorted by row with a fixed
// capacity (1 + iterations * lfil <= kMrCap).  r_j is formed from at most
// kMrCand candidates sorted by row (insertion sort, stable); z_j = sum_l r_lj
// x_l is a k-way merge of the sorted columns x_l by a binary heap keyed by
// (row, list), run twice (norm, then selection) so no list of z_j is stored.
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

constexpr int kMrCap = 32;     // entries per column of X
constexpr int kMrCand = 256;   // candidates of r_j (and of w_j)

// stable insertion sort of (key, val) by key, then sum equal keys; returns
// the number of distinct keys
__device__ __forceinline__ int mr_sort_combine(int cnt, int *key, double *val) {
  for (int a = 1; a < cnt; a++) {
    const int k = key[a];
    const double v = val[a];
    int b = a - 1;
    while (b >= 0 && key[b] > k) { key[b + 1] = key[b]; val[b + 1] = val[b]; b--; }
    key[b + 1] = k;
    val[b + 1] = v;
  }
  int u = 0;
  for (int a = 0; a < cnt; a++) {
    if (u > 0 && key[u - 1] == key[a]) val[u - 1] += val[a];
    else { key[u] = key[a]; val[u] = val[a]; u++; }
  }
  return u;
}

struct MrX {             // columns of X: count, rows ascending, values
  int *cnt, *row;
  double *val;
};

// k-way merge of columns x_l (l = rk[0..nr)) weighted by rv: calls emit(row,
// value) once per distinct row, rows ascending, each value summed over the
// lists in ascending list order
template <typename Emit>
__device__ __forceinline__ void mr_merge(const MrX X, int nr, const int *rk, const double *rv, int *hk, int *hl,
                                         int *hp, Emit emit) {
  int hn = 0;
  auto less = [&](int a, int b) { return hk[a] < hk[b] || (hk[a] == hk[b] && hl[a] < hl[b]); };
  auto swap_ = [&](int a, int b) {
    int t = hk[a]; hk[a] = hk[b]; hk[b] = t;
    t = hl[a]; hl[a] = hl[b]; hl[b] = t;
    t = hp[a]; hp[a] = hp[b]; hp[b] = t;
  };
  auto push = [&](int key, int list, int pos) {
    int c = hn++;
    hk[c] = key; hl[c] = list; hp[c] = pos;
    while (c > 0) {
      const int par = (c - 1) >> 1;
      if (!less(c, par)) break;
      swap_(c, par);
      c = par;
    }
  };
  auto pop = [&]() {
    hn--;
    if (hn > 0) {
      hk[0] = hk[hn]; hl[0] = hl[hn]; hp[0] = hp[hn];
      int c = 0;
      while (true) {
        const int a = 2 * c + 1, b = a + 1;
        int m = c;
        if (a < hn && less(a, m)) m = a;
        if (b < hn && less(b, m)) m = b;
        if (m == c) break;
        swap_(c, m);
        c = m;
      }
    }
  };
  for (int t = 0; t < nr; t++) {
    const int l = rk[t];
    if (rv[t] != 0.0 && X.cnt[l] > 0) push(X.row[(long long)l * kMrCap], t, 0);
  }
  int cur = -1;
  double acc = 0.0;
  while (hn > 0) {
    const int key = hk[0], t = hl[0], pos = hp[0];
    const int l = rk[t];
    const double v = X.val[(long long)l * kMrCap + pos] * rv[t];
    if (key != cur) {
      if (cur >= 0) emit(cur, acc);
      cur = key;
      acc = v;
    } else {
      acc += v;
    }
    pop();
    if (pos + 1 < X.cnt[l]) push(X.row[(long long)l * kMrCap + pos + 1], t, pos + 1);
  }
  if (cur >= 0) emit(cur, acc);
}

// X_0 = diag(C_a)^-1
__global__ void k_mr_init(int s, const int *cc_diag, const double *cc, MrX X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  X.cnt[j] = 1;
  X.row[(long long)j * kMrCap] = j;
  X.val[(long long)j * kMrCap] = 1.0 / cc[cc_diag[j]];
}

// one MR iteration's column work: z_j (dropped, rows ascending) and the
// trace / norm terms num_j = r_j . w_j, den_j = ||w_j||^2 with w_j = C_a z_j
__global__ void __launch_bounds__(128)
k_mr_column(int s, const int *rp, const int *ci, const double *cv, const MrX X, int lfil, double droptol,
            int *zcnt, int *zrow, double *zval, double *num, double *den) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  int rk[kMrCand], hk[kMrCand], hl[kMrCand], hp[kMrCand];
  double rv[kMrCand];
  // r_j = e_j - C_a x_j (C_a symmetric: column i = row i)
  int nc = 0;
  for (int t = 0; t < X.cnt[j]; t++) {
    const int i = X.row[(long long)j * kMrCap + t];
    const double xv = X.val[(long long)j * kMrCap + t];
    for (int q = rp[i]; q < rp[i + 1]; q++) { rk[nc] = ci[q]; rv[nc] = -cv[q] * xv; nc++; }
  }
  rk[nc] = j;
  rv[nc] = 1.0;
  nc++;
  const int nr = mr_sort_combine(nc, rk, rv);
  // pass 1: ||z_j||^2
  double nz2 = 0.0;
  mr_merge(X, nr, rk, rv, hk, hl, hp, [&](int, double v) { nz2 += v * v; });
  const double thr = droptol * sqrt(nz2);
  // pass 2: the lfil largest |z_ij| above the threshold (ties: lower row)
  int sk[kMrCap] = {0};
  double sv[kMrCap] = {0.0};
  int ns = 0;
  mr_merge(X, nr, rk, rv, hk, hl, hp, [&](int row, double v) {
    if (v == 0.0 || !(fabs(v) > thr)) return;
    const double a = fabs(v);
    if (ns == lfil && !(a > fabs(sv[ns - 1]))) return;   // rows arrive ascending: equal loses
    int b = ns < lfil ? ns++ : lfil - 1;
    while (b > 0 && fabs(sv[b - 1]) < a) { sk[b] = sk[b - 1]; sv[b] = sv[b - 1]; b--; }
    sk[b] = row;
    sv[b] = v;
  });
  // kept entries by row
  for (int a = 1; a < ns; a++) {
    const int k = sk[a];
    const double v = sv[a];
    int b = a - 1;
    while (b >= 0 && sk[b] > k) { sk[b + 1] = sk[b]; sv[b + 1] = sv[b]; b--; }
    sk[b + 1] = k;
    sv[b + 1] = v;
  }
  zcnt[j] = ns;
  for (int a = 0; a < ns; a++) { zrow[(long long)j * kMrCap + a] = sk[a]; zval[(long long)j * kMrCap + a] = sv[a]; }
  // w_j = C_a z_j (keys in the heap's key array, reused), then the two terms
  double wv[kMrCand];
  int nw = 0;
  for (int a = 0; a < ns; a++)
    for (int q = rp[sk[a]]; q < rp[sk[a] + 1]; q++) { hk[nw] = ci[q]; wv[nw] = cv[q] * sv[a]; nw++; }
  const int nwu = mr_sort_combine(nw, hk, wv);
  double sn = 0.0, sd = 0.0;
  int a = 0;
  for (int b = 0; b < nwu; b++) {
    sd += wv[b] * wv[b];
    while (a < nr && rk[a] < hk[b]) a++;
    if (a < nr && rk[a] == hk[b]) sn += rv[a] * wv[b];
  }
  num[j] = sn;
  den[j] = sd;
}

// beta = sum num / sum den (fixed order, one CTA of 256); beta = 0 when the
// denominator vanishes (R = 0 after dropping: X is final)
__global__ void k_mr_beta(int s, const double *num, const double *den, double *beta) {
  __shared__ double sm[8];
  double a = 0, b = 0;
  for (int j = threadIdx.x; j < s; j += 256) { a += num[j]; b += den[j]; }
  a = block_sum<double, 256>(a, sm);
  b = block_sum<double, 256>(b, sm);
  if (threadIdx.x == 0) *beta = (b > 0.0) ? a / b : 0.0;
}

// x_j += beta z_j (merge of two row-sorted lists)
__global__ void k_mr_update(int s, MrX X, const int *zcnt, const int *zrow, const double *zval, const double *beta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  const double bt = *beta;
  if (bt == 0.0) return;
  int rr[kMrCap];
  double vv[kMrCap];
  const long long o = (long long)j * kMrCap;
  const int na = X.cnt[j], nb = zcnt[j];
  int a = 0, b = 0, t = 0;
  while ((a < na || b < nb) && t < kMrCap) {
    if (b >= nb || (a < na && X.row[o + a] < zrow[o + b])) { rr[t] = X.row[o + a]; vv[t] = X.val[o + a]; a++; }
    else if (a >= na || zrow[o + b] < X.row[o + a]) { rr[t] = zrow[o + b]; vv[t] = bt * zval[o + b]; b++; }
    else { rr[t] = X.row[o + a]; vv[t] = X.val[o + a] + bt * zval[o + b]; a++; b++; }
    t++;
  }
  X.cnt[j] = t;
  for (int q = 0; q < t; q++) { X.row[o + q] = rr[q]; X.val[o + q] = vv[q]; }
}

// symmetric part (X + X^T)/2 as row CSR: count, (scan), fill, sort + combine
__global__ void k_mr_sym_count(int s, const MrX X, int *rcnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  for (int t = 0; t < X.cnt[j]; t++) {
    const int i = X.row[(long long)j * kMrCap + t];
    atomicAdd(&rcnt[i], 1);     // entry (i, j)
    atomicAdd(&rcnt[j], 1);     // mirrored entry (j, i)
  }
}

// exclusive scan of cnt[0..s) into ptr[0..s] by one CTA of 1024 threads
__global__ void k_mr_scan(int s, const int *cnt, int *ptr) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const long long chunk = (s + 1023) / 1024;
  const long long a = (long long)t * chunk, b = min((long long)s, a + chunk);
  int sum = 0;
  for (long long i = a; i < b; i++) sum += cnt[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int q = 0; q < 1024; q++) { const int v = part[q]; part[q] = run; run += v; }
    ptr[s] = run;
  }
  __syncthreads();
  int run = part[t];
  for (long long i = a; i < b; i++) { ptr[i] = run; run += cnt[i]; }
}

__global__ void k_mr_sym_fill(int s, const MrX X, const int *ptr, int *cursor, int *col, double *val) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  for (int t = 0; t < X.cnt[j]; t++) {
    const int i = X.row[(long long)j * kMrCap + t];
    const double v = 0.5 * X.val[(long long)j * kMrCap + t];
    int e = ptr[i] + atomicAdd(&cursor[i], 1);
    col[e] = j;
    val[e] = v;
    e = ptr[j] + atomicAdd(&cursor[j], 1);
    col[e] = i;
    val[e] = v;
  }
}

// row r: sort by column and combine the (at most two) entries per column;
// ucnt[r] = distinct entries, kept at the front of the row
__global__ void k_mr_sym_sort(int s, const int *ptr, int *col, double *val, int *ucnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const int b = ptr[r], n = ptr[r + 1] - b;
  for (int a = 1; a < n; a++) {
    const int k = col[b + a];
    const double v = val[b + a];
    int q = a - 1;
    // equal columns ordered by value so the pair is summed in one order
    while (q >= 0 && (col[b + q] > k || (col[b + q] == k && val[b + q] > v))) {
      col[b + q + 1] = col[b + q];
      val[b + q + 1] = val[b + q];
      q--;
    }
    col[b + q + 1] = k;
    val[b + q + 1] = v;
  }
  int u = 0;
  for (int a = 0; a < n; a++) {
    if (u > 0 && col[b + u - 1] == col[b + a]) val[b + u - 1] += val[b + a];
    else { col[b + u] = col[b + a]; val[b + u] = val[b + a]; u++; }
  }
  ucnt[r] = u;
}

// z_C = Xs x_C on the interface rows (rows: ptr / ucnt), R columns row-major
template <typename T>
__global__ void k_mr_apply(int s, int m, int R, const int *ptr, const int *ucnt, const int *col, const T *val,
                           const T *x, T *z, const int *gate) {
  if (gate && *gate) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)s * R) return;
  const int i = R == 1 ? int(e) : int(unsigned(e) / unsigned(R)), q = int(e - (long long)i * R);
  T acc = 0;
  const int b = ptr[i];
  for (int t = 0; t < ucnt[i]; t++) acc += val[b + t] * x[(long long)(m + col[b + t]) * R + q];
  z[(long long)(m + i) * R + q] = acc;
}

}  // namespace ddlr
