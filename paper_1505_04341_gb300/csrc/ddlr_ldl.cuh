// ddlr_ldl.cuh -- L D L^T local factors for symmetric indefinite blocks
// (factor 2: incomplete on the block pattern, factor 3: on the symbolic fill
// pattern; Sec. 5 names "incomplete Cholesky or LDL" as the local solver).
//
// Storage is that of the Cholesky factors: CSR in device order, columns
// ascending, the diagonal slot last, but L has a unit diagonal and the slot
// holds d_i.  The solve layouts are unchanged (k_solve_layout then stores
// 1 / d_i as the inverse diagonal).  The Cholesky sweeps scale both the
// forward and the backward row by the same inverse diagonal, which no real
// factor of an indefinite L D L^T allows, so these factors have their own
// level sweeps: forward z = L^-1 x, backward z = L^-T (D^-1 z).
#pragma once
#include "ddlr_kernels.cuh"

namespace ddlr {

constexpr int kChunkThreads = 256;   // rows of a level chunk (the plan's kChunk)

// One dependency level of the up-looking incomplete L D L^T (rows of one
// level read only rows of lower levels, as for k_ic_level):
//   l_ij = (a_ij - sum_{t in P_i, P_j, t < j} l_it d_t l_jt) / d_j,
//   d_i  = a_ii - sum_t l_it^2 d_t.
// No pivoting: a zero or non-finite pivot sets *err = 1 (BREAKDOWN).
__global__ void k_ildl_level(int cnt, const int *rows, const int *f_rp, const int *f_ci, double *fval, int *err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int i = rows[t];
  const int b = f_rp[i], e = f_rp[i + 1];
  for (int q = b; q < e - 1; q++) {
    const int j = f_ci[q];
    double s = fval[q];
    int qa = b, qb = f_rp[j];
    const int eb = f_rp[j + 1] - 1;
    while (qa < q && qb < eb) {
      const int ca = f_ci[qa], cb = f_ci[qb];
      if (ca == cb) {
        s -= fval[qa] * fval[f_rp[ca + 1] - 1] * fval[qb];
        qa++;
        qb++;
      } else if (ca < cb) {
        qa++;
      } else {
        qb++;
      }
    }
    fval[q] = s / fval[eb];
  }
  double d = fval[e - 1];
  for (int q = b; q < e - 1; q++) d -= fval[q] * fval[q] * fval[f_rp[f_ci[q] + 1] - 1];
  if (!(d != 0.0) || !isfinite(d)) {
    *err = 1;
    d = 1.0;
  }
  fval[e - 1] = d;
}

// One dependency level of every block (CTA q = chunk q, a thread per row, as
// the chunk tables of the Cholesky sweeps): forward (fwd 1)
// z_r = x_r - sum_c L_rc z_c; backward z_r = z_r / d_r - sum_c L_cr z_c
// (dinv = 1 / d).  Padding slots carry 0 and point at final rows.
template <typename T>
__global__ void __launch_bounds__(kChunkThreads)
k_ldl_sweep(SolveLayout S, const int4 *chunks, int fwd, const T *lval, const T *uval, const T *dinv, const T *x,
            T *z, const int *gate) {
  if (gate && *gate) return;
  const int4 ch = chunks[blockIdx.x];
  const int t = threadIdx.x;
  if (t >= ch.z) return;
  const int i = ch.y + t;
  const int r = S.lvl_row0[ch.x] + i, sl = S.lvl_slice0[ch.x] + (i >> 5), ln = i & 31;
  const int off = (fwd ? S.l_soff : S.u_soff)[sl] + ln, w = (fwd ? S.l_sw : S.u_sw)[sl];
  const int *col = fwd ? S.l_col : S.u_col;
  const T *val = fwd ? lval : uval;
  T acc = fwd ? x[r] : z[r] * dinv[r];
  for (int kk = 0; kk < w; kk++) acc -= val[off + kk * 32] * z[col[off + kk * 32]];
  z[r] = acc;
}

}  // namespace ddlr
