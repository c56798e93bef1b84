// ddlr_persist.cuh -- persistent cooperative kernels: a whole PCG solve
// (Sec. 5) and the whole Lanczos process (Sec. 4.4) in one launch each.
//
// On the shallow factors of multicolour orders every phase of a PCG iteration
// or of a Lanczos step touches a few hundred thousand rows once; launched as
// separate kernels, the dependent launch gaps cost more than the work.  Here
// one CTA per SM stays resident for the whole solve and the phases are
// separated by a grid-wide barrier.  Scalars (alpha, beta, the convergence
// and breakdown decisions) are reduced by every CTA from the same per-CTA
// partials in the same fixed order, so all CTAs take the same branch without
// a broadcast.  Elementwise work runs on a contiguous row range per CTA
// (a multiple of 32 rows, one SELL slice per warp); the level solves walk the
// level-order row descriptors of all blocks as the level-by-level kernels do.
#pragma once
#include "ddlr_kernels.cuh"
#include "ddlr_plan.h"

namespace ddlr {

// threads per CTA of the persistent kernels (one CTA per SM): their phases are
// gathers and streaming passes bound by load latency, so they run with 32
// warps per SM (64 registers per thread)
constexpr int kPzThreads = 1024;
constexpr int kPzLzThreads = kPzThreads;
constexpr int kPzMaxLevels = 8;          // deepest factor served (levels per block)


// loads of operator data, which no kernel writes while a persistent kernel
// runs: through the read-only path, so they can stay in L1 across barriers
template <typename T>
__device__ __forceinline__ T ro(const T *p) { return __ldg(p); }

// arrival counter of the grid barrier (zeroed before each launch) and the
// shared timeout flag
struct GridSync {
  unsigned *count;
  int *err;
  unsigned long long wait_ns;   // wait limit of one barrier (the handle's wait_limit_s)
  int unmet;                    // tests: the first barrier waits for one arrival that
                                // never comes, so it runs out after wait_ns
};

__device__ __forceinline__ unsigned pz_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long pz_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch (every CTA resident).  The counter only
// grows: barrier number e is passed once e * gridDim.x arrivals are visible
// (release add on arrival, acquire loads while waiting).
// Thread 0 waits at most g.wait_ns, or until another CTA has reported a
// timeout; then the flag is set and every thread gets false (the kernel
// returns).  Writes before the barrier are visible to every CTA after it.
__device__ __forceinline__ bool pz_sync(const GridSync &g, unsigned &epoch) {
  __shared__ int s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    const unsigned target = epoch * gridDim.x + ((g.unmet && epoch == 1) ? 1u : 0u);
    // release: the CTA's writes (ordered before by the CTA barrier) become
    // visible to every CTA whose acquire load sees this arrival
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(g.count) : "memory");
    int ok = 1;
    unsigned long long t0 = 0;
    unsigned it = 0;
    while (pz_ld_acquire(g.count) < target) {
      if ((++it & 63u) == 0) {
        if (*(volatile int *)g.err) { ok = 0; break; }
        const unsigned long long t = pz_clock_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > g.wait_ns) {
          atomicExch(g.err, 1);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Operator data of the preconditioner in device order: local factors, E and
// the low-rank data in precision T (U_k in TU), A and the scaling in FP64.
template <typename T, typename TU>
struct PzOp {
  int n, m, s, k, variant, nL, pstride;
  double a, ia;
  int lvl_ptr[kPzMaxLevels + 1];       // level-order descriptor offsets, levels of all blocks
  const int4 *desc;                    // {row, first L slot, first L^T slot, counts} per row
  const int *l_col, *u_col;            // sliced-ELL columns of L and L^T
  const T *lval, *uval, *dinv;
  const int *eh_rp, *eh_ci;
  const T *eh;
  const int *eht_rp, *eht_ci;
  const T *eht;
  const TU *U;
  const T *coef, *inv1mt, *Hk;
  const int *a_soff, *a_sw, *a_col;
  const double *a_val;
  const double *dsc;                   // D^-1/2 (scaled systems) or null
  const unsigned char *lvl0;           // 1 for rows on the first level of their block
  int fuse0;                           // >= 2 levels: the producer of a solve's input
                                       // also does its first forward level
  double *part;                        // 3 x gridDim.x x pstride partial sums
  GridSync gs;
};

// x_r as the preconditioner reads it: (xsc_r x_r) rounded to T
template <typename T, typename TX>
__device__ __forceinline__ T pz_in(const TX *x, const double *xsc, int r) {
  return xsc ? T(double(x[r]) * ro(xsc + r)) : T(x[r]);
}

// The first forward level of z = A0^-1 x for row r, done by the phase that
// produces x_r (xv = x_r as read): rows on the first level of their block
// have no lower neighbours, so z_r = x_r / L_rr, exactly what the level solve
// computes for them.
template <typename T, typename TU>
__device__ __forceinline__ void pz_l0(const PzOp<T, TU> &O, int r, T xv, T *z) {
  if (O.fuse0 && ro(O.lvl0 + r)) z[r] = xv * ro(O.dinv + r);
}

// this CTA's rows [r0, r1) of a vector of N rows
__device__ __forceinline__ void pz_range(int N, int &r0, int &r1) {
  const int per = (((N + (int)gridDim.x - 1) / (int)gridDim.x) + 31) & ~31;
  r0 = min(N, (int)blockIdx.x * per);
  r1 = min(N, r0 + per);
}

template <typename T, typename TU>
__device__ __forceinline__ double *pz_buf(const PzOp<T, TU> &O, int slot) {
  return O.part + (size_t)(slot % 3) * gridDim.x * O.pstride;
}

// CTA sum of v written to pt[blockIdx.x * pstride] (sm: NT/32 doubles)
template <int NT>
__device__ __forceinline__ void pz_put(double v, double *pt, int pstride, double *sm) {
  v = block_sum<double, NT>(v, sm);
  if (threadIdx.x == 0) pt[(size_t)blockIdx.x * pstride] = v;
}

// sum over CTAs of pt[g * pstride] in a fixed order, returned to every thread
__device__ __forceinline__ double pz_get(const double *pt, int pstride, double *bc) {
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    double s = 0;
    for (int g = l; g < (int)gridDim.x; g += 32) s += pt[(size_t)g * pstride];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) bc[0] = s;
  }
  __syncthreads();
  const double r = bc[0];
  __syncthreads();
  return r;
}

// out[c] = (coef ? coef[c] : 1) * sum_g pt[g * pstride + c], c < ncol, in
// precision T in shared memory; with H (ncol x ncol row-major): out = H *
// (those sums)
template <int NT, typename T>
__device__ __forceinline__ void pz_get_cols(const double *pt, int pstride, int ncol, const T *coef, const T *H,
                                            T *out, T *tmp) {
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  T *dst = H ? tmp : out;
  for (int c = wi; c < ncol; c += NT / 32) {
    T s = 0;
    for (int g = l; g < (int)gridDim.x; g += 32) s += T(pt[(size_t)g * pstride + c]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) dst[c] = coef ? ro(coef + c) * s : s;
  }
  __syncthreads();
  if (H) {
    for (int c = threadIdx.x; c < ncol; c += NT) {
      T s = 0;
      for (int b = 0; b < ncol; b++) s += ro(H + c * ncol + b) * tmp[b];
      out[c] = s;
    }
    __syncthreads();
  }
}

// this CTA's partials pt[blockIdx.x * pstride + c] = sum_{r in [r0,r1)} U[r][c] x_r
// in precision T (U row-major, k columns, x read as pz_in); red: NT doubles
template <int NT, typename T, typename TU, typename TX>
__device__ __forceinline__ void pz_utx(int k, const TU *U, const TX *x, const double *xsc, int r0, int r1,
                                       double *pt, int pstride, double *red) {
  const int G = NT / k;
  const int c = threadIdx.x % k, g = threadIdx.x / k;
  T acc = 0;
  if (g < G)
    for (int r = r0 + g; r < r1; r += G) acc += T(to_acc(ro(U + (size_t)r * k + c))) * pz_in<T>(x, xsc, r);
  T *rt = reinterpret_cast<T *>(red);
  rt[threadIdx.x] = (g < G) ? acc : T(0);
  __syncthreads();
  if (threadIdx.x < k) {
    T s = 0;
    for (int gg = 0; gg < G; gg++) s += rt[gg * k + threadIdx.x];
    pt[(size_t)blockIdx.x * pstride + threadIdx.x] = double(s);
  }
  __syncthreads();
}

// One level L of every block: mode 0 forward, 1 backward, 2 forward then
// backward (the top level).  x is read as pz_in.  Rows finalised here (modes
// 1, 2) add racc_r (zsc_r z_r) to acc when racc is given; z2 (level 0,
// backward) receives the first forward level of a solve whose input is z.
template <int NT, typename T, typename TU, typename TX>
__device__ __forceinline__ void pz_level(const PzOp<T, TU> &O, int L, int mode, const TX *x, const double *xsc,
                                         T *z, const double *racc, const double *zsc, double &acc, T *z2) {
  const int c0 = O.lvl_ptr[L], cnt = O.lvl_ptr[L + 1] - c0;
  for (int v = blockIdx.x * NT + threadIdx.x; v < cnt; v += gridDim.x * NT) {
    const int4 d = ro(O.desc + c0 + v);
    const int r = d.x;
    T zr;
    const T dr = ro(O.dinv + r);
    if (mode == 1) {
      const int off = d.z, w = int(unsigned(d.w) >> 16);
      T t = z[r];
      for (int kk = 0; kk < w; kk++) t -= ro(O.uval + off + kk * 32) * z[ro(O.u_col + off + kk * 32)];
      zr = t * dr;
    } else {
      const int off = d.y, w = int(unsigned(d.w) & 0xffffu);
      T t = pz_in<T>(x, xsc, r);
      for (int kk = 0; kk < w; kk++) t -= ro(O.lval + off + kk * 32) * z[ro(O.l_col + off + kk * 32)];
      zr = t * dr;
      if (mode == 2) zr = zr * dr;
    }
    z[r] = zr;
    if (racc && mode != 0) acc += racc[r] * (zsc ? ro(zsc + r) * double(zr) : double(zr));
    if (z2) z2[r] = zr * dr;          // first forward level of a solve with input z
  }
}

// z = A0^-1 x (Sec. 4.2), x read as pz_in, phases separated by grid barriers;
// the last phase is left open (the caller adds its own work and barrier).
// l0_done: the producer of x has already done the first forward level
// (pz_l0).  z2: see pz_level (only with fuse0).
template <int NT, typename T, typename TU, typename TX>
__device__ __forceinline__ bool pz_a0(const PzOp<T, TU> &O, const TX *x, const double *xsc, T *z,
                                      const double *racc, const double *zsc, double &acc, unsigned &ep,
                                      bool l0_done, T *z2 = nullptr) {
  const int nL = O.nL;
  for (int L = l0_done ? 1 : 0; L + 1 < nL; L++) {
    pz_level<NT>(O, L, 0, x, xsc, z, nullptr, nullptr, acc, (T *)nullptr);
    if (!pz_sync(O.gs, ep)) return false;
  }
  pz_level<NT>(O, nL - 1, 2, x, xsc, z, racc, zsc, acc, (T *)nullptr);
  for (int L = nL - 2; L >= 0; L--) {
    if (!pz_sync(O.gs, ep)) return false;
    pz_level<NT>(O, L, 1, x, xsc, z, racc, zsc, acc, L == 0 ? z2 : (T *)nullptr);
  }
  return true;
}

// u = M^-1 (dsc .* x) in precision T without the final dsc scaling, DDLR-1
// (Algorithm 1, prop. gkt) or DDLR-2 (eq. Form2a); x (FP64) is rounded to T
// as it is read.  acc collects sum_r racc_r (dsc_r u_r) over the rows this CTA
// finalises.  Scratch: z (n), y, w (s), rhs (n).  The last phase is left
// open.  `slot` is the next partial-sum buffer.
template <int NT, typename T, typename TU>
__device__ __forceinline__ bool pz_apply(const PzOp<T, TU> &O, const double *x, T *u, T *z, T *y, T *w, T *rhs,
                                         const double *racc, double &acc, unsigned &ep, int &slot, double *red,
                                         T *vec, bool l0_done) {
  const double *xsc = O.dsc;
  const int n = O.n, m = O.m, s = O.s, k = O.k;
  if (O.variant == 2) {
    int i0, i1;
    pz_range(n, i0, i1);
    double *pt = pz_buf(O, slot++);
    pz_utx<NT, T>(k, O.U, x, xsc, i0, i1, pt, O.pstride, red);     // t = U^T x, this CTA's rows
    double dummy = 0;
    if (!pz_a0<NT>(O, x, xsc, u, nullptr, nullptr, dummy, ep, l0_done)) return false;
    if (!pz_sync(O.gs, ep)) return false;
    pz_get_cols<NT, T>(pt, O.pstride, k, nullptr, O.Hk, vec, reinterpret_cast<T *>(red));   // H_k t
    for (int r = i0 + threadIdx.x; r < i1; r += NT) {
      T t = 0;
      const TU *row = O.U + (size_t)r * k;
      for (int c = 0; c < k; c++) t += T(to_acc(ro(row + c))) * vec[c];
      const T ur = u[r] + t;
      u[r] = ur;
      if (racc) acc += racc[r] * (O.dsc ? ro(O.dsc + r) * double(ur) : double(ur));
    }
    return true;
  }
  double dummy = 0;
  if (!pz_a0<NT>(O, x, xsc, z, nullptr, nullptr, dummy, ep, l0_done)) return false;
  if (!pz_sync(O.gs, ep)) return false;
  const T a = T(O.a), ia = T(O.ia);
  int j0, j1;
  pz_range(s, j0, j1);
  for (int j = j0 + threadIdx.x; j < j1; j += NT) {                // y = E^T z
    T t = 0;
    const int q1 = ro(O.eht_rp + j + 1);
    for (int q = ro(O.eht_rp + j); q < q1; q++) t += ro(O.eht + q) * z[ro(O.eht_ci + q)];
    y[j] = ia * t - a * z[m + j];
  }
  __syncthreads();
  double *pt = pz_buf(O, slot++);
  pz_utx<NT, T>(k, O.U, y, (const double *)nullptr, j0, j1, pt, O.pstride, red);   // D U^T y, this CTA's rows
  if (!pz_sync(O.gs, ep)) return false;
  pz_get_cols<NT, T>(pt, O.pstride, k, O.coef, (const T *)nullptr, vec, reinterpret_cast<T *>(red));
  const T i1mt = ro(O.inv1mt);
  for (int j = j0 + threadIdx.x; j < j1; j += NT) {                // w = G^-1 y; x_C - a w
    T t = 0;
    const TU *row = O.U + (size_t)j * k;
    for (int c = 0; c < k; c++) t += T(to_acc(ro(row + c))) * vec[c];
    const T wj = i1mt * y[j] + t;
    w[j] = wj;
    const T rv = pz_in<T>(x, xsc, m + j) - a * wj;
    rhs[m + j] = rv;
    pz_l0(O, m + j, rv, u);
  }
  if (!pz_sync(O.gs, ep)) return false;
  int i0, i1;
  pz_range(m, i0, i1);
  for (int i = i0 + threadIdx.x; i < i1; i += NT) {                // x_B + a^-1 Ehat w
    T t = 0;
    const int q1 = ro(O.eh_rp + i + 1);
    for (int q = ro(O.eh_rp + i); q < q1; q++) t += ro(O.eh + q) * w[ro(O.eh_ci + q)];
    const T rv = pz_in<T>(x, xsc, i) + ia * t;
    rhs[i] = rv;
    pz_l0(O, i, rv, u);
  }
  if (!pz_sync(O.gs, ep)) return false;
  return pz_a0<NT>(O, rhs, (const double *)nullptr, u, racc, O.dsc, acc, ep, O.fuse0 != 0);
}

// ------------------------------------------------------------------- PCG
template <typename T>
struct PzPcg {
  const double *b;
  double *x, *r, *p0, *p1, *q, *t, *zo;
  T *u, *z, *y, *w, *rhs;
  PcgState *st;
  double tol;
  int maxit;
};

// z_i of the preconditioned residual: u_i in FP64, scaled back on scaled
// systems
template <typename T, typename TU>
__device__ __forceinline__ double pz_zval(const PzOp<T, TU> &O, const T *u, int i) {
  return O.dsc ? ro(O.dsc + i) * double(u[i]) : double(u[i]);
}

// PCG from x0 = 0 (Sec. 5) with the stopping rule, true-residual confirmation
// and restart of the level-by-level path; the final state goes to P.st.  With
// an FP32 preconditioner (T = float) the outer loop is flexible CG in FP64:
// beta = (r_new.z_new - r_new.z_old) / r.z.
template <int NT, typename T, typename TU>
__global__ void __launch_bounds__(NT, 1) k_pcg_persist(PzOp<T, TU> O, PzPcg<T> P) {
  constexpr bool kFlex = sizeof(T) < sizeof(double);
  extern __shared__ double pz_sm[];
  double *red = pz_sm, *bc = pz_sm + NT;
  T *vec = reinterpret_cast<T *>(pz_sm + NT + 32);
  unsigned ep = 0;
  int slot = 0;
  const int n = O.n;
  int i0, i1;
  pz_range(n, i0, i1);
  // the first A0 solve of the preconditioner writes here (its first level
  // is done by whoever produces r)
  T *a0out = O.variant == 2 ? P.u : P.z;
  double acc = 0;
  for (int i = i0 + threadIdx.x; i < i1; i += NT) {
    const double bi = P.b[i];
    P.x[i] = 0.0;
    P.r[i] = bi;
    P.p0[i] = 0.0;
    acc += bi * bi;
    pz_l0(O, i, pz_in<T>(P.b, O.dsc, i), a0out);
  }
  double *pt = pz_buf(O, slot++);
  pz_put<NT>(acc, pt, O.pstride, red);
  if (!pz_sync(O.gs, ep)) return;
  const double bb = pz_get(pt, O.pstride, bc);
  const double tol2 = P.tol * P.tol * bb;
  int its = 0, status = 0;
  bool done = (bb == 0.0);
  double rz = 0, beta = 0, rr = bb, rt2 = 0, pq = 0, alpha = 0, rzo = 0;
  if (!done) {
    acc = 0;
    if (!pz_apply<NT>(O, P.r, P.u, P.z, P.y, P.w, P.rhs, P.r, acc, ep, slot, red, vec, O.fuse0 != 0)) return;
    pt = pz_buf(O, slot++);
    pz_put<NT>(acc, pt, O.pstride, red);
    if (!pz_sync(O.gs, ep)) return;
    rz = pz_get(pt, O.pstride, bc);
    if (!(rz == rz) || isinf(rz)) { status = 7; done = true; }
  }
  double *pold = P.p0, *pnew = P.p1;
  bool restart = false;
  while (!done) {
    // p = z + beta p_old (into the other buffer), then q = A p, p.q: two
    // phases, since forming p inside the product would double its FP64
    // instructions, the scarce resource of this part
    for (int i = i0 + threadIdx.x; i < i1; i += NT) {
      const double zi = pz_zval(O, P.u, i);
      pnew[i] = fma(beta, pold[i], zi);
      if (kFlex) P.zo[i] = zi;
    }
    if (!pz_sync(O.gs, ep)) return;
    acc = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += NT) {
      const int g = i >> 5, l = i & 31;
      const int off = ro(O.a_soff + g) + l, wd = ro(O.a_sw + g);
      double qi = 0;
      for (int kk = 0; kk < wd; kk++) qi += ro(O.a_val + off + kk * 32) * pnew[ro(O.a_col + off + kk * 32)];
      P.q[i] = qi;
      acc += pnew[i] * qi;
    }
    pt = pz_buf(O, slot++);
    pz_put<NT>(acc, pt, O.pstride, red);
    if (!pz_sync(O.gs, ep)) return;
    pq = pz_get(pt, O.pstride, bc);
    alpha = rz / pq;
    if (!(alpha == alpha) || isinf(alpha)) { status = 7; break; }
    // x += alpha p; r -= alpha q; r.r (and r.z_old for flexible CG)
    acc = 0;
    double acc2 = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += NT) {
      P.x[i] += alpha * pnew[i];
      const double ri = P.r[i] - alpha * P.q[i];
      P.r[i] = ri;
      acc += ri * ri;
      if (kFlex) acc2 += ri * P.zo[i];
      pz_l0(O, i, pz_in<T>(P.r, O.dsc, i), a0out);
    }
    pt = pz_buf(O, slot++);
    pz_put<NT>(acc, pt, O.pstride, red);
    if (kFlex) pz_put<NT>(acc2, pt + 1, O.pstride, red);
    if (!pz_sync(O.gs, ep)) return;
    rr = pz_get(pt, O.pstride, bc);
    if (kFlex) rzo = pz_get(pt + 1, O.pstride, bc);
    its += 1;
    if (!(rr == rr) || isinf(rr)) { status = 7; break; }
    if (rr <= tol2) {
      // confirm with the true residual t = b - A x
      acc = 0;
      for (int i = i0 + threadIdx.x; i < i1; i += NT) {
        const int g = i >> 5, l = i & 31;
        const int off = ro(O.a_soff + g) + l, wd = ro(O.a_sw + g);
        double ax = 0;
        for (int kk = 0; kk < wd; kk++) ax += ro(O.a_val + off + kk * 32) * P.x[ro(O.a_col + off + kk * 32)];
        const double tr = P.b[i] - ax;
        P.t[i] = tr;
        acc += tr * tr;
      }
      pt = pz_buf(O, slot++);
      pz_put<NT>(acc, pt, O.pstride, red);
      if (!pz_sync(O.gs, ep)) return;
      rt2 = pz_get(pt, O.pstride, bc);
      if (rt2 <= tol2) { status = 0; done = true; break; }
      restart = true;                       // continue from the true residual
      if (its >= P.maxit) { status = 5; break; }
      for (int i = i0 + threadIdx.x; i < i1; i += NT) {
        P.r[i] = P.t[i];
        pz_l0(O, i, pz_in<T>(P.t, O.dsc, i), a0out);
      }
      if (!pz_sync(O.gs, ep)) return;
    } else if (its >= P.maxit) {
      status = 5;
      break;
    }
    acc = 0;
    if (!pz_apply<NT>(O, P.r, P.u, P.z, P.y, P.w, P.rhs, P.r, acc, ep, slot, red, vec, O.fuse0 != 0)) return;
    pt = pz_buf(O, slot++);
    pz_put<NT>(acc, pt, O.pstride, red);
    if (!pz_sync(O.gs, ep)) return;
    const double rzn = pz_get(pt, O.pstride, bc);
    beta = restart ? 0.0 : (kFlex ? (rzn - rzo) / rz : rzn / rz);
    rz = rzn;
    restart = false;
    if (!(rzn == rzn) || isinf(rzn)) { status = 7; break; }
    double *tp = pold;
    pold = pnew;
    pnew = tp;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PcgState *st = P.st;
    st->rz = rz; st->pq = pq; st->alpha = alpha; st->beta = beta; st->rr = rr; st->bb = bb;
    st->tol2 = tol2; st->rt2 = rt2; st->its = its; st->maxit = P.maxit; st->done = 1; st->status = status;
    st->check_true = 0; st->restart = 0; st->flexible = kFlex ? 1 : 0;
  }
}

// --------------------------------------------------------------- Lanczos
struct PzLz {
  double *Q;
  long long ld;
  double *al, *be, *w, *qcur, *qprev, *v, *z, *etop;
  const int *rank;
  LzState *st;
  int check, k;
  double eps;
  int reorth2;      // 1: two Gram-Schmidt passes every step
  float *Q32;       // FP32 copy of Q (same layout), for the Gram-Schmidt corrections
};

// Gram-Schmidt counters of one launch (the same in every CTA)
struct LzCount {
  int npass2, nfp32;
  double q64, q32;
};

// partials of Q_{ncol}^T w over this CTA's rows [r0, r1), warp per column
// (red: NT/32 doubles of shared memory).  With fewer columns than warps the
// rows are split into nseg segments per column so every warp works; the
// segment sums are added in a fixed order.
template <int NT>
__device__ __forceinline__ void pz_gemvT(const double *Q, long long ld, int ncol, const double *w, int r0,
                                         int r1, double *pt, int pstride, double *red) {
  constexpr int NW = NT / 32;
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (ncol >= NW) {
    for (int j = wi; j < ncol; j += NW) {
      const double *q = Q + (long long)j * ld;
      double acc = 0;
      for (int r = r0 + l; r < r1; r += 32) acc += ld_stream(q + r) * w[r];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (l == 0) pt[(size_t)blockIdx.x * pstride + j] = acc;
    }
    return;
  }
  const int nseg = NW / ncol, len = (r1 - r0 + nseg - 1) / nseg;
  if (wi < ncol * nseg) {
    const int j = wi / nseg, sg = wi % nseg;
    const int a = r0 + sg * len, b = min(r1, a + len);
    const double *q = Q + (long long)j * ld;
    double acc = 0;
    for (int r = a + l; r < b; r += 32) acc += ld_stream(q + r) * w[r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (l == 0) red[wi] = acc;
  }
  __syncthreads();
  if (threadIdx.x < ncol) {
    double sum = 0;
    for (int sg = 0; sg < nseg; sg++) sum += red[threadIdx.x * nseg + sg];
    pt[(size_t)blockIdx.x * pstride + threadIdx.x] = sum;
  }
  __syncthreads();
}

// w_r -= sum_j Q[j][r] c_j on this CTA's rows; returns this thread's sum of w_r^2
template <int NT>
__device__ __forceinline__ double pz_gemvN(const double *Q, long long ld, int ncol, const double *cs, double *w,
                                           int r0, int r1) {
  double ww = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += NT) {
    double acc = 0;
    for (int j = 0; j < ncol; j++) acc += ld_stream(Q + (long long)j * ld + r) * cs[j];
    const double v = w[r] - acc;
    w[r] = v;
    ww += v * v;
  }
  return ww;
}

// w_r -= sum_j Q32[j][r] c32_j on this CTA's rows, the sum formed in FP32 and
// subtracted from the FP64 w_r; returns this thread's sum of w_r^2
template <int NT>
__device__ __forceinline__ double pz_gemvN32(const float *Q, long long ld, int ncol, const float *cs, double *w,
                                             int r0, int r1) {
  double ww = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += NT) {
    float acc = 0.f;
#pragma unroll 8
    for (int j = 0; j < ncol; j++) acc = fmaf(ld_stream(Q + (long long)j * ld + r), cs[j], acc);
    const double v = w[r] - double(acc);
    w[r] = v;
    ww += v * v;
  }
  return ww;
}

// Whether the correction Q c of a Gram-Schmidt pass may be formed in FP32
// from the FP32 copy of Q and c rounded to FP32.  With u = 2^-24 its error is
// at most (ncol + 2) u sum_j |Q_rj| |c_j| per row, so at most
// (ncol + 2) sqrt(ncol) u ||c|| in norm; FP32 is taken when that bound is
// below the unit roundoff of FP64 times ||w|| (ww0 = ||w||^2 before the pass),
// i.e. when the update is as accurate as w's own rounding.  After the
// three-term recurrence c holds only the rounding-level loss of orthogonality,
// so the test passes on most steps; restart vectors and second passes after
// cancellation keep FP64.  Warp 0 sums c.c in a fixed order from the shared c,
// so every CTA decides alike.  Fills cs32 when it returns true.
template <int NT>
__device__ __forceinline__ bool pz_use32(const double *cs, int ncol, double ww0, float *cs32, double *flag) {
  if (threadIdx.x < 32) {
    double cc = 0;
    for (int i = threadIdx.x; i < ncol; i += 32) cc += cs[i] * cs[i];
    for (int o = 16; o > 0; o >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, o);
    const double f = double(ncol + 2);
    if (threadIdx.x == 0) *flag = (f * f * double(ncol) * cc <= 0x1p-58 * ww0) ? 1.0 : 0.0;
  }
  for (int i = threadIdx.x; i < ncol; i += NT) cs32[i] = float(cs[i]);
  __syncthreads();
  const bool use = *flag != 0.0;
  __syncthreads();
  return use;
}

// Full reorthogonalisation of w against Q_{ncol} (rows [j0, j1) of this CTA):
// one classical Gram-Schmidt pass, and a second one when always2 or when the
// first left less than half of ||w||^2 (the DGKS criterion; every CTA reads
// the same partials in the same order, so all take the same branch).  ww0 is
// this thread's share of ||w||^2 before the first pass.  Returns ||w||^2
// after the last pass to every thread.
// The correction of each pass is formed in FP32 when pz_use32 allows it.
template <int NT>
__device__ __forceinline__ bool pz_cgs(const PzOp<double, double> &O, const PzLz &L, int ncol, int j0, int j1,
                                       unsigned &ep, int &slot, double *red, double *bc, double *cs, float *cs32,
                                       bool always2, double ww0, double &ww_out, LzCount &cnt) {
  double *pt = pz_buf(O, slot++);
  pz_gemvT<NT>(L.Q, L.ld, ncol, L.w, j0, j1, pt, O.pstride, red);
  __syncthreads();
  pz_put<NT>(ww0, pt + ncol, O.pstride, red);       // column ncol: ||w||^2 before
  if (!pz_sync(O.gs, ep)) return false;
  pz_get_cols<NT, double>(pt, O.pstride, ncol + 1, nullptr, nullptr, cs, red);
  const double w0 = cs[ncol];
  auto update = [&](double wbefore) {
    cnt.q64 += ncol;
    if (pz_use32<NT>(cs, ncol, wbefore, cs32, cs + ncol + 1)) {
      cnt.nfp32 += 1;
      cnt.q32 += ncol;
      return pz_gemvN32<NT>(L.Q32, L.ld, ncol, cs32, L.w, j0, j1);
    }
    cnt.q64 += ncol;
    return pz_gemvN<NT>(L.Q, L.ld, ncol, cs, L.w, j0, j1);
  };
  double ww = update(w0);
  pt = pz_buf(O, slot++);
  pz_put<NT>(ww, pt, O.pstride, red);
  if (!pz_sync(O.gs, ep)) return false;
  ww = pz_get(pt, O.pstride, bc);
  if (!always2 && !(ww < 0.5 * w0)) {
    ww_out = ww;
    return true;
  }
  cnt.npass2 += 1;
  const double w1 = ww;
  pt = pz_buf(O, slot++);
  pz_gemvT<NT>(L.Q, L.ld, ncol, L.w, j0, j1, pt, O.pstride, red);
  if (!pz_sync(O.gs, ep)) return false;
  pz_get_cols<NT, double>(pt, O.pstride, ncol, nullptr, nullptr, cs, red);
  ww = update(w1);
  pt = pz_buf(O, slot++);
  pz_put<NT>(ww, pt, O.pstride, red);
  if (!pz_sync(O.gs, ep)) return false;
  ww_out = pz_get(pt, O.pstride, bc);
  return true;
}

// Lanczos with full reorthogonalisation on the operator of DDLR-1 (E^T A0^-1 E)
// or DDLR-2 (E^T A0^-2 E), from the state in L.st (step j, start vector in
// qcur and Q column j) until m_max steps, a NaN, or the convergence test of
// eq. converge every `check` steps (sums of the k largest eigenvalues of T_m
// and T_{m-1}); breakdown restarts as the level-by-level path does them.
// Shared memory: NT + 32 + (m_max + 2) + 2 m_max doubles and m_max + 2 floats.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_lz_persist(PzOp<double, double> O, PzLz L) {
  extern __shared__ double pz_sm[];
  double *red = pz_sm, *bc = pz_sm + NT;
  LzState S0 = *L.st;
  double *cs = pz_sm + NT + 32, *ea = cs + S0.mmax + 2, *eb2 = ea + S0.mmax;
  float *cs32 = reinterpret_cast<float *>(eb2 + S0.mmax);
  unsigned ep = 0;
  int slot = 0;
  const int n = O.n, m = O.m, s = O.s, k = L.k;
  int j = S0.j, restarts = S0.restarts, conv_m = S0.conv_m, nan_step = S0.nan_step;
  LzCount cnt{S0.npass2, S0.nfp32, S0.qcols64, S0.qcols32};
  bool stop = S0.stop != 0;
  double scale = S0.scale;
  const int mmax = S0.mmax;
  int i0, i1, j0, j1;
  pz_range(n, i0, i1);
  pz_range(s, j0, j1);
  // the FP32 copy of the basis so far, this CTA's rows (its only reader)
  for (int c = 0; c <= j; c++)
    for (int r = j0 + threadIdx.x; r < j1; r += NT) L.Q32[(long long)c * L.ld + r] = float(L.Q[(long long)c * L.ld + r]);
  __syncthreads();
  double bprev = j > 0 ? L.be[j - 1] : 0.0;
  double *v = L.v, *z = L.z;
  // v = E q (eq. EF) on this CTA's rows, q = src, or src * rdiv when rdiv != 0
  // (the product that forms the stored q, so E acts on exactly that vector)
  auto evec = [&](const double *src, double rdiv) {
    for (int i = i0 + threadIdx.x; i < i1; i += NT) {
      double t;
      if (i < m) {
        t = 0;
        const int q1 = ro(O.eh_rp + i + 1);
        for (int q = ro(O.eh_rp + i); q < q1; q++) {
          const int c = ro(O.eh_ci + q);
          t += ro(O.eh + q) * (rdiv != 0.0 ? src[c] * rdiv : src[c]);
        }
        t *= O.ia;
      } else {
        t = -O.a * (rdiv != 0.0 ? src[i - m] * rdiv : src[i - m]);
      }
      v[i] = t;
      pz_l0(O, i, t, z);
    }
  };
  bool have_v = false;   // E q_j already formed in the previous step's last phase
  while (!stop) {
    if (!have_v) {
      evec(L.qcur, 0.0);
      if (!pz_sync(O.gs, ep)) return;
    }
    have_v = false;
    double dummy = 0;
    const bool f0 = O.fuse0 != 0;
    // DDLR-2: the first solve's last level also does the second's first
    if (!pz_a0<NT>(O, v, nullptr, z, nullptr, nullptr, dummy, ep, f0, O.variant == 2 && f0 ? v : nullptr)) return;
    if (!pz_sync(O.gs, ep)) return;
    double *res = z;
    if (O.variant == 2) {
      if (!pz_a0<NT>(O, z, nullptr, v, nullptr, nullptr, dummy, ep, f0)) return;
      if (!pz_sync(O.gs, ep)) return;
      res = v;
    }
    // w = E^T res, alpha_j = q_j . w
    double acc = 0;
    for (int r = j0 + threadIdx.x; r < j1; r += NT) {
      double t = 0;
      const int q1 = ro(O.eht_rp + r + 1);
      for (int q = ro(O.eht_rp + r); q < q1; q++) t += ro(O.eht + q) * res[ro(O.eht_ci + q)];
      const double wr = O.ia * t - O.a * res[m + r];
      L.w[r] = wr;
      acc += L.qcur[r] * wr;
    }
    double *pt = pz_buf(O, slot++);
    pz_put<NT>(acc, pt, O.pstride, red);
    if (!pz_sync(O.gs, ep)) return;
    const double alpha = pz_get(pt, O.pstride, bc);
    if (blockIdx.x == 0 && threadIdx.x == 0) L.al[j] = alpha;
    // three-term recurrence, then full reorthogonalisation against Q_{j+1}
    double ww0 = 0;
    for (int r = j0 + threadIdx.x; r < j1; r += NT) {
      double t = L.w[r] - alpha * L.qcur[r];
      if (j > 0) t -= bprev * L.qprev[r];
      L.w[r] = t;
      ww0 += t * t;
    }
    __syncthreads();
    double ww = 0;
    if (!pz_cgs<NT>(O, L, j + 1, j0, j1, ep, slot, red, bc, cs, cs32, L.reorth2 != 0, ww0, ww, cnt)) return;
    const double beta = sqrt(ww);
    if (blockIdx.x == 0 && threadIdx.x == 0) L.be[j] = beta;
    if (!(alpha == alpha) || isinf(alpha) || !(beta == beta) || isinf(beta)) {
      if (nan_step < 0) nan_step = j;
      stop = true;
      break;
    }
    scale = fmax(scale, fabs(alpha));
    const bool brk = beta <= 1e-12 * (scale > 0 ? scale : 1.0);
    // q_{j+1} = w * (1 / beta): one division, then products (an FP64
    // division is about ten FP64 issue slots on this part)
    double rdiv = 1.0 / beta;
    if (!brk) {
      scale = fmax(scale, beta);
      for (int r = j0 + threadIdx.x; r < j1; r += NT) {
        const double q1 = L.w[r] * rdiv;
        L.Q[(long long)(j + 1) * L.ld + r] = q1;
        L.Q32[(long long)(j + 1) * L.ld + r] = float(q1);
        L.qprev[r] = L.qcur[r];
        L.qcur[r] = q1;
      }
      bprev = beta;
    } else {
      // restart from SplitMix64 stream seed + restarts (interface nodes in
      // ascending original index), orthogonalised against Q_{j+1}
      restarts += 1;
      for (int r = j0 + threadIdx.x; r < j1; r += NT)
        L.w[r] = d_sm64_pm1(S0.seed + (unsigned long long)restarts, (unsigned long long)ro(L.rank + r));
      __syncthreads();
      double nn = 0;
      // a restart vector's passes are counted in bytes, not as second passes
      LzCount rc{0, 0, 0.0, 0.0};
      if (!pz_cgs<NT>(O, L, j + 1, j0, j1, ep, slot, red, bc, cs, cs32, true, 0.0, nn, rc)) return;
      cnt.nfp32 += rc.nfp32;
      cnt.q64 += rc.q64;
      cnt.q32 += rc.q32;
      const double nrm = sqrt(nn);
      rdiv = 1.0 / nrm;
      for (int r = j0 + threadIdx.x; r < j1; r += NT) {
        const double q1 = L.w[r] * rdiv;
        L.Q[(long long)(j + 1) * L.ld + r] = q1;
        L.Q32[(long long)(j + 1) * L.ld + r] = float(q1);
        L.qprev[r] = L.qcur[r];
        L.qcur[r] = q1;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) L.be[j] = 0.0;
      bprev = 0.0;
    }
    j += 1;
    if (j >= mmax) stop = true;
    if (!stop) {        // the next step's E q_{j+1}, in the same phase
      evec(L.w, rdiv);
      have_v = true;
    }
    if (!pz_sync(O.gs, ep)) return;
    if (!stop && L.check > 0 && j % L.check == 0 && j >= k + 1 && j < mmax) {
      // eq. converge: k largest eigenvalues of T_j and T_{j-1}; CTA e
      // computes eigenvalue e % k of T_{j - e / k}
      for (int e = blockIdx.x; e < 2 * k; e += gridDim.x) {
        const int mm = j - e / k;
        for (int i = threadIdx.x; i < mm; i += NT) {
          ea[i] = L.al[i];
          eb2[i] = (i + 1 < mm) ? L.be[i] * L.be[i] : 0.0;
        }
        __syncthreads();
        const double ev = tridiag_eig_cta<kEigPoints, kEigRounds>(mm, ea, eb2, L.be, e % k, bc);
        if (threadIdx.x == 0) L.etop[e] = ev;
        __syncthreads();
      }
      if (!pz_sync(O.gs, ep)) return;
      double s0 = 0, s1 = 0;
      for (int i = 0; i < k; i++) s0 += L.etop[i];
      for (int i = 0; i < k; i++) s1 += L.etop[k + i];
      if (fabs(s0 - s1) < L.eps * fabs(s1)) {
        conv_m = j;
        stop = true;
      }
      // every CTA has read etop before the next test writes it (barriers of
      // the next step come first)
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    LzState *st = L.st;
    st->j = j; st->stop = 1; st->no_break = 1; st->restarts = restarts; st->conv_m = conv_m;
    st->nan_step = nan_step; st->scale = scale; st->npass2 = cnt.npass2; st->nfp32 = cnt.nfp32;
    st->qcols64 = cnt.q64; st->qcols32 = cnt.q32;
  }
}

}  // namespace ddlr
