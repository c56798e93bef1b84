// ddlr_kernels.cuh -- CUDA kernels of the DDLR library (sm_103a).
//
// Vectors live in the device order of the plan: interior rows of block
// 0..p-1, then the interface rows; inside each block rows are sorted by
// dependency level.  All floating-point reductions are two-stage with a fixed
// grid and a fixed summation order (no floating-point atomics), so results do
// not depend on scheduling.
#pragma once
#include <cuda/atomic>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ddlr {

// Loads of the Lanczos basis Q in the persistent kernel's Gram-Schmidt
// passes, with the evict-first cache policy, so that the factor and the
// vectors of the next step's operator keep their place in L2 while the
// 0.8 GB basis streams through.  Other loads keep the default policy: the
// hint measured no faster on the per-phase kernels, slower for the FP32
// sweeps (whose factor the apply's second solve reuses from L2), and slower
// for the L2-resident 64^3 persistent PCG when it also covered the factor.
template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) {
  return __ldcs(p);
}

constexpr int kRedGrid = 304;   // CTAs of every two-stage reduction (2 x 152 SMs)
constexpr int kThreads = 256;

// ---------------------------------------------------------------- helpers
template <typename T> __device__ __forceinline__ T ld_u(const T *p) { return *p; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }

template <typename T> struct AccOf { using type = T; };
template <> struct AccOf<__nv_bfloat16> { using type = float; };

// deterministic block sum of one value per thread (result valid in thread 0)
template <typename T, int NT>
__device__ __forceinline__ T block_sum(T v, T *sm) {
  static_assert((NT / 32 & (NT / 32 - 1)) == 0 && NT / 32 <= 32, "power-of-two warps, at most 32");
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    // the warp sums as a tree (log2 of the warp count dependent adds, not
    // one per warp: FP64 add latency is long on this part)
    r = l < NT / 32 ? sm[l] : T(0);
    for (int o = NT / 64; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// =================================================================== setup
__global__ void k_diag_scale(int n, const int *diag_pos, const double *val,
                             double *dsc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dsc[i] = 1.0 / sqrt(val[diag_pos[i]]);
}

__global__ void k_scale_vals(long long nnz, const int *orow, const int *ocol,
                             const double *val, const double *dsc, double *out) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nnz) out[q] = val[q] * dsc[orow[q]] * dsc[ocol[q]];
}

template <typename T>
__global__ void k_gather(long long cnt, const int *src, const double *in, T *out) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < cnt) { int s = src[q]; out[q] = s >= 0 ? T(in[s]) : T(0); }
}

// initial values of the factor pattern: entries of B_{i,a} = B_i + a^-2 E_i E_i^T
// and C_a = C + a^2 I (eq. split)
// L values of a two-level factor scaled by the inverse diagonal of their
// column: lx[slot] = l[slot] / L_cc (padding slots hold 0 and stay 0)
template <typename T>
__global__ void k_prescale_cols(long long nslot, const int *col, const T *l, const T *dinv, T *lx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nslot) lx[i] = l[i] * dinv[col[i]];
}

__global__ void k_factor_init(int nf, const int *f_src, const int *f_prp,
                              const int *pa, const int *pb,
                              const unsigned char *cdiag, const double *as,
                              double ia2, double a2, double *fval) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nf) return;
  double v = f_src[q] >= 0 ? as[f_src[q]] : 0.0;
  double e = 0.0;
  for (int t = f_prp[q]; t < f_prp[q + 1]; t++) e += as[pa[t]] * as[pb[t]];
  v += ia2 * e;
  if (cdiag[q]) v += a2;
  fval[q] = v;
}

// One dependency level of the up-looking incomplete Cholesky on the given
// pattern (IC(0), or exact Cholesky on the symbolic fill pattern):
//   l_ij = (a_ij - sum_{t in P_i, P_j} l_it l_jt) / l_jj,
//   l_ii = sqrt(a_ii - sum_t l_it^2).
// Rows of one level only read rows of lower levels; columns ascend in device
// order, which is a topological order of the factor, so l_it is final before
// l_ij is formed.  A non-positive pivot sets *err = 1 (BREAKDOWN).
__global__ void k_ic_level(int cnt, const int *rows, const int *f_rp,
                           const int *f_ci, double *fval, int *err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
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
      if (ca == cb) { s -= fval[qa] * fval[qb]; qa++; qb++; }
      else if (ca < cb) qa++;
      else qb++;
    }
    fval[q] = s / fval[eb];
  }
  double d = fval[e - 1];
  for (int q = b; q < e - 1; q++) d -= fval[q] * fval[q];
  if (!(d > 0.0)) { *err = 1; d = 1.0; }
  fval[e - 1] = sqrt(d);
}

// scatter the factor into the sliced-ELL solve layouts (L rows and L^T rows)
template <typename T>
__global__ void k_solve_layout(int nf, const int *f_row, const int *f_rp,
                               const int *map_l, const int *map_u,
                               const int *row_slot, const double *fval, T *lval,
                               T *uval, T *dinv, T *dinv_s) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nf) return;
  const int g = f_row[q];
  if (q == f_rp[g + 1] - 1) {
    dinv[g] = T(1.0 / fval[q]);
    dinv_s[row_slot[g]] = T(1.0 / fval[q]);
  } else {
    lval[map_l[q]] = T(fval[q]);
    uval[map_u[q]] = T(fval[q]);
  }
}

// ====================================================== triangular solves
struct SolveLayout {
  const int *blk_lvl0, *lvl_row0, *lvl_nrows, *lvl_slice0;
  const int *l_soff, *l_sw, *l_col;
  const int *u_soff, *u_sw, *u_col;
};

// forward row:  z_r = (x_r - sum_c L_rc z_c) / L_rr
// backward row: z_r = (z_r - sum_c (L^T)_rc z_c) / L_rr
template <typename T, bool FWD>
__device__ __forceinline__ void solve_row(const SolveLayout &S, const T *val,
                                          const T *dinv, const T *x, T *z,
                                          int slice, int lane, int r) {
  const int *soff = FWD ? S.l_soff : S.u_soff;
  const int *sw = FWD ? S.l_sw : S.u_sw;
  const int *col = FWD ? S.l_col : S.u_col;
  const int off = soff[slice] + lane, w = sw[slice];
  T acc = FWD ? x[r] : z[r];
  for (int kk = 0; kk < w; kk++) {
    const int c = col[off + kk * 32];
    acc -= val[off + kk * 32] * z[c];
  }
  z[r] = acc * dinv[r];
}

// All interior blocks B_{i,a} of A0 in one launch, one CTA per block: forward
// sweep over the block's levels, then backward sweep, with a CTA barrier
// between levels (Sec. 4.2: the p local solves are independent).
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_sptrsv_blocks(SolveLayout S, const T *lval, const T *uval, const T *dinv,
                const T *x, T *z, const int *gate) {
  if (gate && *gate) return;
  const int b = blockIdx.x;
  const int l0 = S.blk_lvl0[b], l1 = S.blk_lvl0[b + 1];
  for (int l = l0; l < l1; l++) {
    const int r0 = S.lvl_row0[l], nr = S.lvl_nrows[l], s0 = S.lvl_slice0[l];
    for (int i = threadIdx.x; i < nr; i += NT)
      solve_row<T, true>(S, lval, dinv, x, z, s0 + (i >> 5), i & 31, r0 + i);
    __syncthreads();
  }
  for (int l = l1 - 1; l >= l0; l--) {
    const int r0 = S.lvl_row0[l], nr = S.lvl_nrows[l], s0 = S.lvl_slice0[l];
    for (int i = threadIdx.x; i < nr; i += NT)
      solve_row<T, false>(S, uval, dinv, x, z, s0 + (i >> 5), i & 31, r0 + i);
    __syncthreads();
  }
}

// ----------------------------------------- TMA-pipelined interior solves
// Shared-memory geometry of k_sptrsv_blocks_tma, chosen on the host.
struct TmaCfg {
  int zs_cap;      // rows of the largest interior block
  int nl_cap;      // levels of the deepest block
  int ns_cap;      // slices of the largest block + 1
  int ring_bytes;  // staging ring (multiple of 128, >= the largest stage)
};
// nanoseconds of the global timer (bounded waits)
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kNBar = 64;       // mbarriers = stages in flight at most
// the TMA solve waits at least this long for its copies (a CTA must not exit
// with copies still in flight into its shared memory)
constexpr unsigned long long kTmaMinWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (TMA), completion counted on `bar`
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__host__ __device__ inline size_t al128(size_t b) { return (b + 127) & ~size_t(127); }

template <typename T>
__host__ __device__ inline size_t tma_smem_bytes(const TmaCfg &c) {
  // barriers | ring | block solution | stage table (2 int4 + 1 int64 per stage) | slice table
  return 8 * kNBar + size_t(c.ring_bytes) + al128(size_t(c.zs_cap) * sizeof(T)) +
         al128(size_t(2 * c.nl_cap) * 40) + size_t(4 * c.ns_cap) * 4;
}

// All interior blocks of A0 in one launch, one CTA per block (Sec. 4.2: the p
// local solves are independent).  The block's solution lives in shared
// memory.  The sliced-ELL data of each level (values, column indices and the
// inverse diagonal in slice layout; every piece a multiple of 128 bytes) is a
// "stage"; stages are brought in by 1-D TMA bulk copies into a byte ring,
// placed one after the other (wrapping to the ring start when a stage does
// not fit before the end), as far ahead as the ring and the 64 mbarriers
// allow.  Placement is a pure function of the stage sizes and is tabulated in
// the prologue.  The last thread of the CTA issues the copies after the
// barrier that ends a level (it has no row in levels narrower than NT-32, so
// this stays off the level chain).  Forward sweep with L, backward sweep with
// L^T.  Waits are bounded: on timeout *err is set and the CTA returns.
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_sptrsv_blocks_tma(SolveLayout S, const T *lval, const T *uval, const T *dinv_s,
                    const T *x, T *z, const int *gate, TmaCfg cfg, int *err, unsigned long long limit_ns) {
  if (gate && *gate) return;
  __shared__ int s_abort;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw);
  unsigned char *ring = smraw + 8 * kNBar;
  const int R = cfg.ring_bytes;
  T *zs = reinterpret_cast<T *>(ring + R);
  unsigned char *tab = reinterpret_cast<unsigned char *>(zs) + al128(size_t(cfg.zs_cap) * sizeof(T));
  int4 *sg0 = reinterpret_cast<int4 *>(tab);                  // {r0, nr, sa, oa}
  int4 *sg1 = sg0 + 2 * cfg.nl_cap;                           // {ne, nsl, pos, bytes}
  long long *slin = reinterpret_cast<long long *>(sg1 + 2 * cfg.nl_cap);  // linear start
  int *st = reinterpret_cast<int *>(tab + al128(size_t(2 * cfg.nl_cap) * 40));
  const int b = blockIdx.x, tid = threadIdx.x;
  const int l0 = S.blk_lvl0[b], l1 = S.blk_lvl0[b + 1], NL = l1 - l0;
  if (NL == 0) return;
  const int rb0 = S.lvl_row0[l0], sb0 = S.lvl_slice0[l0];
  const int NS = S.lvl_slice0[l1] - sb0;
  const int nb = S.lvl_row0[l1 - 1] + S.lvl_nrows[l1 - 1] - rb0;
  const int nstage = 2 * NL;
  constexpr int PROD = NT - 1;
  // stage j: forward level j (j < NL) or backward level 2NL-1-j
  for (int j = tid; j < nstage; j += NT) {
    const bool fwd = j < NL;
    const int li = fwd ? j : nstage - 1 - j;
    const int sa = S.lvl_slice0[l0 + li] - sb0, sbn = S.lvl_slice0[l0 + li + 1] - sb0;
    const int *soff = fwd ? S.l_soff : S.u_soff;
    const int oa = soff[sb0 + sa], ne = soff[sb0 + sbn] - oa;
    sg0[j] = make_int4(S.lvl_row0[l0 + li] - rb0, S.lvl_nrows[l0 + li], sa, oa);
    sg1[j] = make_int4(ne, sbn - sa, 0, ne * int(sizeof(T) + 4) + (sbn - sa) * 32 * int(sizeof(T)));
  }
  for (int i = tid; i <= NS; i += NT) {
    st[4 * i] = S.l_soff[sb0 + i];
    st[4 * i + 1] = i < NS ? S.l_sw[sb0 + i] : 0;
    st[4 * i + 2] = S.u_soff[sb0 + i];
    st[4 * i + 3] = i < NS ? S.u_sw[sb0 + i] : 0;
  }
  for (int i = tid; i < nb; i += NT) zs[i] = x[rb0 + i];
  __syncthreads();
  if (tid == PROD) {
    // ring placement: consecutive, wrapping to 0 when a stage does not fit
    long long lin = 0;
    int pos = 0;
    for (int j = 0; j < nstage; j++) {
      const int by = sg1[j].w;
      if (pos + by > R) { lin += R - pos; pos = 0; }
      sg1[j].z = pos;
      slin[j] = lin;
      lin += by;
      pos += by;
    }
    for (int q = 0; q < kNBar; q++) mbar_init(bar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_abort = 0;
  }
  int jn = 0;   // producer: next stage to issue
  auto produce = [&](int jc) {
    const long long lim = slin[jc] + R;
    while (jn < nstage && jn - jc < kNBar) {
      const int4 g0 = sg0[jn], g1 = sg1[jn];
      if (slin[jn] + g1.w > lim) break;          // would reach the oldest live stage
      const bool fwd = jn < NL;
      unsigned char *dst = ring + g1.z;
      uint64_t *bj = bar + (jn % kNBar);
      mbar_expect_tx(bj, unsigned(g1.w));
      if (g1.x > 0) {
        tma_load_1d(dst, (fwd ? lval : uval) + g0.w, unsigned(g1.x) * (unsigned)sizeof(T), bj);
        tma_load_1d(dst + size_t(g1.x) * sizeof(T), (fwd ? S.l_col : S.u_col) + g0.w, unsigned(g1.x) * 4u, bj);
      }
      tma_load_1d(dst + size_t(g1.x) * (sizeof(T) + 4), dinv_s + size_t(sb0 + g0.z) * 32,
                  unsigned(g1.y) * 32u * (unsigned)sizeof(T), bj);
      jn++;
    }
  };
  if (tid == PROD) produce(0);
  __syncthreads();
  for (int j = 0; j < nstage; j++) {
    const unsigned par = unsigned(j / kNBar) & 1u;
    if (!mbar_try_wait(bar + (j % kNBar), par)) {
      // bounded wait; a thread that gives up tells the others (the decision
      // to stop is the CTA's, taken at the barrier below)
      const unsigned long long t0 = gtimer_ns();
      while (!mbar_try_wait(bar + (j % kNBar), par)) {
        if (*(volatile int *)&s_abort) break;
        if (gtimer_ns() - t0 > limit_ns) { atomicExch(&s_abort, 1); break; }
      }
    }
    __syncthreads();
    if (s_abort) {
      // the copies issued for stages j .. jn-1 may still be in flight into
      // this CTA's shared memory: the producer waits for them (bounded)
      // before the CTA exits
      if (tid == PROD) {
        *err = 1;
        for (int q = j; q < jn; q++) {
          const unsigned pq = unsigned(q / kNBar) & 1u;
          const unsigned long long t0 = gtimer_ns();
          while (!mbar_try_wait(bar + (q % kNBar), pq) && gtimer_ns() - t0 < limit_ns) {
          }
        }
      }
      return;
    }
    const int4 g0 = sg0[j], g1 = sg1[j];
    const bool fwd = j < NL;
    const unsigned char *slot = ring + g1.z;
    const T *sv = reinterpret_cast<const T *>(slot);
    const int *sc = reinterpret_cast<const int *>(slot + size_t(g1.x) * sizeof(T));
    const T *sd = reinterpret_cast<const T *>(slot + size_t(g1.x) * (sizeof(T) + 4));
    const int r0 = g0.x, nr = g0.y, sa = g0.z, oa = g0.w;
    for (int i = tid; i < nr; i += NT) {
      const int sl = sa + (i >> 5), ln = i & 31;
      const int2 so = *reinterpret_cast<const int2 *>(st + 4 * sl + (fwd ? 0 : 2));
      const int o = so.x - oa + ln, w = so.y;
      T acc = zs[r0 + i];
      for (int kk = 0; kk < w; kk++) acc -= sv[o + 32 * kk] * zs[sc[o + 32 * kk] - rb0];
      zs[r0 + i] = acc * sd[i];
    }
    __syncthreads();
    if (tid == PROD && jn < nstage) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      produce(j + 1);
    }
  }
  for (int i = tid; i < nb; i += NT) z[rb0 + i] = zs[i];
}

// --------------------------------------- synchronisation-free interior solve
// Row r of the factor (device order) keeps {first slot, number of entries} of
// its strictly-lower L row and of its strictly-upper L^T row in the sliced-ELL
// arrays (entries kk at first + 32 kk).
struct RowSpan { const int2 *l, *u; };

template <typename T>
__device__ __forceinline__ void sf_wait(int *flag, int target, int *err, bool &late,
                                        unsigned long long limit_ns) {
  cuda::atomic_ref<int, cuda::thread_scope_block> f(*flag);
  if (f.load(cuda::memory_order_acquire) >= target) return;
  const unsigned long long t0 = gtimer_ns();
  while (f.load(cuda::memory_order_acquire) < target) {
    __nanosleep(32);
    if (!late && gtimer_ns() - t0 > limit_ns) { late = true; *err = 1; }
    if (late) return;                 // give up waiting; the result is flagged invalid
  }
}

// All interior blocks of A0 in one launch, one CTA per block (Sec. 4.2), with
// no barrier per level: thread t solves rows t, t+NT, ... of its block in
// topological order (ascending for L, descending for L^T), waiting only on the
// rows each row depends on through a ready flag per row in shared memory
// (release/acquire at block scope).  The block's solution lives in shared
// memory; every thread loads the factor data of its next row before it waits
// on the current one.  Dependencies point to rows earlier in the thread's
// order or to rows of other threads at earlier positions, so every wait
// ends; waits are bounded all the same (on timeout *err is set).
template <typename T, int NT, int WR>
__global__ void __launch_bounds__(NT)
k_sptrsv_blocks_sf(const int *blk_row0, RowSpan rs, const int *l_col, const T *l_val,
                   const int *u_col, const T *u_val, const T *dinv, const T *x, T *z,
                   const int *gate, int *err, unsigned long long limit_ns) {
  if (gate && *gate) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int rb0 = blk_row0[b], nb = blk_row0[b + 1] - rb0;
  T *zs = reinterpret_cast<T *>(smraw);
  int *flag = reinterpret_cast<int *>(smraw + ((size_t(nb) * sizeof(T) + 15) & ~size_t(15)));
  for (int i = tid; i < nb; i += NT) { zs[i] = x[rb0 + i]; flag[i] = 0; }
  __syncthreads();
  bool late = false;
  for (int sweep = 0; sweep < 2; sweep++) {
    const bool fwd = sweep == 0;
    const int2 *span = fwd ? rs.l : rs.u;
    const int *col = fwd ? l_col : u_col;
    const T *val = fwd ? l_val : u_val;
    const int target = fwd ? 1 : 2;
    // this thread's rows in dependency order
    const int count = tid < nb ? (nb - 1 - tid) / NT + 1 : 0;
    const int first = fwd ? tid : tid + (count - 1) * NT;
    const int step = fwd ? NT : -NT;
    // prefetched data of the next row
    int2 nsp = make_int2(0, 0);
    T nv[WR]; int nc[WR]; T nd = T(0);
    auto fetch = [&](int i) {
      const int r = rb0 + i;
      nsp = span[r];
      nd = dinv[r];
#pragma unroll
      for (int kk = 0; kk < WR; kk++)
        if (kk < nsp.y) { nv[kk] = val[nsp.x + 32 * kk]; nc[kk] = col[nsp.x + 32 * kk] - rb0; }
    };
    if (count > 0) fetch(first);
    for (int t = 0, i = first; t < count; t++, i += step) {
      const int2 sp = nsp;
      T cv[WR]; int cc[WR];
#pragma unroll
      for (int kk = 0; kk < WR; kk++) { cv[kk] = nv[kk]; cc[kk] = nc[kk]; }
      const T dd = nd;
      if (t + 1 < count) fetch(i + step);
      T acc = zs[i];
#pragma unroll
      for (int kk = 0; kk < WR; kk++) {
        if (kk < sp.y) {
          sf_wait<T>(flag + cc[kk], target, err, late, limit_ns);
          acc -= cv[kk] * zs[cc[kk]];
        }
      }
      for (int kk = WR; kk < sp.y; kk++) {          // rows wider than WR
        const int c = col[sp.x + 32 * kk] - rb0;
        sf_wait<T>(flag + c, target, err, late, limit_ns);
        acc -= val[sp.x + 32 * kk] * zs[c];
      }
      zs[i] = acc * dd;
      cuda::atomic_ref<int, cuda::thread_scope_block> fi(flag[i]);
      fi.store(target, cuda::memory_order_release);
    }
    __syncthreads();
  }
  for (int i = tid; i < nb; i += NT) z[rb0 + i] = zs[i];
}

// solve_row without the store: the value z_r takes (forward or backward).
// FROM_X: the first forward level was not stored; its value x_c / L_cc is
// formed where it is read (forward: the dependencies of a second-level row,
// all on the first level; backward on the first level: the row's own value).
// PRE (forward FROM_X only): the values are L_rc / L_cc, scaled once at setup,
// so an entry costs one FMA on x_c and no gather of 1 / L_cc.
template <typename T, bool FWD, bool FROM_X, bool PRE = false>
__device__ __forceinline__ T solve_row_value(const SolveLayout &S, const T *val, const T *dinv, const T *x,
                                             const T *z, int slice, int lane, int r) {
  const int *soff = FWD ? S.l_soff : S.u_soff;
  const int *sw = FWD ? S.l_sw : S.u_sw;
  const int *col = FWD ? S.l_col : S.u_col;
  const int off = soff[slice] + lane, w = sw[slice];
  T acc = FWD ? x[r] : (FROM_X ? x[r] * dinv[r] : z[r]);
  for (int kk = 0; kk < w; kk++) {
    const int c = col[off + kk * 32];
    acc -= val[off + kk * 32] * ((FWD && FROM_X) ? (PRE ? x[c] : x[c] * dinv[c]) : z[c]);
  }
  return acc * dinv[r];
}

// One dependency level of many blocks in one launch: CTA q solves chunk q
// = (level record, first row, rows <= kThreads) of that level; mode 0
// forward, 1 backward, 2 forward then backward (a level that is the top
// level of every block it contains).  Two-level factors skip the first
// forward level: mode 3 = mode 2 on the second level reading its
// dependencies as x_c / L_cc, mode 4 = mode 1 on the first level starting
// from x_r / L_rr (the values that level would have stored); mode 5 = mode 3
// with the second level's L values pre-scaled by 1 / L_cc of their columns.  Each of the kThreads / R threads
// solves R rows: it computes all R values (loads only: rows of one level do
// not depend on each other) before storing any, so R dependent load chains
// are in flight per thread.  The value of each row does not depend on R.
template <typename T, int R>
__global__ void __launch_bounds__(kThreads / R)
k_sptrsv_chunks(SolveLayout S, const int4 *chunks, int mode, const T *lval, const T *uval, const T *dinv,
                const T *x, T *z, const int *gate) {
  if (gate && *gate) return;
  constexpr int NT = kThreads / R;
  const int4 ch = chunks[blockIdx.x];
  const int lvl = ch.x, r0 = S.lvl_row0[lvl], s0 = S.lvl_slice0[lvl];
  T v[R];
#pragma unroll
  for (int u = 0; u < R; u++) {
    const int t = threadIdx.x + u * NT;
    if (t >= ch.z) continue;
    const int i = ch.y + t;
    const int r = r0 + i, sl = s0 + (i >> 5), ln = i & 31;
    if (mode == 1) {
      v[u] = solve_row_value<T, false, false>(S, uval, dinv, x, z, sl, ln, r);
    } else if (mode == 4) {
      v[u] = solve_row_value<T, false, true>(S, uval, dinv, x, z, sl, ln, r);
    } else if (mode == 3) {
      v[u] = solve_row_value<T, true, true>(S, lval, dinv, x, z, sl, ln, r) * dinv[r];
    } else if (mode == 5) {
      v[u] = solve_row_value<T, true, true, true>(S, lval, dinv, x, z, sl, ln, r) * dinv[r];
    } else {
      v[u] = solve_row_value<T, true, false>(S, lval, dinv, x, z, sl, ln, r);
      if (mode == 2) v[u] = v[u] * dinv[r];
    }
  }
#pragma unroll
  for (int u = 0; u < R; u++) {
    const int t = threadIdx.x + u * NT;
    if (t < ch.z) z[r0 + ch.y + t] = v[u];
  }
}

// Row value from a level-order descriptor d = {row, first L slot, first L^T
// slot, L entries | L^T entries << 16} (the row's own entries only, no slice
// padding); FROM_X and PRE as in solve_row_value, dr = 1 / L_rr.
// x may be of a wider type TX (the FP64 residual read by the FP32
// preconditioner): it is rounded to T as it is read.
template <typename T, bool FWD, bool FROM_X, bool PRE = false, typename TX = T>
__device__ __forceinline__ T desc_row_value(const int4 d, const int *col, const T *val, const T *dinv,
                                            const TX *x, const T *z, T dr) {
  const int off = FWD ? d.y : d.z;
  const int w = FWD ? int(unsigned(d.w) & 0xffffu) : int(unsigned(d.w) >> 16);
  const int r = d.x;
  T acc = FWD ? T(x[r]) : (FROM_X ? T(x[r]) * dr : z[r]);
  for (int kk = 0; kk < w; kk++) {
    const int c = col[off + kk * 32];
    acc -= val[off + kk * 32] * ((FWD && FROM_X) ? (PRE ? T(x[c]) : T(x[c]) * dinv[c]) : z[c]);
  }
  return acc * dr;
}

// mode 0-4 as k_sptrsv_chunks for one row given by its descriptor
template <typename T, typename TX = T>
__device__ __forceinline__ T desc_row_mode(int mode, const int4 d, const int *l_col, const int *u_col,
                                           const T *lval, const T *uval, const T *dinv, const TX *x,
                                           const T *z, T dr) {
  if (mode == 1) return desc_row_value<T, false, false, false, TX>(d, u_col, uval, dinv, x, z, dr);
  if (mode == 4) return desc_row_value<T, false, true, false, TX>(d, u_col, uval, dinv, x, z, dr);
  if (mode == 3) return desc_row_value<T, true, true, false, TX>(d, l_col, lval, dinv, x, z, dr) * dr;
  if (mode == 5) return desc_row_value<T, true, true, true, TX>(d, l_col, lval, dinv, x, z, dr) * dr;
  const T v = desc_row_value<T, true, false, false, TX>(d, l_col, lval, dinv, x, z, dr);
  return mode == 2 ? v * dr : v;
}

// One dependency level of every block, rows from the level-order descriptor
// list (count rows): three dependent loads per row (descriptor, entries,
// gathered values) instead of five through the chunk tables.  R rows per
// thread as k_sptrsv_chunks; the value of each row does not depend on R.
// x of type TX (rounded to T as read); z64 (optional): the rows' final values
// also written in FP64 (the preconditioner's FP64 output)
template <typename T, int R, typename TX = T>
__global__ void __launch_bounds__(kThreads / R)
k_sptrsv_desc(const int4 *desc, int count, int mode, const int *l_col, const int *u_col, const T *lval,
              const T *uval, const T *dinv, const TX *x, T *z, const int *gate, double *z64 = nullptr) {
  if (gate && *gate) return;
  constexpr int NT = kThreads / R;
  const int base = blockIdx.x * kThreads + threadIdx.x;
  T v[R];
  int rr[R];
#pragma unroll
  for (int u = 0; u < R; u++) {
    const int idx = base + u * NT;
    rr[u] = -1;
    if (idx >= count) continue;
    const int4 d = desc[idx];
    v[u] = desc_row_mode<T, TX>(mode, d, l_col, u_col, lval, uval, dinv, x, z, dinv[d.x]);
    rr[u] = d.x;
  }
#pragma unroll
  for (int u = 0; u < R; u++)
    if (rr[u] >= 0) {
      z[rr[u]] = v[u];
      if (z64) z64[rr[u]] = double(v[u]);
    }
}

// ======================================================= E, E^T products
// v = E w + xadd = [a^-1 Ehat w ; -a w] + xadd   (eq. EF), rows [0, n)
template <typename T>
__global__ void k_e_vec(int m, int s, const int *eh_rp, const int *eh_ci,
                        const T *eh_val, T ia, T a, const T *w, const T *xadd,
                        T *v, const int *gate) {
  if (gate && *gate) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m + s) return;
  T acc;
  if (r < m) {
    acc = 0;
    for (int q = eh_rp[r]; q < eh_rp[r + 1]; q++) acc += eh_val[q] * w[eh_ci[q]];
    acc *= ia;
  } else {
    acc = -a * w[r - m];
  }
  v[r] = xadd ? xadd[r] + acc : acc;
}

// interior rows only: v_r = xadd_r + a^-1 (Ehat w)_r
template <typename T, typename TX = T>
__global__ void k_e_interior(int m, const int *eh_rp, const int *eh_ci,
                             const T *eh_val, T ia, const T *w, const TX *xadd,
                             T *v, const int *gate) {
  if (gate && *gate) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  T acc = 0;
  for (int q = eh_rp[r]; q < eh_rp[r + 1]; q++) acc += eh_val[q] * w[eh_ci[q]];
  v[r] = T(xadd[r]) + ia * acc;
}

// y = E^T z = a^-1 Ehat^T z_B - a z_C  (interface rows j in [0, s))
template <typename T>
__global__ void k_et(int s, int m, const int *eht_rp, const int *eht_ci,
                     const T *eht_val, T ia, T a, const T *z, T *y,
                     const int *gate) {
  if (gate && *gate) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  T acc = 0;
  for (int q = eht_rp[j]; q < eht_rp[j + 1]; q++) acc += eht_val[q] * z[eht_ci[q]];
  y[j] = ia * acc - a * z[m + j];
}

// ================================================ tall-skinny U products
// partials[blk][c] = sum over this CTA's rows r of U[r][c] * x[r]
// (U row-major nrows x k; k <= NT).  Stage 1 of t = U^T x.
template <typename T, typename TU, int NT>
__global__ void __launch_bounds__(NT)
k_utx_partial(int nrows, int k, const TU *U, const T *x, T *partials,
              const int *gate) {
  if (gate && *gate) return;
  __shared__ T xs[NT];
  __shared__ T red[NT];
  const int G = NT / k;
  const int c = threadIdx.x % k, g = threadIdx.x / k;
  T acc = 0;
  for (long long base = (long long)blockIdx.x * NT; base < nrows;
       base += (long long)gridDim.x * NT) {
    const long long r = base + threadIdx.x;
    xs[threadIdx.x] = r < nrows ? x[r] : T(0);
    __syncthreads();
    if (g < G) {
      const int lim = (int)min((long long)NT, nrows - base);
      for (int rr = g; rr < lim; rr += G)
        acc += T(to_acc(U[(base + rr) * k + c])) * xs[rr];
    }
    __syncthreads();
  }
  red[threadIdx.x] = (g < G) ? acc : T(0);
  __syncthreads();
  if (threadIdx.x < k) {
    T s = 0;
    for (int gg = 0; gg < G; gg++) s += red[gg * k + threadIdx.x];
    partials[(long long)blockIdx.x * k + threadIdx.x] = s;
  }
}

// out[c] = coef[c] * sum_g partials[g][c]  (warp per column, fixed order);
// if H != null: out = H * (that k-vector) with H k x k row-major.
template <typename T>
__global__ void k_reduce_cols(int G, int k, const T *partials, const T *coef,
                              const T *H, T *out, const int *gate) {
  if (gate && *gate) return;
  extern __shared__ unsigned char smraw[];
  T *tmp = reinterpret_cast<T *>(smraw);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = w; c < k; c += nw) {
    T s = 0;
    for (int g = l; g < G; g += 32) s += partials[(long long)g * k + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) tmp[c] = coef ? coef[c] * s : s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    if (H) {
      T s = 0;
      for (int b = 0; b < k; b++) s += H[c * k + b] * tmp[b];
      out[c] = s;
    } else {
      out[c] = tmp[c];
    }
  }
}

// DDLR-1 (Algorithm 1): G_{k,theta}^-1 y and the interface half of x + E w:
//   w_j = y_j / (1 - theta) + sum_c U[j][c] t_c   (prop. gkt, t = D U^T y)
//   rhs_{m+j} = x_{m+j} - a w_j
template <typename T, typename TU>
__global__ void k_w_rhs(int s, int m, int k, const TU *U, const T *t,
                        const T *y, const T *inv1mt, T a, const T *x, T *w,
                        T *rhs, const int *gate) {
  if (gate && *gate) return;
  extern __shared__ unsigned char smraw[];
  T *ts = reinterpret_cast<T *>(smraw);
  for (int c = threadIdx.x; c < k; c += blockDim.x) ts[c] = t[c];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  T acc = 0;
  const TU *u = U + (long long)j * k;
  for (int c = 0; c < k; c++) acc += T(to_acc(u[c])) * ts[c];
  const T wj = (*inv1mt) * y[j] + acc;
  w[j] = wj;
  rhs[m + j] = x[m + j] - a * wj;
}

// u_r += sum_c U[r][c] h_c   (DDLR-2, eq. Form2a)
template <typename T, typename TU>
__global__ void k_u_add(int nrows, int k, const TU *U, const T *h, T *u,
                        const int *gate) {
  if (gate && *gate) return;
  extern __shared__ unsigned char smraw[];
  T *hs = reinterpret_cast<T *>(smraw);
  for (int c = threadIdx.x; c < k; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  T acc = 0;
  const TU *row = U + r * k;
  for (int c = 0; c < k; c++) acc += T(to_acc(row[c])) * hs[c];
  u[r] += acc;
}

// --------------------------------------------- vector-load U products
// U row-major (rows x k) read as 16-byte vectors: E = 16 / sizeof(TU) values
// per load, L = k / E lanes per row, so one warp load covers 32 / L whole rows
// (512 contiguous bytes) and every thread keeps UNR loads in flight before
// its FMAs.  Used when k * sizeof(TU) is a multiple of 16 and L divides 32
// (k = 16 or 32 with FP64, FP32 or BF16 U_k); else the kernels above.
template <typename TU> struct Unpack16;
template <> struct Unpack16<double> {
  static constexpr int E = 2;
  template <typename T> __device__ __forceinline__ static void run(const uint4 &v, T *o) {
    o[0] = T(__hiloint2double(int(v.y), int(v.x)));
    o[1] = T(__hiloint2double(int(v.w), int(v.z)));
  }
};
template <> struct Unpack16<float> {
  static constexpr int E = 4;
  template <typename T> __device__ __forceinline__ static void run(const uint4 &v, T *o) {
    o[0] = T(__uint_as_float(v.x));
    o[1] = T(__uint_as_float(v.y));
    o[2] = T(__uint_as_float(v.z));
    o[3] = T(__uint_as_float(v.w));
  }
};
template <> struct Unpack16<__nv_bfloat16> {
  static constexpr int E = 8;
  template <typename T> __device__ __forceinline__ static void run(const uint4 &v, T *o) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      __nv_bfloat162 b;
      memcpy(&b, &w[i], sizeof(b));
      const float2 f = __bfloat1622float2(b);
      o[2 * i] = T(f.x);
      o[2 * i + 1] = T(f.y);
    }
  }
};

// stage 1 of t = U^T x: partials[blk][c] over this CTA's rows (fixed grid,
// fixed order)
// With done != nullptr the CTA that finishes last (arrival counter, no
// waiting) also does stage 2 in the order of k_reduce_cols: out = coef .* sum
// (coef != nullptr), then out = H out (H != nullptr, k x k), and re-arms the
// counter.
template <typename T, typename TU, int L, int NT, int UNR>
__global__ void __launch_bounds__(NT, 2)   // two CTAs per SM: the fixed grid of 2 x 152 in one wave
k_utx_vec(long long nrows, const TU *U, const T *x, T *partials, const int *gate, unsigned *done = nullptr,
          const T *coef = nullptr, const T *H = nullptr, T *out = nullptr) {
  if (gate && *gate) return;
  constexpr int E = Unpack16<TU>::E, K = L * E, RW = 32 / L, NW = NT / 32;
  __shared__ T red[NW][K];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int cg = lane % L, ro = lane / L;
  const long long gw = (long long)blockIdx.x * NW + wi, W = (long long)gridDim.x * NW;
  const uint4 *U4 = reinterpret_cast<const uint4 *>(U);
  T acc[E];
#pragma unroll
  for (int i = 0; i < E; i++) acc[i] = T(0);
  for (long long r0 = gw * RW; r0 < nrows; r0 += W * RW * UNR) {
    uint4 v[UNR];
    T xv[UNR];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      const long long r = r0 + (long long)u * W * RW + ro;
      v[u] = r < nrows ? U4[r * L + cg] : make_uint4(0u, 0u, 0u, 0u);
      xv[u] = r < nrows ? x[r] : T(0);
    }
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      T e[E];
      Unpack16<TU>::run(v[u], e);
#pragma unroll
      for (int i = 0; i < E; i++) acc[i] += e[i] * xv[u];
    }
  }
  // lanes cg, cg + L, ... hold the same columns
#pragma unroll
  for (int o = L; o < 32; o <<= 1)
#pragma unroll
    for (int i = 0; i < E; i++) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  if (ro == 0)
#pragma unroll
    for (int i = 0; i < E; i++) red[wi][cg * E + i] = acc[i];
  __syncthreads();
  for (int c = threadIdx.x; c < K; c += NT) {
    T sum = 0;
    for (int w = 0; w < NW; w++) sum += red[w][c];
    partials[(long long)blockIdx.x * K + c] = sum;
  }
  if (!done) return;
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int G = gridDim.x;
  T *tmp = &red[0][0];   // K values
  for (int c = wi; c < K; c += NW) {
    T sum = 0;
    for (int g = lane; g < G; g += 32) sum += __ldcg(partials + (long long)g * K + c);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) tmp[c] = coef ? coef[c] * sum : sum;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < K; c += NT) {
    if (H) {
      T sum = 0;
      for (int b = 0; b < K; b++) sum += H[c * K + b] * tmp[b];
      out[c] = sum;
    } else {
      out[c] = tmp[c];
    }
  }
  if (threadIdx.x == 0) *done = 0u;
}

// row dot products d_r = U[r][:] . t, L lanes per row, UNR rows in flight per
// thread; the epilogue gets (row, d_r) in lane cg == 0 of each row group:
// DDLR-1 (rows = s): w_j = t_0 y_j + d_j, rhs_{m+j} = x_{m+j} - a w_j;
// DDLR-2 (rows = n): u_r += d_r.
template <typename T, typename TU, int L, int UNR, typename Pre, typename Epi>
__device__ __forceinline__ void u_rows_dot(long long nrows, const TU *U, const T *t, Pre pre, Epi epi) {
  constexpr int E = Unpack16<TU>::E, RW = 32 / L;
  const int lane = threadIdx.x & 31;
  const int cg = lane % L, ro = lane / L;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long W = ((long long)gridDim.x * blockDim.x) >> 5;
  T tv[E];
#pragma unroll
  for (int i = 0; i < E; i++) tv[i] = t[cg * E + i];
  const uint4 *U4 = reinterpret_cast<const uint4 *>(U);
  using PV = decltype(pre(0LL));
  for (long long r0 = gw * RW; r0 < nrows; r0 += W * RW * UNR) {
    uint4 v[UNR];
    PV pv[UNR];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      const long long r = r0 + (long long)u * W * RW + ro;
      v[u] = r < nrows ? U4[r * L + cg] : make_uint4(0u, 0u, 0u, 0u);
      if (cg == 0 && r < nrows) pv[u] = pre(r);
    }
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      T e[E];
      Unpack16<TU>::run(v[u], e);
      T d = 0;
#pragma unroll
      for (int i = 0; i < E; i++) d += e[i] * tv[i];
#pragma unroll
      for (int o = 1; o < L; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      const long long r = r0 + (long long)u * W * RW + ro;
      if (cg == 0 && r < nrows) epi(r, d, pv[u]);
    }
  }
}

// FP64 row dot products d_r = U[r][:] . t, one thread per row: on this part an
// FP64 warp instruction costs the same whatever the active lanes, so a
// cross-lane reduction would multiply the FP64 instructions; instead a tile of
// kRowTile rows is loaded with coalesced 16-byte loads into shared memory
// (row stride k + 1) and each thread sums its row there.  k even, k <= 64.
constexpr int kRowTile = 128;
template <typename Epi>
__device__ __forceinline__ void u_rows_dot_smem(long long nrows, int k, const double *U, const double *t,
                                                double *tile, double *ts, Epi epi) {
  for (int c = threadIdx.x; c < k; c += blockDim.x) ts[c] = t[c];
  const int ld = k + 1;
  const long long ntiles = (nrows + kRowTile - 1) / kRowTile;
  for (long long tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const long long r0 = tl * kRowTile;
    const int rows = (int)min((long long)kRowTile, nrows - r0);
    const int half = rows * k / 2;   // 16-byte chunks of the tile (k even)
    const double2 *src = reinterpret_cast<const double2 *>(U + r0 * k);
    __syncthreads();                 // previous tile consumed (and ts written)
    for (int q = threadIdx.x; q < half; q += blockDim.x) {
      const double2 v = src[q];
      const int e = 2 * q, rr = e / k, cc = e - rr * k;   // cc even, cc + 1 < k
      tile[rr * ld + cc] = v.x;
      tile[rr * ld + cc + 1] = v.y;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const double *row = tile + i * ld;
      double d = 0;
      for (int c = 0; c < k; c++) d += row[c] * ts[c];
      epi(r0 + i, d);
    }
  }
}

__global__ void __launch_bounds__(kRowTile)
k_w_rhs_smem(int s, int m, int k, const double *U, const double *t, const double *y, const double *inv1mt,
             double a, const double *x, double *w, double *rhs, const int *gate) {
  if (gate && *gate) return;
  extern __shared__ double dsm[];
  const double it = *inv1mt;
  u_rows_dot_smem(s, k, U, t, dsm + 64, dsm, [&](long long j, double d) {
    const double wj = it * y[j] + d;
    w[j] = wj;
    rhs[m + j] = x[m + j] - a * wj;
  });
}

__global__ void __launch_bounds__(kRowTile)
k_u_add_smem(long long nrows, int k, const double *U, const double *h, double *u, const int *gate) {
  if (gate && *gate) return;
  extern __shared__ double dsm[];
  u_rows_dot_smem(nrows, k, U, h, dsm + 64, dsm, [&](long long r, double d) { u[r] += d; });
}

// The same FP64 row dot products without the tile: thread per row, its row
// read as KV = k/2 16-byte loads issued back to back, at most 8 at a time (the
// warp's loads cover 32 whole rows, so every sector fetched is used), then k
// FMAs in two chains; t is read from shared memory (broadcast).
template <int KV, typename Pre, typename Epi>
__device__ __forceinline__ void u_rows_dot_direct(long long nrows, const double *U, const double *t, Pre pre,
                                                  Epi epi) {
  constexpr int CH = KV < 8 ? KV : 8;
  __shared__ double ts[2 * KV];
  for (int c = threadIdx.x; c < 2 * KV; c += blockDim.x) ts[c] = t[c];
  __syncthreads();
  const double2 *U2 = reinterpret_cast<const double2 *>(U);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    const auto pv = pre(r);
    double d0 = 0, d1 = 0;
#pragma unroll 1
    for (int q0 = 0; q0 < KV; q0 += CH) {
      double2 v[CH];
#pragma unroll
      for (int q = 0; q < CH; q++) v[q] = U2[r * KV + q0 + q];
#pragma unroll
      for (int q = 0; q < CH; q++) {
        d0 += v[q].x * ts[2 * (q0 + q)];
        d1 += v[q].y * ts[2 * (q0 + q) + 1];
      }
    }
    epi(r, d0 + d1, pv);
  }
}

template <int KV>
__global__ void __launch_bounds__(kThreads, 3) k_w_rhs_direct(int s, int m, const double *U, const double *t, const double *y,
                               const double *inv1mt, double a, const double *x, double *w, double *rhs,
                               const int *gate) {
  if (gate && *gate) return;
  const double it = *inv1mt;
  u_rows_dot_direct<KV>(
      s, U, t, [&](long long j) { return make_double2(y[j], x[m + j]); },
      [&](long long j, double d, double2 yx) {
        const double wj = it * yx.x + d;
        w[j] = wj;
        rhs[m + j] = yx.y - a * wj;
      });
}

template <int KV>
__global__ void __launch_bounds__(kThreads, 3) k_u_add_direct(long long nrows, const double *U, const double *h, double *u, const int *gate) {
  if (gate && *gate) return;
  u_rows_dot_direct<KV>(
      nrows, U, h, [&](long long r) { return u[r]; }, [&](long long r, double d, double ur) { u[r] = ur + d; });
}

template <typename T, typename TU, int L, int UNR, typename TX = T>
__global__ void k_w_rhs_vec(int s, int m, const TU *U, const T *t, const T *y, const T *inv1mt, T a,
                            const TX *x, T *w, T *rhs, const int *gate) {
  if (gate && *gate) return;
  const T it = *inv1mt;
  struct YX { T y, x; };
  u_rows_dot<T, TU, L, UNR>(
      s, U, t, [&](long long j) { return YX{y[j], T(x[m + j])}; },
      [&](long long j, T d, YX yx) {
        const T wj = it * yx.y + d;
        w[j] = wj;
        rhs[m + j] = yx.x - a * wj;
      });
}

template <typename T, typename TU, int L, int UNR>
__global__ void k_u_add_vec(long long nrows, const TU *U, const T *h, T *u, const int *gate) {
  if (gate && *gate) return;
  u_rows_dot<T, TU, L, UNR>(
      nrows, U, h, [&](long long r) { return u[r]; }, [&](long long r, T d, T ur) { u[r] = ur + d; });
}

// ===================================================== vectors and PCG
// y = A x with A in sliced ELL (device order)
template <typename T>
__global__ void k_spmv(int n, const int *soff, const int *sw, const int *col,
                       const T *val, const T *x, T *y, const int *gate) {
  if (gate && *gate) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int g = r >> 5, l = r & 31;
  const int off = soff[g] + l, w = sw[g];
  T acc = 0;
  for (int kk = 0; kk < w; kk++) acc += val[off + kk * 32] * x[col[off + kk * 32]];
  y[r] = acc;
}

// Streaming loops over n elements on a fixed grid: thread t of CTA b takes
// elements i0 + u * G * NT (u = 0..3) per round, i0 = b * NT + t + 4 G NT *
// round, so a thread has the loads of four elements in flight at once (one at
// a time kept a few MB in flight, ~2.5 TB/s here) and warps stay coalesced.
constexpr int kStreamUnr = 4;

template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_dot_partial(long long n, const T *a, const T *b, T *partials, const int *gate) {
  if (gate && *gate) return;
  __shared__ T sm[NT / 32];
  T acc = 0;
  const long long st = (long long)gridDim.x * NT;
  for (long long i0 = (long long)blockIdx.x * NT + threadIdx.x; i0 < n; i0 += kStreamUnr * st) {
    T av[kStreamUnr], bv[kStreamUnr];
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) {
      const long long i = i0 + u * st;
      av[u] = i < n ? a[i] : T(0);
      bv[u] = i < n ? b[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) acc += av[u] * bv[u];
  }
  acc = block_sum<T, NT>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}


// partial sums of two dot products a.b and a.c
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_dot2_partial(long long n, const T *a, const T *b, const T *c, T *partials,
               const int *gate) {
  if (gate && *gate) return;
  __shared__ T sm[NT / 32];
  T acc = 0, acc2 = 0;
  for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n;
       i += (long long)gridDim.x * NT) {
    acc += a[i] * b[i];
    acc2 += a[i] * c[i];
  }
  acc = block_sum<T, NT>(acc, sm);
  acc2 = block_sum<T, NT>(acc2, sm);
  if (threadIdx.x == 0) { partials[blockIdx.x] = acc; partials[gridDim.x + blockIdx.x] = acc2; }
}

// sum of G partials in a fixed order (one warp)
__device__ __forceinline__ double warp_sum_partials(const double *p, int G) {
  const int l = threadIdx.x & 31;
  double s = 0;
  for (int g = l; g < G; g += 32) s += p[g];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return __shfl_sync(0xffffffffu, s, 0);
}

__global__ void k_reduce_scalar(int G, const double *partials, double *out,
                                int do_sqrt, const int *gate) {
  if (gate && *gate) return;
  double s = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) *out = do_sqrt ? sqrt(s) : s;
}

template <typename T, typename S>
__global__ void k_cast(long long n, const S *in, T *out, const int *gate) {
  if (gate && *gate) return;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = T(in[i]);
}

// out = a .* b
template <typename T>
__global__ void k_mulv_t(long long n, const T *a, const T *b, T *out, const int *gate) {
  if (gate && *gate) return;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] * b[i];
}

__global__ void k_to_bf16(long long n, const double *in, __nv_bfloat16 *out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(float(in[i]));
}

// out[g] = in[perm[g]] (original -> device order)
template <typename T>
__global__ void k_permute_in(int n, const int *perm, const T *in, T *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] = in[perm[g]];
}
template <typename T>
__global__ void k_permute_out(int n, const int *perm, const T *in, T *out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[perm[g]] = in[g];
}

// partial sums of ||b - q||^2
template <int NT>
__global__ void __launch_bounds__(NT)
k_resid2_partial(long long n, const double *b, const double *q, double *partials) {
  __shared__ double sm[NT / 32];
  double acc = 0;
  for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n;
       i += (long long)gridDim.x * NT) {
    const double d = b[i] - q[i];
    acc += d * d;
  }
  acc = block_sum<double, NT>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// --------------------------------------------------------- PCG control
struct PcgState {
  double rz, rz_new, pq, alpha, beta, rr, bb, tol2, rt2, rzold;
  int its, maxit, done, status, check_true, restart, flexible, pad;
};

__global__ void k_pcg_init(PcgState *st, const double *partials, int G,
                           double tol, int maxit, int flexible) {
  double bb = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    st->bb = bb;
    st->tol2 = tol * tol * bb;
    st->its = 0; st->maxit = maxit; st->status = 0; st->check_true = 0;
    st->restart = 0; st->flexible = flexible;
    st->done = (bb == 0.0) ? 1 : 0;
    st->rz = 0; st->rr = bb;
  }
}

// rz = r.z after the first preconditioning
__global__ void k_pcg_rz0(PcgState *st, const double *partials, int G) {
  if (st->done) return;
  double s = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    st->rz = s;
    if (!(s == s) || isinf(s)) { st->status = 7; st->done = 1; }
  }
}

// alpha = rz / (p.q)
__global__ void k_pcg_alpha(PcgState *st, const double *partials, int G) {
  if (st->done) return;
  double pq = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    st->pq = pq;
    st->alpha = st->rz / pq;
    if (!(st->alpha == st->alpha) || isinf(st->alpha)) { st->status = 7; st->done = 1; }
  }
}

// x += alpha p; r -= alpha q; partial r.r
template <int NT>
__global__ void __launch_bounds__(NT)
k_pcg_update(long long n, PcgState *st, const double *p, const double *q,
             double *x, double *r, double *partials) {
  if (st->done) return;
  __shared__ double sm[NT / 32];
  const double a = st->alpha;
  double acc = 0;
  for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n;
       i += (long long)gridDim.x * NT) {
    x[i] += a * p[i];
    const double ri = r[i] - a * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  acc = block_sum<double, NT>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// recursive residual test; a pass schedules the true-residual check
__global__ void k_pcg_rr(PcgState *st, const double *partials, int G) {
  if (st->done) return;
  double rr = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    st->rr = rr;
    st->its += 1;
    if (!(rr == rr) || isinf(rr)) { st->status = 7; st->done = 1; return; }
    st->check_true = (rr <= st->tol2) ? 1 : 0;
    if (!st->check_true && st->its >= st->maxit) { st->status = 5; st->done = 1; }
  }
}

// t = b - A x for the true-residual check, partial t.t
template <int NT>
__global__ void __launch_bounds__(NT)
k_pcg_true_res(int n, const PcgState *st, const int *soff, const int *sw,
               const int *col, const double *val, const double *b,
               const double *x, double *t, double *partials) {
  if (st->done || !st->check_true) return;
  __shared__ double sm[NT / 32];
  double acc = 0;
  for (int r = blockIdx.x * NT + threadIdx.x; r < n; r += gridDim.x * NT) {
    const int g = r >> 5, l = r & 31;
    const int off = soff[g] + l, w = sw[g];
    double ax = 0;
    for (int kk = 0; kk < w; kk++) ax += val[off + kk * 32] * x[col[off + kk * 32]];
    const double tr = b[r] - ax;
    t[r] = tr;
    acc += tr * tr;
  }
  acc = block_sum<double, NT>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_pcg_true_dec(PcgState *st, const double *partials, int G) {
  if (st->done || !st->check_true) return;
  double rt2 = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) {
    st->rt2 = rt2;
    st->check_true = 0;
    if (rt2 <= st->tol2) { st->status = 0; st->done = 1; return; }
    st->restart = 1;     // continue from the true residual
    if (st->its >= st->maxit) { st->status = 5; st->done = 1; }
  }
}

__global__ void k_pcg_copy_r(long long n, const PcgState *st, const double *t,
                             double *r) {
  if (st->done || !st->restart) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = t[i];
}

// beta = rz_new / rz (Hestenes-Stiefel) or (rz_new - r.z_old) / rz (flexible)
__global__ void k_pcg_beta(PcgState *st, const double *partials, int G) {
  if (st->done) return;
  double rzn = warp_sum_partials(partials, G);
  double rzo = warp_sum_partials(partials + G, G);
  if (threadIdx.x == 0) {
    double beta = st->flexible ? (rzn - rzo) / st->rz : rzn / st->rz;
    if (st->restart) beta = 0.0;
    st->beta = beta;
    st->rz = rzn;
    st->restart = 0;
    if (!(rzn == rzn) || isinf(rzn)) { st->status = 7; st->done = 1; }
  }
}

// ---- fused forms of the per-phase PCG (one launch instead of a reduction
// kernel plus a one-CTA scalar kernel): every CTA writes its partial sum; the
// CTA that arrives last (arrival counter, no waiting) sums all partials in a
// fixed order, updates the PCG state and re-arms the counter.
__device__ __forceinline__ bool pcg_last_cta(unsigned *done) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// fixed-order sum of G partials by one CTA (valid in thread 0)
template <int NT>
__device__ __forceinline__ double pcg_sum_partials(const double *partials, int G, double *sm) {
  double v = 0;
  for (int g = threadIdx.x; g < G; g += NT) v += __ldcg(partials + g);
  return block_sum<double, NT>(v, sm);
}

// x += alpha p; r -= alpha q; then the recursive-residual test of k_pcg_rr
template <int NT>
__global__ void __launch_bounds__(NT)
k_pcg_update_rr(long long n, PcgState *st, const double *p, const double *q, double *x, double *r,
                double *partials, unsigned *done) {
  if (st->done) return;
  __shared__ double sm[NT / 32];
  const double a = st->alpha;
  double acc = 0;
  const long long stp = (long long)gridDim.x * NT;
  for (long long i0 = (long long)blockIdx.x * NT + threadIdx.x; i0 < n; i0 += kStreamUnr * stp) {
    double pv[kStreamUnr], qv[kStreamUnr], xv[kStreamUnr], rv[kStreamUnr];
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) {
      const long long i = i0 + u * stp;
      if (i < n) { pv[u] = p[i]; qv[u] = q[i]; xv[u] = x[i]; rv[u] = r[i]; }
    }
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) {
      const long long i = i0 + u * stp;
      if (i < n) {
        x[i] = xv[u] + a * pv[u];
        const double ri = rv[u] - a * qv[u];
        r[i] = ri;
        acc += ri * ri;
      }
    }
  }
  acc = block_sum<double, NT>(acc, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (!pcg_last_cta(done)) return;
  const double rr = pcg_sum_partials<NT>(partials, gridDim.x, sm);
  if (threadIdx.x == 0) {
    *done = 0u;
    st->rr = rr;
    st->its += 1;
    if (!(rr == rr) || isinf(rr)) { st->status = 7; st->done = 1; return; }
    st->check_true = (rr <= st->tol2) ? 1 : 0;
    if (!st->check_true && st->its >= st->maxit) { st->status = 5; st->done = 1; }
  }
}

// r.z and r.zold, then the beta update of k_pcg_beta
template <int NT>
__global__ void __launch_bounds__(NT)
k_dot2_beta(long long n, const double *r, const double *z, const double *zo, double *partials, PcgState *st,
            unsigned *done) {
  if (st->done) return;
  __shared__ double sm[NT / 32];
  // zo == z (plain CG): r.zold is not needed, and neither its loads nor its
  // FP64 products are spent
  const bool two = zo != z;
  double a1 = 0, a2 = 0;
  const long long stp = (long long)gridDim.x * NT;
  for (long long i0 = (long long)blockIdx.x * NT + threadIdx.x; i0 < n; i0 += kStreamUnr * stp) {
    double rv[kStreamUnr], zv[kStreamUnr], ov[kStreamUnr];
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) {
      const long long i = i0 + u * stp;
      rv[u] = i < n ? r[i] : 0.0;
      zv[u] = i < n ? z[i] : 0.0;
      ov[u] = two && i < n ? zo[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kStreamUnr; u++) a1 += rv[u] * zv[u];
    if (two)
#pragma unroll
      for (int u = 0; u < kStreamUnr; u++) a2 += rv[u] * ov[u];
  }
  a1 = block_sum<double, NT>(a1, sm);
  if (two) a2 = block_sum<double, NT>(a2, sm);
  if (threadIdx.x == 0) { partials[blockIdx.x] = a1; partials[gridDim.x + blockIdx.x] = a2; }
  if (!pcg_last_cta(done)) return;
  const double rzn = pcg_sum_partials<NT>(partials, gridDim.x, sm);
  const double rzo = two ? pcg_sum_partials<NT>(partials + gridDim.x, gridDim.x, sm) : rzn;
  if (threadIdx.x == 0) {
    *done = 0u;
    double beta = st->flexible ? (rzn - rzo) / st->rz : rzn / st->rz;
    if (st->restart) beta = 0.0;
    st->beta = beta;
    st->rz = rzn;
    st->restart = 0;
    if (!(rzn == rzn) || isinf(rzn)) { st->status = 7; st->done = 1; }
  }
}

// p = z + beta p (and z_old = z for flexible CG)
__global__ void k_pcg_p(long long n, const PcgState *st, const double *z,
                        double *p, double *zold) {
  if (st->done) return;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double zi = z[i];
  p[i] = zi + st->beta * p[i];
  if (zold) zold[i] = zi;
}

// ================================================================ Lanczos
// ------------------------------------------------ device-driven Lanczos step
// Control state of the Lanczos recurrence kept on the device, so a step needs
// no host round trip and can be replayed as one CUDA graph: the step index,
// the stop flag (set at m = m_max, by the convergence test of eq. converge,
// or on NaN), the breakdown decision and the running scale of the tridiagonal.
struct LzState {
  int j;            // current step (0-based)
  int stop;         // nonzero: later step kernels return at once
  int no_break;     // 1: normal step; 0: breakdown -> restart kernels run
  int restarts;     // restarts so far (SplitMix64 stream seed + restarts)
  int conv_m;       // m at which eq. converge was met (0: not met)
  int nan_step;     // first step with a non-finite alpha or beta (-1: none)
  int mmax;
  int pass2;        // 1: this step's reorthogonalisation takes a second pass
  int npass2;       // steps that took the second pass (restart vectors excluded)
  int nfp32;        // Gram-Schmidt corrections formed from the FP32 copy of Q
  double scale;     // max |alpha_i|, beta_i seen (breakdown threshold)
  unsigned long long seed;
  double qcols64, qcols32;  // basis columns read by the Gram-Schmidt passes in FP64 / FP32
};

// SplitMix64 (Steele, Lea & Flood 2014): output i of stream `seed`, mapped to
// [-1, 1) as 2 (z >> 11) 2^-53 - 1
__device__ __forceinline__ double d_sm64_pm1(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return 2.0 * (double(z >> 11) * 0x1.0p-53) - 1.0;
}

// arr[st->j] = sum of G partials (sqrt when asked)
__global__ void k_lz_reduce_at(int G, const double *partials, double *arr, const LzState *st,
                               int do_sqrt, const int *gate) {
  if (gate && *gate) return;
  double s = warp_sum_partials(partials, G);
  if (threadIdx.x == 0) arr[st->j] = do_sqrt ? sqrt(s) : s;
}

// w -= alpha_j q_j + beta_{j-1} q_{j-1}
__global__ void k_lz_three_term_d(int s, const double *al, const double *be, const LzState *st,
                                  const double *qcur, const double *qprev, double *w) {
  if (st->stop) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const int j = st->j;
  double v = w[r] - al[j] * qcur[r];
  if (j > 0) v -= be[j - 1] * qprev[r];
  w[r] = v;
}

// partials of Q_{j+1}^T w (columns 0..j), warp per column; gate: return when
// *gate != 0 (gate_inv: return when *gate_inv == 0)
template <int NT>
__global__ void __launch_bounds__(NT)
k_gemvT_partial_d(int s, const double *Q, long long ld, const double *w, double *partials,
                  const LzState *st, const int *gate, const int *gate_inv) {
  if ((gate && *gate) || (gate_inv && !*gate_inv)) return;
  const int ncol = st->j + 1;
  const int nw = NT / 32, wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  const long long chunk = ((long long)s + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * chunk;
  const long long r1 = min((long long)s, r0 + chunk);
  for (int j = wi; j < ncol; j += nw) {
    const double *q = Q + (long long)j * ld;
    double acc = 0;
    for (long long r = r0 + l; r < r1; r += 32) acc += q[r] * w[r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (l == 0) partials[(long long)blockIdx.x * ncol + j] = acc;
  }
}

// c[j] = sum_g partials[g][j], j <= st->j (warp per column, fixed order)
__global__ void k_reduce_cols_d(int G, const double *partials, double *c, const LzState *st,
                                const int *gate, const int *gate_inv) {
  if ((gate && *gate) || (gate_inv && !*gate_inv)) return;
  const int ncol = st->j + 1;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int col = blockIdx.x * nw + w; col < ncol; col += gridDim.x * nw) {
    double s = 0;
    for (int g = l; g < G; g += 32) s += partials[(long long)g * ncol + col];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) c[col] = s;
  }
}

// w -= Q_{j+1} c
__global__ void k_gemvN_sub_d(int s, const double *Q, long long ld, const double *c, double *w,
                              const LzState *st, const int *gate, const int *gate_inv) {
  if ((gate && *gate) || (gate_inv && !*gate_inv)) return;
  extern __shared__ unsigned char smraw[];
  double *cs = reinterpret_cast<double *>(smraw);
  const int ncol = st->j + 1;
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) cs[j] = c[j];
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  double acc = 0;
  for (int j = 0; j < ncol; j++) acc += Q[(long long)j * ld + r] * cs[j];
  w[r] -= acc;
}

// breakdown decision of step j (beta_j <= 1e-12 max(|alpha_i|, beta_i))
// Second Gram-Schmidt pass of a Lanczos step: always when always2, else when
// the first pass left less than half of ||w||^2 (nrm[0] before, nrm[1] after)
__global__ void k_lz_dgks(LzState *st, const double *nrm, int always2) {
  if (st->stop || threadIdx.x != 0) return;
  st->pass2 = (always2 || nrm[1] < 0.5 * nrm[0]) ? 1 : 0;
  st->npass2 += st->pass2;
}

__global__ void k_lz_decide(LzState *st, const double *al, const double *be) {
  if (st->stop || threadIdx.x != 0) return;
  const int j = st->j;
  const double a = al[j], b = be[j];
  if (!(a == a) || isinf(a) || !(b == b) || isinf(b)) {
    if (st->nan_step < 0) st->nan_step = j;
    st->stop = 1;
    return;
  }
  st->scale = fmax(st->scale, fabs(a));
  const bool brk = b <= 1e-12 * (st->scale > 0 ? st->scale : 1.0);
  st->no_break = brk ? 0 : 1;
  if (brk) st->restarts += 1;
  else st->scale = fmax(st->scale, b);
}

// normal step: q_{j+1} = w / beta_j into Q, qprev <- qcur, qcur <- q_{j+1}
__global__ void k_lz_normalize(int s, const double *w, const double *be, double *Q, long long ld,
                               double *qcur, double *qprev, const LzState *st) {
  if (st->stop || !st->no_break) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const int j = st->j;
  const double v = w[r] / be[j];
  Q[(long long)(j + 1) * ld + r] = v;
  qprev[r] = qcur[r];
  qcur[r] = v;
}

// breakdown: w = SplitMix64 stream (seed + restarts), drawn in the order of
// rank[] (ascending original index of the interface nodes)
__global__ void k_lz_randvec(int s, const int *rank, const LzState *st, double *w) {
  if (st->stop || st->no_break) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  w[r] = d_sm64_pm1(st->seed + (unsigned long long)st->restarts, (unsigned long long)rank[r]);
}

// breakdown: q_{j+1} = w / ||w|| (w orthogonalised), beta_j = 0
__global__ void k_lz_restart_norm(int s, const double *w, const double *nrm, double *Q, long long ld,
                                  double *qcur, double *qprev, double *be, const LzState *st) {
  if (st->stop || st->no_break) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const int j = st->j;
  const double v = w[r] / (*nrm);
  Q[(long long)(j + 1) * ld + r] = v;
  qprev[r] = qcur[r];
  qcur[r] = v;
  if (r == 0) be[j] = 0.0;
}

// end of step j: j += 1; stop at m_max
__global__ void k_lz_advance(LzState *st) {
  if (st->stop || threadIdx.x != 0) return;
  st->j += 1;
  st->no_break = 1;
  if (st->j >= st->mmax) st->stop = 1;
}

// eq. converge on the sums of the k largest Ritz values of T_m and T_{m-1}
__global__ void k_lz_converged(const double *esum, double eps, int m, LzState *st) {
  if (threadIdx.x != 0 || st->conv_m > 0) return;
  if (fabs(esum[0] - esum[1]) < eps * fabs(esum[1])) { st->conv_m = m; st->stop = 1; }
}

// ------------------------------------------------ tridiagonal eigensolver
// Eigenvalues of the symmetric tridiagonal T_m (diagonal al, off-diagonal be)
// by Sturm-sequence multisection, eigenvectors by inverse iteration
// (Wilkinson; Golub & Van Loan Sec. 8.4-8.5).  Everything is parallel and
// uses fused multiply-adds only in the inner loops: FP64 division and square
// root are slow on this part, and one-thread QR sweeps were the bottleneck.

// number of eigenvalues of T smaller than x: sign changes of the three-term
// Sturm recurrence p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}; a zero term is
// replaced by a tiny value of the opposite sign.  Every 8 terms |p| is brought
// back into [2^-500, 2^500] by an exact power-of-two rescaling (T comes from
// a bounded operator: its entries are O(1), so 8 terms stay far inside the
// double range).  Signs and zero tests read the bit pattern (integer pipe):
// on this part every FP64 instruction takes a long issue slot of the narrow
// FP64 pipe, and only the three of the recurrence remain on the path.
__device__ __forceinline__ bool neg_nonzero(long long b) { return b < 0 && (b << 1) != 0; }
__device__ __forceinline__ int sturm_count(int m, const double *a, const double *b2, double x) {
  constexpr long long kBig = 0x5F30000000000000LL;     // bits of 2^500
  constexpr long long kSmall = 0x20B0000000000000LL;   // bits of 2^-500
  double pm = 1.0, p = a[0] - x;
  if (p == 0.0) p = -1e-300;
  long long pb = __double_as_longlong(p);
  int cnt = neg_nonzero(pb) ? 1 : 0;
  for (int i = 1; i < m; i++) {
    double q = fma(a[i] - x, p, -b2[i - 1] * pm);
    long long qb = __double_as_longlong(q);
    if ((qb << 1) == 0) {
      q = neg_nonzero(pb) ? 1e-300 * fabs(p) : -1e-300 * fabs(p);
      qb = __double_as_longlong(q);
    }
    cnt += neg_nonzero(qb) != neg_nonzero(pb) ? 1 : 0;
    pm = p;
    p = q;
    pb = qb;
    if ((i & 7) == 0) {
      const long long ab = qb & 0x7FFFFFFFFFFFFFFFLL;
      if (ab > kBig) { p *= 0x1.0p-500; pm *= 0x1.0p-500; pb = __double_as_longlong(p); }
      else if (ab < kSmall) { p *= 0x1.0p+500; pm *= 0x1.0p+500; pb = __double_as_longlong(p); }
    }
  }
  return cnt;
}

// Eigenvalue gi (0 = largest) of T_m by Sturm-sequence multisection.  Every
// thread of the CTA calls it; the first P threads (P a multiple of 32, one
// warp per SM sub-partition for P = 128) evaluate P interior points of the
// current bracket per round (log2(P + 1) bits per round), starting from the
// Gershgorin interval widened by 1e-9 of its span.  a, b2: diagonal and
// squared off-diagonal (b2[i] = be[i]^2, i + 1 < m) in shared memory; be:
// off-diagonal; bc: 2 doubles of shared memory.  All threads get the value.
template <int P, int ROUNDS>
__device__ __forceinline__ double tridiag_eig_cta(int m, const double *a, const double *b2,
                                                  const double *be, int gi, double *bc) {
  const int tid = threadIdx.x;
  if (tid < 32) {
    double lo = 1e300, hi = -1e300;
    for (int i = tid; i < m; i += 32) {
      const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (tid == 0) { bc[0] = lo; bc[1] = hi; }
  }
  __syncthreads();
  const double lo = bc[0], hi = bc[1];
  __syncthreads();
  const double span = fmax(hi - lo, 1e-300);
  double blo = lo - 1e-9 * span, bhi = hi + 1e-9 * span;
  const int target = m - 1 - gi;
  constexpr double kStep = 1.0 / double(P + 1);
  for (int round = 0; round < ROUNDS; round++) {
    int below = 0;
    if (tid < P) {
      const double x = blo + (bhi - blo) * double(tid + 1) * kStep;
      below = sturm_count(m, a, b2, x) <= target;   // points below the eigenvalue
    }
    const int nb = __syncthreads_count(below);        // counts are monotone in x
    const double nlo = nb > 0 ? blo + (bhi - blo) * double(nb) * kStep : blo;
    const double nhi = nb < P ? blo + (bhi - blo) * double(nb + 1) * kStep : bhi;
    blo = nlo;
    bhi = nhi;
  }
  return 0.5 * (blo + bhi);
}
constexpr int kEigPoints = 128;   // points per round (4 warps)
constexpr int kEigRounds = 9;     // 9 x log2(129) = 63 bits

// The nv largest eigenvalues of T_m, descending, into vals: CTA gi computes
// eigenvalue gi with kEigPoints threads.  Spreading the eigenvalues over
// many SMs matters because the FP64 pipe of one SM is narrow.  Dynamic
// shared memory: 2m + 2 doubles.
__global__ void __launch_bounds__(kEigPoints) k_tridiag_values(int m, const double *al, const double *be,
                                                                int nv, double *vals) {
  extern __shared__ double shm[];
  double *a = shm, *b2 = shm + m, *bc = shm + 2 * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    a[i] = al[i];
    b2[i] = (i + 1 < m) ? be[i] * be[i] : 0.0;
  }
  __syncthreads();
  const int gi = blockIdx.x;
  if (gi >= nv) return;
  const double v = tridiag_eig_cta<kEigPoints, kEigRounds>(m, a, b2, be, gi, bc);
  if (threadIdx.x == 0) vals[gi] = v;
}

// *out = sum of the first k entries of v (fixed order)
__global__ void k_sum_first(int k, const double *v, double *out) {
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < k; i++) s += v[i];
    *out = s;
  }
}

// Eigenvectors of T_m for the nv given eigenvalues (descending) by inverse
// iteration: one thread per vector factors T - lambda I by Gaussian
// elimination with partial pivoting (tridiagonal, second superdiagonal from
// the row swaps) and solves three times from a fixed start vector,
// normalising each time.  Vectors whose eigenvalues lie within 1e-3 ||T|| of
// each other (a cluster) are then re-orthogonalised by modified Gram-Schmidt
// in order.  Y is column-major m x nv; work holds 5m doubles per vector.
__global__ void k_tridiag_vectors(int m, const double *al, const double *be,
                                  int nv, const double *vals, double *Y,
                                  double *work) {
  __shared__ double red[32];
  __shared__ double s_tn;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double tn = 0;
    for (int i = 0; i < m; i++)
      tn = fmax(tn, fabs(al[i]) + (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0));
    s_tn = fmax(tn, 1e-300);
  }
  __syncthreads();
  const double tnorm = s_tn;
  for (int v = tid; v < nv; v += blockDim.x) {
    double *d = work + size_t(v) * 5 * m, *du = d + m, *du2 = du + m, *dl = du2 + m, *y = dl + m;
    const double lam = vals[v];
    for (int i = 0; i < m; i++) {
      d[i] = al[i] - lam;
      du[i] = (i + 1 < m) ? be[i] : 0.0;
      du2[i] = 0.0;
    }
    double *flags = y;   // flags[i] = 1 when rows i and i+1 were swapped
    for (int i = 0; i + 1 < m; i++) {
      const double sub = be[i];
      if (fabs(d[i]) >= fabs(sub)) {
        const double piv_d = (d[i] != 0.0) ? d[i] : 1e-15 * tnorm;
        d[i] = piv_d;
        const double l = sub / piv_d;
        dl[i] = l;
        d[i + 1] -= l * du[i];
        flags[i] = 0.0;
      } else {
        const double l = d[i] / sub;
        dl[i] = l;
        const double old_du = du[i];
        d[i] = sub;
        du[i] = d[i + 1];
        const double nxt = (i + 1 < m - 1) ? du[i + 1] : 0.0;
        du2[i] = nxt;
        d[i + 1] = old_du - l * du[i];
        if (i + 1 < m - 1) du[i + 1] = -l * nxt;
        flags[i] = 1.0;
      }
    }
    if (d[m - 1] == 0.0) d[m - 1] = 1e-15 * tnorm;
    // reciprocal pivots, once: the three solves below multiply (an FP64
    // division costs about ten times a multiply on this part)
    for (int i = 0; i < m; i++) d[i] = 1.0 / d[i];
    double *b = Y + size_t(v) * m;
    for (int r = 0; r < m; r++) {
      // start vector: 1 + small deterministic perturbation per (v, r)
      unsigned int h = (unsigned)(r * 2654435761u) ^ (unsigned)(v * 40503u + 12345u);
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      b[r] = 1.0 + 0.5 * (double(h & 0xffff) / 65536.0 - 0.5);
    }
    for (int it = 0; it < 3; it++) {
      // forward: apply the row swaps and multipliers
      for (int i = 0; i + 1 < m; i++) {
        if (flags[i] != 0.0) { const double t = b[i]; b[i] = b[i + 1]; b[i + 1] = t; }
        b[i + 1] -= dl[i] * b[i];
      }
      // back substitution with U (reciprocal diagonal d, super du, second super du2)
      b[m - 1] = b[m - 1] * d[m - 1];
      if (m > 1) b[m - 2] = (b[m - 2] - du[m - 2] * b[m - 1]) * d[m - 2];
      for (int i = m - 3; i >= 0; i--) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) * d[i];
      double nn = 0;
      for (int r = 0; r < m; r++) nn = fma(b[r], b[r], nn);
      const double inv = 1.0 / sqrt(nn);
      for (int r = 0; r < m; r++) b[r] *= inv;
    }
  }
  __syncthreads();
  // modified Gram-Schmidt inside clusters, in order of decreasing eigenvalue
  for (int v = 1; v < nv; v++) {
    double *yv = Y + size_t(v) * m;
    int first = v;
    while (first > 0 && fabs(vals[first - 1] - vals[first]) <= 1e-3 * tnorm) first--;
    if (first == v) continue;
    for (int j = first; j < v; j++) {
      const double *yj = Y + size_t(j) * m;
      double part = 0;
      for (int r = tid; r < m; r += blockDim.x) part = fma(yv[r], yj[r], part);
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((tid & 31) == 0) red[tid >> 5] = part;
      __syncthreads();
      if (tid == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        red[0] = t;
      }
      __syncthreads();
      const double dt = red[0];
      for (int r = tid; r < m; r += blockDim.x) yv[r] -= dt * yj[r];
      __syncthreads();
    }
    double part = 0;
    for (int r = tid; r < m; r += blockDim.x) part = fma(yv[r], yv[r], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
      red[0] = 1.0 / sqrt(t);
    }
    __syncthreads();
    const double sc = red[0];
    for (int r = tid; r < m; r += blockDim.x) yv[r] *= sc;
    __syncthreads();
  }
}

// U (s x k row-major) = Q_m Y_k   (Ritz vectors; Q column-major ld, Y
// column-major m x m with the wanted vectors in its first k columns)
template <int CH>
__global__ void k_ritz_gemm(int s, int m, int k, const double *Q, long long ld,
                            const double *Y, double *U) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  for (int c0 = 0; c0 < k; c0 += CH) {
    double acc[CH];
#pragma unroll
    for (int t = 0; t < CH; t++) acc[t] = 0;
    for (int j = 0; j < m; j++) {
      const double q = Q[(long long)j * ld + r];
#pragma unroll
      for (int t = 0; t < CH; t++)
        if (c0 + t < k) acc[t] += q * Y[(long long)(c0 + t) * m + j];
    }
#pragma unroll
    for (int t = 0; t < CH; t++)
      if (c0 + t < k) U[r * k + c0 + t] = acc[t];
  }
}

// DDLR-1 scalars: theta, 1/(1-theta) and D_c = (1-lambda_c)^-1 - (1-theta)^-1
// (prop. gkt); flags NOT_SPD when lambda_max >= 1 or theta >= 1.
__global__ void k_ddlr1_coef(int m, int k, int theta_mode, const double *vals,
                             double *theta, double *inv1mt, double *coef,
                             int *notspd) {
  if (threadIdx.x != 0) return;
  const double th = (theta_mode == 1 && k < m) ? vals[k] : 0.0;
  *theta = th;
  *inv1mt = 1.0 / (1.0 - th);
  for (int c = 0; c < k; c++) coef[c] = 1.0 / (1.0 - vals[c]) - 1.0 / (1.0 - th);
  if (!(vals[0] < 1.0) || !(th < 1.0)) *notspd = 1;
}

// column c of a row-major n x k matrix <-> contiguous vector
__global__ void k_get_col(long long n, int k, int c, const double *M, double *v) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) v[r] = M[r * k + c];
}
__global__ void k_set_col(long long n, int k, int c, const double *v, double *M) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) M[r * k + c] = v[r];
}

// partials of K = U^T EV over row chunks (U, EV row-major n x k)
__global__ void k_utv_partial(long long n, int k, const double *U,
                              const double *EV, double *partials) {
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int pr = threadIdx.x; pr < k * k; pr += blockDim.x) {
    const int a = pr / k, b = pr % k;
    double acc = 0;
    for (long long r = r0; r < r1; r++) acc += U[r * k + a] * EV[r * k + b];
    partials[(long long)blockIdx.x * k * k + pr] = acc;
  }
}

// H_k = (I - (K + K^T)/2)^-1 by Cholesky (lemma 1 / prop. spd-2); failure of
// the Cholesky flags NOT_SPD.  One thread; k is small.
__global__ void k_hk_finalize(int G, int k, const double *partials, double *work,
                              double *Hk, int *notspd) {
  if (threadIdx.x != 0) return;
  double *M = work;            // k x k
  double *e = work + k * k;    // k
  for (int a = 0; a < k; a++)
    for (int b = 0; b < k; b++) {
      double s1 = 0, s2 = 0;
      for (int g = 0; g < G; g++) {
        s1 += partials[(long long)g * k * k + a * k + b];
        s2 += partials[(long long)g * k * k + b * k + a];
      }
      M[a * k + b] = (a == b ? 1.0 : 0.0) - 0.5 * (s1 + s2);
    }
  for (int j = 0; j < k; j++) {
    double dj = M[j * k + j];
    for (int t = 0; t < j; t++) dj -= M[j * k + t] * M[j * k + t];
    if (!(dj > 0.0)) { *notspd = 1; return; }
    dj = sqrt(dj);
    M[j * k + j] = dj;
    for (int i = j + 1; i < k; i++) {
      double sm = M[i * k + j];
      for (int t = 0; t < j; t++) sm -= M[i * k + t] * M[j * k + t];
      M[i * k + j] = sm / dj;
    }
  }
  for (int c = 0; c < k; c++) {
    for (int r = 0; r < k; r++) e[r] = (r == c) ? 1.0 : 0.0;
    for (int i = 0; i < k; i++) {
      double sm = e[i];
      for (int t = 0; t < i; t++) sm -= M[i * k + t] * e[t];
      e[i] = sm / M[i * k + i];
    }
    for (int i = k - 1; i >= 0; i--) {
      double sm = e[i];
      for (int t = i + 1; t < k; t++) sm -= M[t * k + i] * e[t];
      e[i] = sm / M[i * k + i];
    }
    for (int r = 0; r < k; r++) Hk[r * k + c] = e[r];
  }
}

}  // namespace ddlr
