// ddlr_api.cu -- C ABI of the DDLR library: setup, A0 solve, M^-1 apply,
// Lanczos and PCG orchestration on one GB300 (sm_103a).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <type_traits>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "ddlr.h"
#include "ddlr_batch.cuh"
#include "ddlr_cheb.cuh"
#include "ddlr_rand.cuh"
#include "ddlr_mr.cuh"
#include "ddlr_lbd.cuh"
#include "ddlr_gmres.cuh"
#include "ddlr_ldl.cuh"
#include "ddlr_internal.h"
#include "ddlr_kernels.cuh"
#include "ddlr_plan.h"
#include "ddlr_persist.cuh"

using namespace ddlr;

namespace {

struct Fail {
  ddlr_status st;
  std::string msg;
};

inline void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) throw Fail{DDLR_ERR_OOM, std::string(what) + ": out of device memory"};
    throw Fail{DDLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

inline unsigned nblk(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// SplitMix64 (Steele, Lea & Flood 2014): output i of the stream `seed`
inline double sm64_pm1(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return 2.0 * (double(z >> 11) * 0x1.0p-53) - 1.0;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

thread_local std::string g_setup_error;

}  // namespace

struct ddlr_ctx {
  ddlr_options opt{};
  int device = 0;                  // the device current at setup; all its memory is there
  unsigned long long wait_ns = 2000000000ull;   // limit of every bounded device wait
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t stream2 = nullptr;  // C_a solve branch (forked with events)
  cudaStream_t gstream = nullptr;  // internal stream of the PCG graph
  cudaGraphExec_t pcg_exec = nullptr;
  int pcg_exec_flexible = -1;
  long long pcg_nodes = 0;
  std::vector<long long> pcg_fam_nodes;
  long long lz_nodes = 0;
  std::vector<long long> lz_fam_nodes;
  // batched (multi right-hand side) path
  struct Batch {
    int R = 0;
    std::vector<void *> mem;
    double *B = nullptr, *X = nullptr, *Rr = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr,
           *T = nullptr, *Zo = nullptr, *S = nullptr;
    double *w64[5] = {nullptr};
    float *w32[7] = {nullptr};
    double *cb64[5] = {nullptr};   // Chebyshev C_a solve: x, s (two), r, D^-1 r
    float *cb32[5] = {nullptr};
    double *part64 = nullptr;
    float *part32 = nullptr;
    double *fpart = nullptr;   // per-64-row-block column partials of the fused step kernels
    PcgStateMR *st = nullptr;
    struct G {
      cudaGraphExec_t exec = nullptr;
      int flex = -1;
      long long nodes = 0;
      std::vector<long long> fam_nodes;
    };
    std::map<int, G> graphs;            // one captured PCG iteration per width R
    int chunk_per = 0, bd_elem = 256;   // autotuned: rows per pass of the level solve, row-kernel block
    bool tuned = false;
    int last_R = 0;                     // width of the last batched solve (byte accounting)
    bool tc = true;                     // U_k products on the tensor cores (FP32 vectors; DDLR_BATCH_TC=0: scalar)
  } bt;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Plan P;
  std::string err;
  std::vector<void *> allocs;   // device chunks of the handle's arena
  char *arena_cur = nullptr;
  size_t arena_left = 0;
  static constexpr size_t kArenaChunk = size_t(32) << 20;
  long long dev_bytes = 0;

  // plan arrays on the device
  int *perm = nullptr;
  int *a_soff = nullptr, *a_sw = nullptr, *a_col = nullptr, *a_src = nullptr;
  int *eh_rp = nullptr, *eh_ci = nullptr, *eh_src = nullptr;
  int *eht_rp = nullptr, *eht_ci = nullptr, *eht_src = nullptr;
  int *f_rp = nullptr, *f_ci = nullptr, *f_row = nullptr, *f_src = nullptr;
  int *f_prp = nullptr, *f_pa = nullptr, *f_pb = nullptr;
  unsigned char *f_cdiag = nullptr;
  int *fl_rows = nullptr;
  int *map_l = nullptr, *map_u = nullptr;
  int *orow = nullptr, *ocol = nullptr, *diag_pos = nullptr;
  SolveLayout S{};
  // numeric data
  double *val = nullptr;      // caller's values (original CSR order)
  double *vals = nullptr;     // scaled values (alias of val without scaling)
  double *dsc = nullptr;      // D^-1/2 in ORIGINAL order (scale_diag)
  double *dsc_dev = nullptr;  // D^-1/2 in device order
  double *a_val = nullptr;    // A (unscaled) in sliced ELL, device order
  double *fval = nullptr;     // factor values (CSR)
  double *l64 = nullptr, *u64 = nullptr, *dinv64 = nullptr, *eh64 = nullptr, *eht64 = nullptr;
  float *l32 = nullptr, *u32 = nullptr, *dinv32 = nullptr, *eh32 = nullptr, *eht32 = nullptr;
  // two-level factors: L values pre-scaled by 1 / L_cc of their column (the
  // second level's forward sweep reads x_c directly); DDLR_PRESCALE=0 keeps
  // the unscaled form
  double *lx64 = nullptr;
  float *lx32 = nullptr;
  double *dinvs64 = nullptr;  // inverse diagonal in slice layout (TMA solve)
  float *dinvs32 = nullptr;
  int *row_slot = nullptr;
  TmaCfg tma64{}, tma32{};
  bool use_tma64 = false, use_tma32 = false;
  bool use_sf64 = false, use_sf32 = false;   // synchronisation-free interior solve
  bool uvec = true;           // vector-load U_k products (DDLR_UVEC=0: scalar kernels)
  unsigned *udone = nullptr;  // arrival counter of the fused U^T x reduction (0 between launches)
  unsigned *pdone = nullptr;  // arrival counter of the fused per-phase PCG reductions
  int chunk_rows = 0;         // rows per thread of the level-chunk solve: 0 = 2 (FP64) / 4 (FP32);
                              // DDLR_CHUNK_ROWS=1|2|4 fixes it
  int2 *l_span = nullptr, *u_span = nullptr;
  int *blk_row0 = nullptr;
  int *chunks = nullptr;
  int4 *lv_desc = nullptr;    // level-order row descriptors (shallow factors)
  // Chebyshev solve with C_a (c_solver 1): C_a as CSR over the interface
  // rows, the coefficient table (see ddlr_cheb.cuh), single-RHS workspaces
  int *cc_rp = nullptr, *cc_ci = nullptr, *cc_src = nullptr, *cc_diag = nullptr, *cz_rank = nullptr;
  double *cc64 = nullptr, *ctab64 = nullptr;
  float *cc32 = nullptr, *ctab32 = nullptr;
  double *cb64[5] = {nullptr};
  float *cb32[5] = {nullptr};
  double *cz_al = nullptr, *cz_be = nullptr, *cz_vals = nullptr, *cz_Y = nullptr, *cz_work = nullptr,
         *cz_b0 = nullptr;
  // randomized low-rank build (lowrank_method 1), allocated at first use
  struct RandWork {
    bool ready = false;
    int L = 0;
    double *Yb = nullptr, *Qb = nullptr, *V = nullptr, *Z = nullptr, *Z2 = nullptr, *part = nullptr, *G = nullptr,
           *Linv = nullptr, *d = nullptr, *e = nullptr, *Hv = nullptr, *vals = nullptr, *eY = nullptr, *work = nullptr;
    double *Vk = nullptr, *EV = nullptr, *vc = nullptr, *ev = nullptr, *uc = nullptr, *kp = nullptr, *hw = nullptr;
    int *rank = nullptr;
  } rw;
  // Lanczos bidiagonalisation (lowrank_method 2), allocated at first use
  struct LbdWork {
    bool ready = false;
    int mmax = 0;
    double *Vq = nullptr, *Uq = nullptr, *al = nullptr, *be = nullptr, *td = nullptr, *te = nullptr, *t = nullptr,
           *u = nullptr, *v = nullptr, *cpart = nullptr, *cvec = nullptr, *evals = nullptr, *eY = nullptr,
           *work = nullptr, *esum = nullptr, *etop = nullptr, *G = nullptr, *Vk = nullptr, *EV = nullptr,
           *vc = nullptr, *ev = nullptr, *kp = nullptr, *hw = nullptr, *q0 = nullptr;
  } lb;
  // restarted GMRES: Arnoldi basis V (n x (m+1)), Z = M^-1 V (n x m), H
  // ((m+1) x m), rotations, g, y, CGS partials, device scalars
  struct GmresWork {
    int m = 0;
    double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr,
           *cpart = nullptr, *cvec = nullptr, *st = nullptr;
    // Arnoldi step j of a cycle as one CUDA graph each (captured at first
    // use; they hold the arrays above and the handle's wait limit)
    std::vector<cudaGraphExec_t> step;
    int step_m = 0;                   // the restart length they were captured for
    std::vector<long long> nodes;
    std::vector<std::vector<long long>> fam_nodes;
    void free_graphs() {
      for (auto &e : step)
        if (e) cudaGraphExecDestroy(e);
      step.clear();
      nodes.clear();
      fam_nodes.clear();
    }
  } gm;
  int cheb_msteps = 0;
  // approximate inverse of C_a (c_solver 2): columns of X during the MR
  // iterations, then the symmetric part as row CSR (ptr, distinct counts)
  struct MrWork {
    int *xcnt = nullptr, *xrow = nullptr, *zcnt = nullptr, *zrow = nullptr;
    double *xval = nullptr, *zval = nullptr, *num = nullptr, *den = nullptr, *beta = nullptr;
    int *rcnt = nullptr, *ptr = nullptr, *cursor = nullptr, *col = nullptr, *ucnt = nullptr;
    double *val = nullptr;
    float *val32 = nullptr;
    long long nnz = 0;       // distinct entries of the symmetric part
  } mr;
  // low-rank data (device order)
  int urows = 0;
  double *U64 = nullptr, *coef64 = nullptr, *Hk64 = nullptr, *theta_d = nullptr, *inv1mt64 = nullptr;
  float *U32 = nullptr, *coef32 = nullptr, *Hk32 = nullptr, *inv1mt32 = nullptr;
  __nv_bfloat16 *Ub16 = nullptr;
  std::vector<double> ritz;
  int msteps = 0;
  int lz_passes = 0;          // Gram-Schmidt passes of the last Lanczos build
  int lz_fp32 = 0;            // of their corrections, those formed in FP32
  double theta = 0.0;
  int *dflag = nullptr;       // device error flags [0]=breakdown [1]=notspd [2]=eig fail
  // Lanczos workspace, start vector and step graph, kept for refactors
  struct LzWork {
    bool ready = false;
    double *Q = nullptr, *al = nullptr, *be = nullptr, *cvec = nullptr, *w = nullptr, *qcur = nullptr,
           *qprev = nullptr, *nrm = nullptr, *ework = nullptr, *etop = nullptr, *evals = nullptr,
           *esum = nullptr, *eY = nullptr, *q0 = nullptr;
    float *Q32 = nullptr;             // FP32 copy of Q (persistent Lanczos)
    double *V = nullptr, *EV = nullptr, *vc = nullptr, *ev = nullptr, *uc = nullptr, *kp = nullptr, *hw = nullptr;
    int *rank = nullptr;
    LzState *st = nullptr;
    LzState *h_st = nullptr;          // pinned
    cudaEvent_t ev_chk = nullptr, ev_done = nullptr;
    cudaGraphExec_t exec = nullptr;   // one captured step (kernel-per-phase path)
  } lw;
  // persistent cooperative kernels (shallow factors): one CTA per SM
  double *pz_part = nullptr;  // 3 x pz_grid x pz_pstride partial sums
  unsigned *pz_bar = nullptr; // grid-barrier arrival counter
  unsigned char *pz_lvl0 = nullptr;  // rows on the first level of their block
  int pz_grid = 0, pz_pstride = 0, pz_mmax = 0;
  bool pz_pcg = false, pz_lz = false;
  // algorithmic bytes moved by the persistent launches since the last reset
  double pz_pcg_bytes = 0, pz_lz_bytes = 0;
  long long pz_pcg_runs = 0, pz_lz_runs = 0;
  // workspaces
  double *w64[8] = {nullptr};
  float *w32[8] = {nullptr};
  double *part64 = nullptr;
  float *part32 = nullptr;
  PcgState *pcg = nullptr;
  double *pv[8] = {nullptr};
  double *stg_in = nullptr, *stg_out = nullptr;  // staging of host vector arguments
  double *h_pin = nullptr;    // pinned host scratch
  // accounting
  long long launches = 0;
  bool timing = false;
  struct Rec { int fam; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> evpool;
  std::vector<std::string> fam_names;
  std::map<std::string, int> fam_idx;
  std::vector<double> fam_ms;
  std::vector<long long> fam_cnt;
  double setup_ms = 0;
  double plan_ms = 0;

  template <typename T>
  T *alloc(size_t n) {
    // bump allocation (256-byte aligned) from chunks of at least kArenaChunk
    // bytes: one cudaMalloc per chunk instead of one per array
    if (n == 0) n = 1;
    const size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
    if (bytes > arena_left) {
      const size_t chunk = std::max(bytes, kArenaChunk);
      void *p = nullptr;
      ck(cudaMalloc(&p, chunk), "cudaMalloc");
      allocs.push_back(p);
      arena_cur = static_cast<char *>(p);
      arena_left = chunk;
    }
    T *r = reinterpret_cast<T *>(arena_cur);
    arena_cur += bytes;
    arena_left -= bytes;
    dev_bytes += (long long)bytes;
    return r;
  }
  template <typename V>
  auto upload(const V &v) -> typename V::value_type * {
    using T = typename V::value_type;
    T *d = alloc<T>(v.size());
    if (!v.empty()) ck(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream), "upload");
    return d;
  }
  void release() {
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
    arena_cur = nullptr;
    arena_left = 0;
    dev_bytes = 0;
  }

  // ---- launch accounting
  int fam(const char *name) {
    auto it = fam_idx.find(name);
    if (it != fam_idx.end()) return it->second;
    int id = int(fam_names.size());
    fam_names.push_back(name);
    fam_ms.push_back(0.0);
    fam_cnt.push_back(0);
    fam_idx[name] = id;
    return id;
  }
  cudaEvent_t get_ev() {
    if (evpool.empty()) resolve();
    if (evpool.empty()) {
      cudaEvent_t e;
      ck(cudaEventCreate(&e), "cudaEventCreate");
      return e;
    }
    cudaEvent_t e = evpool.back();
    evpool.pop_back();
    return e;
  }
  void resolve() {
    if (pending.empty()) return;
    for (auto &r : pending) {
      cudaEventSynchronize(r.b);
      float ms = 0;
      cudaEventElapsedTime(&ms, r.a, r.b);
      fam_ms[r.fam] += ms;
      evpool.push_back(r.a);
      evpool.push_back(r.b);
    }
    pending.clear();
  }
  struct Scope {
    ddlr_ctx *c; int f; cudaStream_t s; cudaEvent_t a = nullptr;
    Scope(ddlr_ctx *c_, const char *name, cudaStream_t s_) : c(c_), f(c_->fam(name)), s(s_) {
      c->launches++;
      c->fam_cnt[f]++;
      if (c->timing) { a = c->get_ev(); cudaEventRecord(a, s); }
    }
    ~Scope() {
      if (c->timing) {
        cudaEvent_t b = c->get_ev();
        cudaEventRecord(b, s);
        c->pending.push_back({f, a, b});
        if (c->pending.size() > 4096) c->resolve();
      }
    }
  };
};

#define KL(ctx, name, strm, kern, grid, block, smem, ...)                      \
  do {                                                                          \
    ddlr_ctx::Scope _sc((ctx), (name), (strm));                                 \
    kern<<<(grid), (block), (smem), (strm)>>>(__VA_ARGS__);                     \
  } while (0)

namespace {

// The dynamic shared-memory limit of a kernel (cudaFuncSetAttribute) holds
// per device for the whole process, for every handle: it is only ever
// raised, so that a handle created later with a smaller need does not leave
// an earlier handle's launches above the limit.
void raise_smem_limit(const void *fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> limit;
  int dev = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  size_t &cur = limit[{fn, dev}];
  if (bytes <= cur) return;
  ck(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)), "attr");
  cur = bytes;
}

template <typename T>
size_t sf_smem_bytes(const Plan &P) {
  return ((size_t(P.tma_zs) * sizeof(T) + 15) & ~size_t(15)) + size_t(P.tma_zs) * 4;
}

// geometry of the TMA-pipelined interior solve for element type T: the ring
// takes what the shared memory of one SM leaves for each co-resident CTA
// (enough CTAs per SM to hold every interior block in one wave, up to 4),
// capped at one block's total staged bytes; false if a stage does not fit
template <typename T>
bool tma_config(const Plan &P, TmaCfg &cfg) {
  int dev = 0, sms = 0, per_sm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (P.tma_zs <= 0 || sms <= 0) return false;
  const int cps = std::max(1, std::min(4, (P.p + sms - 1) / sms));
  // the kernel's static shared memory (its abort word) comes out of the same
  // per-block limit as the dynamic part
  constexpr long long kStatic = 128;
  const long long budget = std::min<long long>(optin, per_sm / cps - 1024) - kStatic;
  cfg = TmaCfg{P.tma_zs, P.tma_nl, P.tma_ns, 0};
  const long long fixed = (long long)tma_smem_bytes<T>(cfg);
  const long long stage_max = (long long)P.tma_e * (long long)(sizeof(T) + 4) +
                              (long long)P.tma_s * 32 * (long long)sizeof(T);
  const long long block_total = P.tma_blk_e * (long long)(sizeof(T) + 4) +
                                P.tma_blk_s * 32 * (long long)sizeof(T);
  long long ring = std::min(budget - fixed, block_total + stage_max);
  ring &= ~127LL;
  if (ring < stage_max || ring <= 0) return false;
  cfg.ring_bytes = int(ring);
  return true;
}

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double *l(ddlr_ctx *c) { return c->l64; }
  static const double *lx(ddlr_ctx *c) { return c->lx64; }
  static const double *u(ddlr_ctx *c) { return c->u64; }
  static const double *dinv(ddlr_ctx *c) { return c->dinv64; }
  static const double *dinvs(ddlr_ctx *c) { return c->dinvs64; }
  static const double *eh(ddlr_ctx *c) { return c->eh64; }
  static const double *eht(ddlr_ctx *c) { return c->eht64; }
  static double *w(ddlr_ctx *c, int i) { return c->w64[i]; }
  static double *part(ddlr_ctx *c) { return c->part64; }
  static const double *coef(ddlr_ctx *c) { return c->coef64; }
  static const double *inv1mt(ddlr_ctx *c) { return c->inv1mt64; }
  static const double *Hk(ddlr_ctx *c) { return c->Hk64; }
};
template <> struct Prec<float> {
  static const float *l(ddlr_ctx *c) { return c->l32; }
  static const float *lx(ddlr_ctx *c) { return c->lx32; }
  static const float *u(ddlr_ctx *c) { return c->u32; }
  static const float *dinv(ddlr_ctx *c) { return c->dinv32; }
  static const float *dinvs(ddlr_ctx *c) { return c->dinvs32; }
  static const float *eh(ddlr_ctx *c) { return c->eh32; }
  static const float *eht(ddlr_ctx *c) { return c->eht32; }
  static float *w(ddlr_ctx *c, int i) { return c->w32[i]; }
  static float *part(ddlr_ctx *c) { return c->part32; }
  static const float *coef(ddlr_ctx *c) { return c->coef32; }
  static const float *inv1mt(ddlr_ctx *c) { return c->inv1mt32; }
  static const float *Hk(ddlr_ctx *c) { return c->Hk32; }
};

// ----------------------------------------------------------- A0 solve
// z = A0^-1 x in device order: all interior blocks in one launch (CTA per
// block) on the main stream, the C_a levels on the second stream.
static_assert(kChunk == kThreads, "a level chunk is one CTA's rows");
constexpr int kShallowLevels = 8;   // at most this deep: solve level by level over all blocks

// levels [L0, L1) of the chunk lists ptr: forward up to the top, the top
// level forward and backward in one pass, then backward down
template <typename T>
void chunk_sweeps(ddlr_ctx *c, cudaStream_t st, const std::vector<int> &ptr, const char *fam,
                  const T *lv0, const T *uv, const T *di, const T *x, T *z, const int *gate) {
  const int nL = int(ptr.size()) - 1;
  const T *lx = Prec<T>::lx(c);
  auto launch = [&](int L, int mode) {
    const int nch = ptr[L + 1] - ptr[L];
    if (nch <= 0) return;
    const int4 *chk = reinterpret_cast<const int4 *>(c->chunks) + ptr[L];
    const T *lv = mode == 5 ? lx : lv0;
    // measured at 128^3 (A0 solve): FP64 best with 2 rows per thread, FP32 with 4
    const int rows = c->chunk_rows ? c->chunk_rows : (sizeof(T) == 8 ? 2 : 4);
    if (rows == 4)
      KL(c, fam, st, (k_sptrsv_chunks<T, 4>), nch, kThreads / 4, 0, c->S, chk, mode, lv, uv, di, x, z, gate);
    else if (rows == 2)
      KL(c, fam, st, (k_sptrsv_chunks<T, 2>), nch, kThreads / 2, 0, c->S, chk, mode, lv, uv, di, x, z, gate);
    else
      KL(c, fam, st, (k_sptrsv_chunks<T, 1>), nch, kThreads, 0, c->S, chk, mode, lv, uv, di, x, z, gate);
  };
  if (nL == 2) {            // multicolour factors: two launches, see modes 3 (5) and 4
    launch(1, lx ? 5 : 3);
    launch(0, 4);
    return;
  }
  for (int L = 0; L + 1 < nL; L++) launch(L, 0);
  if (nL > 0) launch(nL - 1, 2);
  for (int L = nL - 2; L >= 0; L--) launch(L, 1);
}

// the same sweeps over the level-order descriptor list (all blocks); x may be
// wider than T (rounded as read), z64 (optional) also receives the result in
// FP64 (every row's final value is written in FP64 too)
template <typename T, typename TX = T>
void desc_sweeps(ddlr_ctx *c, cudaStream_t st, const char *fam, const T *lv0, const T *uv, const T *di,
                 const TX *x, T *z, const int *gate, double *z64 = nullptr) {
  const std::vector<int> &ptr = c->P.lv_ptr;
  const int nL = int(ptr.size()) - 1;
  const int rows = c->chunk_rows ? c->chunk_rows : (sizeof(T) == 8 ? 2 : 4);
  const T *lx = Prec<T>::lx(c);
  auto launch = [&](int L, int mode) {
    const int cnt = ptr[L + 1] - ptr[L];
    if (cnt <= 0) return;
    const T *lv = mode == 5 ? lx : lv0;
    const int4 *d = c->lv_desc + ptr[L];
    const int grid = (cnt + kThreads - 1) / kThreads;
    const int *lc = c->S.l_col, *uc = c->S.u_col;
    // rows are final after the top level (modes 2, 3, 5) and the backward
    // levels (modes 1, 4)
    double *o64 = mode == 0 ? nullptr : z64;
    if (rows == 4)
      KL(c, fam, st, (k_sptrsv_desc<T, 4, TX>), grid, kThreads / 4, 0, d, cnt, mode, lc, uc, lv, uv, di, x, z, gate,
         o64);
    else if (rows == 2)
      KL(c, fam, st, (k_sptrsv_desc<T, 2, TX>), grid, kThreads / 2, 0, d, cnt, mode, lc, uc, lv, uv, di, x, z, gate,
         o64);
    else
      KL(c, fam, st, (k_sptrsv_desc<T, 1, TX>), grid, kThreads, 0, d, cnt, mode, lc, uc, lv, uv, di, x, z, gate,
         o64);
  };
  if (nL == 2) {
    launch(1, lx ? 5 : 3);
    launch(0, 4);
    return;
  }
  for (int L = 0; L + 1 < nL; L++) launch(L, 0);
  if (nL > 0) launch(nL - 1, 2);
  for (int L = nL - 2; L >= 0; L--) launch(L, 1);
}

// ------------------------------------------- Chebyshev solve with C_a
template <typename T> struct ChebP;
template <> struct ChebP<double> {
  static const double *cv(ddlr_ctx *c) { return c->cc64; }
  static const double *tab(ddlr_ctx *c) { return c->ctab64; }
  static double *buf(ddlr_ctx *c, int R, int i) { return R == 1 ? c->cb64[i] : c->bt.cb64[i]; }
};
template <> struct ChebP<float> {
  static const float *cv(ddlr_ctx *c) { return c->cc32; }
  static const float *tab(ddlr_ctx *c) { return c->ctab32; }
  static float *buf(ddlr_ctx *c, int R, int i) { return R == 1 ? c->cb32[i] : c->bt.cb32[i]; }
};

// z_C = Xs x_C by the approximate inverse (c_solver 2)
template <typename T> const T *mr_vals(ddlr_ctx *c);
template <> const double *mr_vals<double>(ddlr_ctx *c) { return c->mr.val; }
template <> const float *mr_vals<float>(ddlr_ctx *c) { return c->mr.val32; }
template <typename T>
void mr_apply_c(ddlr_ctx *c, cudaStream_t st, const T *x, T *z, int R, const int *gate) {
  const int s = c->P.s, m = c->P.m;
  KL(c, "mr_apply", st, k_mr_apply<T>, nblk((long long)s * R), kThreads, 0, s, m, R, c->mr.ptr, c->mr.ucnt,
     c->mr.col, mr_vals<T>(c), x, z, gate);
}

// z = D_a^-1 x on the interface rows (the C_a block's levels alone; R
// right-hand sides row-major)
template <typename T>
void cheb_dsolve(ddlr_ctx *c, cudaStream_t st, const T *x, T *z, int R, const int *gate);

// x_C -> C_a^-1 x_C by cheb_steps Chebyshev steps (ddlr_cheb.cuh).  On entry
// the interface rows of z hold D_a^-1 x_C (the A0 sweeps formed it, since
// block p is D_a); on return they hold the Chebyshev iterate x_t.
template <typename T>
void cheb_tail(ddlr_ctx *c, cudaStream_t st, const T *x, T *z, int R, const int *gate) {
  const Plan &P = c->P;
  const int s = P.s, m = P.m, t = c->opt.cheb_steps;
  const unsigned grid = unsigned(((long long)s * R + kThreads - 1) / kThreads);
  T *xacc = ChebP<T>::buf(c, R, 0), *sd[2] = {ChebP<T>::buf(c, R, 1), ChebP<T>::buf(c, R, 2)};
  T *r = ChebP<T>::buf(c, R, 3), *zt = ChebP<T>::buf(c, R, 4);
  const T *cv = ChebP<T>::cv(c), *tab = ChebP<T>::tab(c);
  KL(c, "cheb", st, k_cheb_first<T>, grid, kThreads, 0, s, m, R, c->cc_rp, c->cc_ci, cv, tab, t, x, z, sd[0],
     xacc, r, gate);
  for (int j = 1; j < t; j++) {
    cheb_dsolve<T>(c, st, r, zt, R, gate);
    KL(c, "cheb", st, k_cheb_step<T>, grid, kThreads, 0, s, m, R, c->cc_rp, c->cc_ci, cv, tab, t, j, zt,
       sd[(j - 1) & 1], sd[j & 1], xacc, r, z, gate);
  }
}

// z = A0^-1 x in device order (Sec. 4.2: the p local solves with B_{i,a} and
// the solve with C_a).  Shallow factors (multicolour orders): every level of
// all blocks in one launch.  Deep factors: all interior blocks in one launch
// (CTA per block) on the main stream, the C_a levels on a forked stream.
template <typename T>
void a0_solve(ddlr_ctx *c, const T *x, T *z, const int *gate) {
  const Plan &P = c->P;
  const T *lv = Prec<T>::l(c), *uv = Prec<T>::u(c), *di = Prec<T>::dinv(c);
  if (c->opt.factor >= 2) {
    // L D L^T factors: forward over the levels of all blocks, then backward
    // with D^-1 (ddlr_ldl.cuh)
    static_assert(kChunk == kChunkThreads, "level chunks are one row per thread");
    const std::vector<int> &ptr = P.ch_all_ptr;
    const int nL = int(ptr.size()) - 1;
    const int4 *chk = reinterpret_cast<const int4 *>(c->chunks);
    for (int s = 0; s < 2 * nL; s++) {
      const int fwd = s < nL, L = fwd ? s : 2 * nL - 1 - s;
      const int nch = ptr[L + 1] - ptr[L];
      if (nch > 0)
        KL(c, "sptrsv_levels", c->stream, k_ldl_sweep<T>, nch, kChunkThreads, 0, c->S, chk + ptr[L], fwd, lv, uv,
           di, x, z, gate);
    }
    return;
  }
  const bool cheb = c->opt.c_solver == 1;
  if (std::max(P.levels_interior, P.levels_c) <= kShallowLevels) {
    if (c->lv_desc) desc_sweeps<T>(c, c->stream, "sptrsv_levels", lv, uv, di, x, z, gate);
    else chunk_sweeps<T>(c, c->stream, P.ch_all_ptr, "sptrsv_levels", lv, uv, di, x, z, gate);
    if (cheb) cheb_tail<T>(c, c->stream, x, z, 1, gate);
    else if (c->opt.c_solver == 2) mr_apply_c<T>(c, c->stream, x, z, 1, gate);
    return;
  }
  ck(cudaEventRecord(c->ev_fork, c->stream), "event");
  ck(cudaStreamWaitEvent(c->stream2, c->ev_fork, 0), "wait");
  if (P.p > 0) {
    const bool use = sizeof(T) == 8 ? c->use_tma64 : c->use_tma32;
    const TmaCfg &cfg = sizeof(T) == 8 ? c->tma64 : c->tma32;
    if (sizeof(T) == 8 ? c->use_sf64 : c->use_sf32) {
      KL(c, "sptrsv_blocks", c->stream, (k_sptrsv_blocks_sf<T, 256, 4>), P.p, 256, sf_smem_bytes<T>(P),
         c->blk_row0, RowSpan{c->l_span, c->u_span}, c->S.l_col, lv, c->S.u_col, uv, di, x, z, gate,
         c->dflag + 3, c->wait_ns);
    } else if (use) {
      KL(c, "sptrsv_blocks", c->stream, (k_sptrsv_blocks_tma<T, 256>), P.p, 256, tma_smem_bytes<T>(cfg),
         c->S, lv, uv, Prec<T>::dinvs(c), x, z, gate, cfg, c->dflag + 3, std::max(c->wait_ns, kTmaMinWaitNs));
    } else {
      KL(c, "sptrsv_blocks", c->stream, (k_sptrsv_blocks<T, 256>), P.p, 256, 0,
         c->S, lv, uv, di, x, z, gate);
    }
  }
  chunk_sweeps<T>(c, c->stream2, P.ch_c_ptr, "sptrsv_c", lv, uv, di, x, z, gate);
  if (cheb) cheb_tail<T>(c, c->stream2, x, z, 1, gate);
  else if (c->opt.c_solver == 2) mr_apply_c<T>(c, c->stream2, x, z, 1, gate);
  ck(cudaEventRecord(c->ev_join, c->stream2), "event");
  ck(cudaStreamWaitEvent(c->stream, c->ev_join, 0), "wait");
}

// ------------------------------------------------ U_k products
// Vector-load kernels (16-byte loads, several rows in flight per thread) when
// a row of U_k is 1..32 loads of 16 bytes; DDLR_UVEC=0 keeps the scalar ones.
constexpr int kUvecNT = 512, kUvecUnr = 4, kUrowsUnr = 4;


template <typename TU>
int uvec_lanes(ddlr_ctx *c, int k) {
  constexpr int E = Unpack16<TU>::E;
  if (!c->uvec || k % E) return 0;
  const int L = k / E;
  return (L == 1 || L == 2 || L == 4 || L == 8 || L == 16 || L == 32) ? L : 0;
}

// out = coef .* (U^T x) or H (U^T x) (rows of U = nrows): the vector kernel
// with the final reduction in its last CTA, else partials over kRedGrid CTAs
// and k_reduce_cols
template <typename T, typename TU>
void launch_utx(ddlr_ctx *c, long long nrows, int k, const TU *U, const T *x, T *part, const T *coef,
                const T *H, T *out, const int *gate) {
#define DDLR_UTX(Lc)                                                                                   \
  KL(c, "utx", c->stream, (k_utx_vec<T, TU, Lc, kUvecNT, kUvecUnr>), kRedGrid, kUvecNT, 0, nrows, U, x, part, \
     gate, c->udone, coef, H, out)
  switch (uvec_lanes<TU>(c, k)) {
    case 1: DDLR_UTX(1); return;
    case 2: DDLR_UTX(2); return;
    case 4: DDLR_UTX(4); return;
    case 8: DDLR_UTX(8); return;
    case 16: DDLR_UTX(16); return;
    case 32: DDLR_UTX(32); return;
    default:
      KL(c, "utx", c->stream, (k_utx_partial<T, TU, 256>), kRedGrid, 256, 0, int(nrows), k, U, x, part, gate);
      KL(c, "reduce", c->stream, k_reduce_cols<T>, 1, 256, k * sizeof(T), kRedGrid, k, part, coef, H, out, gate);
  }
#undef DDLR_UTX
}

// blocks of 256 threads for the row-dot kernels: enough warps for the rows,
// at most 16 CTAs per SM-equivalent of a 152-SM part
inline unsigned urows_grid(long long nrows, int L) {
  const long long rows_per_cta = (long long)(32 / L) * (kThreads / 32) * kUrowsUnr;
  return (unsigned)std::max<long long>(1, std::min<long long>((nrows + rows_per_cta - 1) / rows_per_cta, 152 * 16));
}

// FP64 row products: shared-memory tiles, thread per row (k even, k <= 64)
inline bool urows_smem(ddlr_ctx *c, int k) { return c->uvec && k % 2 == 0 && k <= 64; }
inline size_t urows_smem_bytes(int k) { return size_t(64 + kRowTile * (k + 1)) * sizeof(double); }
// thread-per-row direct kernels (k = 4, 8, 16, 32): one row per thread, at
// most 8 CTAs of 256 per SM-equivalent of a 152-SM part, grid-stride beyond
inline unsigned urows_direct_grid(long long nrows) {
  return (unsigned)std::max<long long>(1, std::min<long long>((nrows + kThreads - 1) / kThreads, 152 * 8));
}
inline unsigned urows_smem_grid(long long nrows) {
  return (unsigned)std::max<long long>(1, std::min<long long>((nrows + kRowTile - 1) / kRowTile, 152 * 8));
}

template <typename T, typename TU>
void launch_w_rhs(ddlr_ctx *c, int s, int m, int k, const TU *U, const T *t, const T *y, const T *inv1mt, T a,
                  const T *x, T *w, T *rhs, const int *gate) {
  if constexpr (std::is_same<T, double>::value && std::is_same<TU, double>::value) {
    const unsigned gd = urows_direct_grid(s);
    switch (c->uvec ? k : 0) {
      case 4: KL(c, "w_rhs", c->stream, k_w_rhs_direct<2>, gd, kThreads, 0, s, m, U, t, y, inv1mt, a, x, w, rhs, gate); return;
      case 8: KL(c, "w_rhs", c->stream, k_w_rhs_direct<4>, gd, kThreads, 0, s, m, U, t, y, inv1mt, a, x, w, rhs, gate); return;
      case 16: KL(c, "w_rhs", c->stream, k_w_rhs_direct<8>, gd, kThreads, 0, s, m, U, t, y, inv1mt, a, x, w, rhs, gate); return;
      case 32: KL(c, "w_rhs", c->stream, k_w_rhs_direct<16>, gd, kThreads, 0, s, m, U, t, y, inv1mt, a, x, w, rhs, gate); return;
      default: break;
    }
    if (urows_smem(c, k)) {
      KL(c, "w_rhs", c->stream, k_w_rhs_smem, urows_smem_grid(s), kRowTile, urows_smem_bytes(k), s, m, k, U, t,
         y, inv1mt, a, x, w, rhs, gate);
      return;
    }
  }
#define DDLR_WR(Lc)                                                                                    \
  KL(c, "w_rhs", c->stream, (k_w_rhs_vec<T, TU, Lc, kUrowsUnr>), urows_grid(s, Lc), kThreads, 0, s, m, U, t, y, \
     inv1mt, a, x, w, rhs, gate)
  switch (uvec_lanes<TU>(c, k)) {
    case 1: DDLR_WR(1); break;
    case 2: DDLR_WR(2); break;
    case 4: DDLR_WR(4); break;
    case 8: DDLR_WR(8); break;
    case 16: DDLR_WR(16); break;
    case 32: DDLR_WR(32); break;
    default:
      KL(c, "w_rhs", c->stream, (k_w_rhs<T, TU>), nblk(s), kThreads, k * sizeof(T), s, m, k, U, t, y, inv1mt, a,
         x, w, rhs, gate);
  }
#undef DDLR_WR
}

template <typename T, typename TU>
void launch_u_add(ddlr_ctx *c, long long n, int k, const TU *U, const T *h, T *u, const int *gate) {
  if constexpr (std::is_same<T, double>::value && std::is_same<TU, double>::value) {
    const unsigned gd = urows_direct_grid(n);
    switch (c->uvec ? k : 0) {
      case 4: KL(c, "u_add", c->stream, k_u_add_direct<2>, gd, kThreads, 0, n, U, h, u, gate); return;
      case 8: KL(c, "u_add", c->stream, k_u_add_direct<4>, gd, kThreads, 0, n, U, h, u, gate); return;
      case 16: KL(c, "u_add", c->stream, k_u_add_direct<8>, gd, kThreads, 0, n, U, h, u, gate); return;
      case 32: KL(c, "u_add", c->stream, k_u_add_direct<16>, gd, kThreads, 0, n, U, h, u, gate); return;
      default: break;
    }
    if (urows_smem(c, k)) {
      KL(c, "u_add", c->stream, k_u_add_smem, urows_smem_grid(n), kRowTile, urows_smem_bytes(k), n, k, U, h, u,
         gate);
      return;
    }
  }
#define DDLR_UA(Lc)                                                                                    \
  KL(c, "u_add", c->stream, (k_u_add_vec<T, TU, Lc, kUrowsUnr>), urows_grid(n, Lc), kThreads, 0, n, U, h, u, gate)
  switch (uvec_lanes<TU>(c, k)) {
    case 1: DDLR_UA(1); break;
    case 2: DDLR_UA(2); break;
    case 4: DDLR_UA(4); break;
    case 8: DDLR_UA(8); break;
    case 16: DDLR_UA(16); break;
    case 32: DDLR_UA(32); break;
    default:
      KL(c, "u_add", c->stream, (k_u_add<T, TU>), nblk(n), kThreads, k * sizeof(T), int(n), k, U, h, u, gate);
  }
#undef DDLR_UA
}

// ----------------------------------------------------------- M^-1 apply
// u = M^-1 x in device order.  DDLR-1: Algorithm 1 with prop. gkt;
// DDLR-2: eq. Form2a.  Uses workspaces 0..3 of precision T.
template <typename T, typename TU>
void apply_dev(ddlr_ctx *c, const TU *U, const T *x, T *u, const int *gate) {
  const Plan &P = c->P;
  const int n = P.n, m = P.m, s = P.s, k = c->opt.rank_k;
  const T a = T(c->opt.alpha), ia = T(1.0 / c->opt.alpha);
  T *part = Prec<T>::part(c);
  if (c->opt.variant == 1) {
    T *z = Prec<T>::w(c, 0), *y = Prec<T>::w(c, 1), *w = Prec<T>::w(c, 2), *rhs = Prec<T>::w(c, 3);
    T *t = Prec<T>::w(c, 4);
    a0_solve<T>(c, x, z, gate);                                      // A0 z = x
    KL(c, "et", c->stream, k_et<T>, nblk(s), kThreads, 0,            // y = E^T z
       s, m, c->eht_rp, c->eht_ci, Prec<T>::eht(c), ia, a, z, y, gate);
    launch_utx<T, TU>(c, s, k, U, y, part, Prec<T>::coef(c), (const T *)nullptr, t, gate);   // t = D U^T y
    launch_w_rhs<T, TU>(c, s, m, k, U, t, y, Prec<T>::inv1mt(c), a, x, w, rhs, gate);   // w, x_C - a w
    KL(c, "e_int", c->stream, k_e_interior<T>, nblk(m), kThreads, 0,
       m, c->eh_rp, c->eh_ci, Prec<T>::eh(c), ia, w, x, rhs, gate);   // x_B + a^-1 Ehat w
    a0_solve<T>(c, rhs, u, gate);                                    // A0 u = x + v
  } else {
    T *t = Prec<T>::w(c, 4);
    a0_solve<T>(c, x, u, gate);
    launch_utx<T, TU>(c, n, k, U, x, part, (const T *)nullptr, Prec<T>::Hk(c), t, gate);
    launch_u_add<T, TU>(c, n, k, U, t, u, gate);
  }
}

// the mixed-precision DDLR-1 apply without separate precision casts: for
// shallow factors solved by the descriptor sweeps, the factored C_a and
// vector U_k products, with no diagonal scaling (the casts are then plain
// roundings, done where the values are read and written)
bool mixed_fused(const ddlr_ctx *c) {
  const Plan &P = c->P;
  const int k = c->opt.rank_k;
  const int E = c->opt.uk_bf16 ? 8 : 4;                  // values per 16-byte load of U_k
  const int L = k / E;
  const bool lanes = k % E == 0 && (L == 1 || L == 2 || L == 4 || L == 8 || L == 16 || L == 32);
  const char *off = getenv("DDLR_NO_FUSED_CAST");
  return c->opt.precision == 1 && c->opt.variant == 1 && !c->dsc_dev && c->opt.c_solver == 0 &&
         c->opt.factor < 2 && c->lv_desc && std::max(P.levels_interior, P.levels_c) <= kShallowLevels &&
         c->uvec && lanes && !(off && off[0] == '1');
}

// DDLR-1 M^-1 x (Algorithm 1) in FP32 on an FP64 x, the result in FP64 u64:
// apply_dev<float, TU> with x rounded as it is read and the last sweeps
// writing FP64 (mixed_fused cases only)
template <typename TU>
void apply_dev_x64(ddlr_ctx *c, const TU *U, const double *x, double *u64, const int *gate) {
  const Plan &P = c->P;
  const int m = P.m, s = P.s, k = c->opt.rank_k;
  const float a = float(c->opt.alpha), ia = float(1.0 / c->opt.alpha);
  float *part = c->part32;
  float *z = c->w32[0], *y = c->w32[1], *w = c->w32[2], *rhs = c->w32[3], *t = c->w32[4], *u = c->w32[7];
  const float *lv = c->l32, *uv = c->u32, *di = c->dinv32;
  desc_sweeps<float, double>(c, c->stream, "sptrsv_levels", lv, uv, di, x, z, gate);     // A0 z = x
  KL(c, "et", c->stream, k_et<float>, nblk(s), kThreads, 0, s, m, c->eht_rp, c->eht_ci, c->eht32, ia, a, z, y,
     gate);                                                                               // y = E^T z
  launch_utx<float, TU>(c, s, k, U, y, part, c->coef32, (const float *)nullptr, t, gate);   // t = D U^T y
  constexpr int E = Unpack16<TU>::E;
#define DDLR_WRX(Lc)                                                                                          \
  KL(c, "w_rhs", c->stream, (k_w_rhs_vec<float, TU, Lc, kUrowsUnr, double>), urows_grid(s, Lc), kThreads, 0, s, m, \
     U, t, y, c->inv1mt32, a, x, w, rhs, gate)
  switch (k / E) {
    case 1: DDLR_WRX(1); break;
    case 2: DDLR_WRX(2); break;
    case 4: DDLR_WRX(4); break;
    case 8: DDLR_WRX(8); break;
    case 16: DDLR_WRX(16); break;
    case 32: DDLR_WRX(32); break;
    default: throw Fail{DDLR_ERR_INVALID, "fused mixed apply: unsupported rank"};
  }
#undef DDLR_WRX
  KL(c, "e_int", c->stream, (k_e_interior<float, double>), nblk(m), kThreads, 0, m, c->eh_rp, c->eh_ci, c->eh32, ia,
     w, x, rhs, gate);                                                                    // x_B + a^-1 Ehat w
  desc_sweeps<float, float>(c, c->stream, "sptrsv_levels", lv, uv, di, rhs, u, gate, u64);   // A0 u = x + v
}

// preconditioner on FP64 vectors in device order (scaled system handled here)
void precond(ddlr_ctx *c, const double *r, double *z, const int *gate) {
  const int n = c->P.n;
  const double *rin = r;
  if (c->dsc_dev) {
    KL(c, "vec", c->stream, k_mulv_t<double>, nblk(n), kThreads, 0, (long long)n, c->dsc_dev, r, c->w64[6], gate);
    rin = c->w64[6];
  }
  if (c->opt.precision == 0) {
    apply_dev<double, double>(c, c->U64, rin, z, gate);
  } else if (mixed_fused(c)) {
    // the FP32 preconditioner reads the FP64 residual and writes the FP64
    // result itself (no separate casts)
    if (c->opt.uk_bf16) apply_dev_x64<__nv_bfloat16>(c, c->Ub16, r, z, gate);
    else apply_dev_x64<float>(c, c->U32, r, z, gate);
  } else {
    float *r32 = c->w32[6], *z32 = c->w32[7];
    KL(c, "vec", c->stream, (k_cast<float, double>), nblk(n), kThreads, 0, (long long)n, rin, r32, gate);
    if (c->opt.uk_bf16) apply_dev<float, __nv_bfloat16>(c, c->Ub16, r32, z32, gate);
    else apply_dev<float, float>(c, c->U32, r32, z32, gate);
    KL(c, "vec", c->stream, (k_cast<double, float>), nblk(n), kThreads, 0, (long long)n, z32, z, gate);
  }
  if (c->dsc_dev)
    KL(c, "vec", c->stream, k_mulv_t<double>, nblk(n), kThreads, 0, (long long)n, c->dsc_dev, z, z, gate);
}

// persistent-kernel helpers (defined with the allocation code)
template <typename T, typename TU>
PzOp<T, TU> make_pzop(ddlr_ctx *c);
bool pz_launch(ddlr_ctx *c, const char *fam, const void *fn, size_t smem, void **args, int threads = kPzThreads);
size_t pz_lz_smem(int mmax);
[[noreturn]] void timeout_fail(ddlr_ctx *c);
void clear_timeout(ddlr_ctx *c);

// ------------------------------------------------------------- Lanczos
void sync(ddlr_ctx *c) { ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize"); }

void read_dev(ddlr_ctx *c, void *h, const void *d, size_t bytes) {
  ck(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, c->stream), "D2H");
  sync(c);
}

// one Lanczos step j (Sec. 4.4) with every scalar and index on the device:
// w = Op q_j; alpha_j; three-term update; full reorthogonalisation against
// Q_{j+1} (one classical Gram-Schmidt pass, a second one on cancellation);
// beta_j; breakdown decision; q_{j+1} (or a restart vector
// orthogonalised against Q_{j+1}); j += 1.  Kernels return at once once the
// stop flag is set.
struct LzBufs {
  double *Q, *al, *be, *cvec, *w, *qcur, *qprev, *nrm;
  int *rank;
  LzState *st;
  long long ld;
  int mmax;
};

void lanczos_step(ddlr_ctx *c, const LzBufs &L) {
  const Plan &P = c->P;
  const int n = P.n, m = P.m, s = P.s;
  const double a = c->opt.alpha, ia = 1.0 / a;
  const int *stop = reinterpret_cast<const int *>(reinterpret_cast<const char *>(L.st) + offsetof(LzState, stop));
  const int *nobrk = reinterpret_cast<const int *>(reinterpret_cast<const char *>(L.st) + offsetof(LzState, no_break));
  double *v = c->w64[0], *z = c->w64[1];
  const size_t csm = size_t(L.mmax + 2) * sizeof(double);
  KL(c, "e_vec", c->stream, k_e_vec<double>, nblk(n), kThreads, 0,
     m, s, c->eh_rp, c->eh_ci, c->eh64, ia, a, L.qcur, (const double *)nullptr, v, stop);
  a0_solve<double>(c, v, z, stop);
  if (c->opt.variant == 2) {
    a0_solve<double>(c, z, v, stop);
    std::swap(v, z);
  }
  KL(c, "et", c->stream, k_et<double>, nblk(s), kThreads, 0, s, m, c->eht_rp, c->eht_ci, c->eht64, ia, a, z,
     L.w, stop);
  KL(c, "dot", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, L.qcur, L.w,
     c->part64, stop);
  KL(c, "dot", c->stream, k_lz_reduce_at, 1, 32, 0, kRedGrid, c->part64, L.al, L.st, 0, stop);
  KL(c, "lanczos", c->stream, k_lz_three_term_d, nblk(s), kThreads, 0, s, L.al, L.be, L.st, L.qcur, L.qprev, L.w);
  // one classical Gram-Schmidt pass against Q_{j+1}; skipped when *gate != 0
  // or *gate_inv == 0
  auto cgs_pass = [&](const int *gate, const int *gate_inv) {
    KL(c, "cgs2", c->stream, k_gemvT_partial_d<256>, kRedGrid, 256, 0, s, L.Q, L.ld, L.w, c->part64, L.st,
       gate, gate_inv);
    KL(c, "cgs2", c->stream, k_reduce_cols_d, (L.mmax + 8) / 8, 256, 0, kRedGrid, c->part64, L.cvec, L.st, gate,
       gate_inv);
    KL(c, "cgs2", c->stream, k_gemvN_sub_d, nblk(s), kThreads, csm, s, L.Q, L.ld, L.cvec, L.w, L.st, gate,
       gate_inv);
  };
  auto wnorm2 = [&](double *out, const int *gate) {
    KL(c, "dot", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, L.w, L.w, c->part64, gate);
    KL(c, "dot", c->stream, k_reduce_scalar, 1, 32, 0, kRedGrid, c->part64, out, 0, gate);
  };
  // full reorthogonalisation: the second pass when the first left less than
  // half of ||w||^2 (or always, lanczos_reorth 1)
  const int *pass2 = reinterpret_cast<const int *>(reinterpret_cast<const char *>(L.st) + offsetof(LzState, pass2));
  wnorm2(L.nrm + 2, stop);
  cgs_pass(stop, nullptr);
  wnorm2(L.nrm + 3, stop);
  KL(c, "lanczos", c->stream, k_lz_dgks, 1, 32, 0, L.st, L.nrm + 2, c->opt.lanczos_reorth);
  cgs_pass(stop, pass2);
  KL(c, "dot", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, L.w, L.w, c->part64, stop);
  KL(c, "dot", c->stream, k_lz_reduce_at, 1, 32, 0, kRedGrid, c->part64, L.be, L.st, 1, stop);
  KL(c, "lanczos", c->stream, k_lz_decide, 1, 32, 0, L.st, L.al, L.be);
  KL(c, "lanczos", c->stream, k_lz_normalize, nblk(s), kThreads, 0, s, L.w, L.be, L.Q, L.ld, L.qcur, L.qprev, L.st);
  // breakdown: restart from a fresh vector orthogonalised against Q_{j+1}
  KL(c, "lanczos", c->stream, k_lz_randvec, nblk(s), kThreads, 0, s, L.rank, L.st, L.w);
  cgs_pass(nobrk, nullptr);
  cgs_pass(nobrk, nullptr);
  KL(c, "dot", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, L.w, L.w, c->part64, nobrk);
  KL(c, "dot", c->stream, k_reduce_scalar, 1, 32, 0, kRedGrid, c->part64, L.nrm, 1, nobrk);
  KL(c, "lanczos", c->stream, k_lz_restart_norm, nblk(s), kThreads, 0, s, L.w, L.nrm, L.Q, L.ld, L.qcur, L.qprev,
     L.be, L.st);
  KL(c, "lanczos", c->stream, k_lz_advance, 1, 32, 0, L.st);
}

void hk_finalize(ddlr_ctx *c, int k, const double *kp, double *hw);
ddlr_status lowrank_status(ddlr_ctx *c, const int *fl);

// Lanczos with full reorthogonalisation and the convergence test of
// eq. converge every `check` steps (Sec. 4.4, Sec. 5).  The host enqueues the
// steps (one CUDA graph each) without waiting; each test runs on the second
// stream while later steps proceed, and sets the device stop flag when met;
// the host reads that flag once per test, one test later.
// resume: continue the process from the device state (more steps for a
// larger k, Sec. 3.4) instead of starting from q_1
ddlr_status run_lanczos(ddlr_ctx *c, bool resume = false) {
  const Plan &P = c->P;
  const int s = P.s, n = P.n, m0 = P.m, k = c->opt.rank_k;
  int mmax = c->opt.lanczos_max > 0 ? c->opt.lanczos_max : 5 * k;
  mmax = std::min(mmax, s);
  mmax = std::max(mmax, k);
  const int check = c->opt.lanczos_check;
  const double eps = c->opt.lanczos_eps;
  auto &W = c->lw;
  cudaStream_t user = c->stream;
  ddlr_status st = DDLR_OK;
  try {
    if (!W.ready) {
      // first run: workspace for m_max steps, the rank of every interface node
      // in ascending original index and the start vector (SplitMix64 stream
      // `seed` drawn in that order, normalised); refactors reuse them
      W.Q = c->alloc<double>(size_t(s) * size_t(mmax + 1));
      W.al = c->alloc<double>(mmax + 1);
      W.be = c->alloc<double>(mmax + 1);
      W.cvec = c->alloc<double>(mmax + 2);
      W.w = c->alloc<double>(s);
      W.qcur = c->alloc<double>(s);
      W.qprev = c->alloc<double>(s);
      W.q0 = c->alloc<double>(s);
      W.nrm = c->alloc<double>(4);
      W.rank = c->alloc<int>(s);
      W.st = c->alloc<LzState>(1);
      W.ework = c->alloc<double>(5 * size_t(mmax) * k);
      W.etop = c->alloc<double>(2 * k + 1);
      W.evals = c->alloc<double>(mmax);
      W.esum = c->alloc<double>(2);
      W.eY = c->alloc<double>(size_t(mmax) * k);
      if (c->opt.variant == 2) {
        W.V = c->alloc<double>(size_t(s) * k);
        W.EV = c->alloc<double>(size_t(n) * k);
        W.vc = c->alloc<double>(s);
        W.ev = c->alloc<double>(n);
        W.uc = c->alloc<double>(n);
        W.kp = c->alloc<double>(size_t(kRedGrid) * k * k);
        W.hw = c->alloc<double>(size_t(k) * k + k);
      }
      ck(cudaMallocHost(&W.h_st, sizeof(LzState)), "cudaMallocHost");
      ck(cudaEventCreateWithFlags(&W.ev_chk, cudaEventDisableTiming), "event");
      ck(cudaEventCreateWithFlags(&W.ev_done, cudaEventDisableTiming), "event");
      const auto &rank = P.iface_rank;
      std::vector<double> byrank(s), hv(s);
      double nn = 0;
      for (int r = 0; r < s; r++) { byrank[r] = sm64_pm1(c->opt.seed, (uint64_t)r); nn += byrank[r] * byrank[r]; }
      nn = std::sqrt(nn);
      for (int j = 0; j < s; j++) hv[j] = byrank[rank[j]] / nn;
      ck(cudaMemcpyAsync(W.q0, hv.data(), sizeof(double) * s, cudaMemcpyHostToDevice, c->stream), "H2D");
      ck(cudaMemcpyAsync(W.rank, rank.data(), sizeof(int) * s, cudaMemcpyHostToDevice, c->stream), "H2D");
      ck(cudaStreamSynchronize(c->stream), "sync");     // host vectors above are locals
      W.ready = true;
    }
    LzBufs L;
    L.mmax = mmax;
    L.ld = s;
    L.Q = W.Q; L.al = W.al; L.be = W.be; L.cvec = W.cvec; L.w = W.w; L.qcur = W.qcur; L.qprev = W.qprev;
    L.nrm = W.nrm; L.rank = W.rank; L.st = W.st;
    double *ework = W.ework, *etop = W.etop, *evals = W.evals, *esum = W.esum, *eY = W.eY;
    cudaEvent_t ev_chk = W.ev_chk, ev_done = W.ev_done;
    LzState &h0 = *W.h_st;
    int j_start = 0;
    if (resume) {
      // the state after the last step (j, scale, restarts, q_j, q_{j-1}, T_j)
      // with the new step limit; a convergence met before is tested again
      ck(cudaMemcpyAsync(&h0, L.st, sizeof(h0), cudaMemcpyDeviceToHost, c->stream), "D2H");
      ck(cudaStreamSynchronize(c->stream), "sync");
      if (h0.nan_step >= 0) throw Fail{DDLR_ERR_NAN, "the Lanczos process met a NaN; set up again"};
      h0.mmax = mmax;
      h0.stop = h0.j >= mmax ? 1 : 0;
      h0.no_break = 1;
      h0.conv_m = 0;
      j_start = h0.j;
    } else {
      ck(cudaMemsetAsync(L.be, 0, sizeof(double) * (mmax + 1), c->stream), "memset");
      ck(cudaMemsetAsync(L.qprev, 0, sizeof(double) * s, c->stream), "memset");
      ck(cudaMemcpyAsync(L.Q, W.q0, sizeof(double) * s, cudaMemcpyDeviceToDevice, c->stream), "copy");
      ck(cudaMemcpyAsync(L.qcur, W.q0, sizeof(double) * s, cudaMemcpyDeviceToDevice, c->stream), "copy");
      h0 = LzState{};
      h0.j = 0; h0.stop = 0; h0.no_break = 1; h0.restarts = 0; h0.conv_m = 0; h0.nan_step = -1;
      h0.mmax = mmax; h0.scale = 0.0; h0.seed = c->opt.seed;
    }
    ck(cudaMemcpyAsync(L.st, &h0, sizeof(h0), cudaMemcpyHostToDevice, c->stream), "H2D");

    const char *ng = getenv("DDLR_NO_GRAPH");
    // every step and test in one persistent kernel when the factors are shallow
    const int nLz = int(P.ch_all_ptr.size()) - 1;
    bool persist = c->pz_lz && mmax <= c->pz_mmax &&
                   (long long)mmax * (4 * (2 * nLz - 1) + 16) * c->pz_grid < (1LL << 31);
    if (persist) {
      // the kernel fills the FP32 copy of the basis from Q when it starts
      if (!W.Q32) W.Q32 = c->alloc<float>(size_t(s) * size_t(mmax + 1));
      PzOp<double, double> O = make_pzop<double, double>(c);
      PzLz Lz{L.Q, L.ld, L.al, L.be, L.w, L.qcur, L.qprev, c->w64[0], c->w64[1], etop, L.rank, L.st, check, k, eps,
              c->opt.lanczos_reorth, W.Q32};
      void *args[] = {&O, &Lz};
      persist = pz_launch(c, "lanczos_persist", (const void *)k_lz_persist<kPzLzThreads>, pz_lz_smem(c->pz_mmax),
                          args, kPzLzThreads);
    }
    const bool use_graph = !persist && !c->timing && !(ng && ng[0] == '1');
    if (use_graph) {
      ck(cudaEventRecord(c->ev_fork, user), "event");
      ck(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0), "wait");
      c->stream = c->gstream;
      if (!W.exec) {
        const long long l0 = c->launches;
        const std::vector<long long> f0 = c->fam_cnt;
        ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture");
        lanczos_step(c, L);
        cudaGraph_t g = nullptr;
        ck(cudaStreamEndCapture(c->stream, &g), "capture");
        cudaError_t e = cudaGraphInstantiate(&W.exec, g, 0);
        cudaGraphDestroy(g);
        ck(e, "cudaGraphInstantiate");
        c->lz_nodes = c->launches - l0;
        c->lz_fam_nodes.assign(c->fam_cnt.size(), 0);
        for (size_t i = 0; i < c->fam_cnt.size(); i++) c->lz_fam_nodes[i] = c->fam_cnt[i] - (i < f0.size() ? f0[i] : 0);
        c->launches = l0;
        for (size_t i = 0; i < f0.size(); i++) c->fam_cnt[i] = f0[i];
        for (size_t i = f0.size(); i < c->fam_cnt.size(); i++) c->fam_cnt[i] = 0;
      }
    }
    int *hstop = reinterpret_cast<int *>(c->h_pin + 8);
    bool pending = false;
    for (int j = j_start; j < (persist ? 0 : mmax); j++) {
      if (use_graph) {
        ck(cudaGraphLaunch(W.exec, c->stream), "cudaGraphLaunch");
        c->launches += c->lz_nodes;
        for (size_t i = 0; i < c->lz_fam_nodes.size(); i++) c->fam_cnt[i] += c->lz_fam_nodes[i];
      } else {
        lanczos_step(c, L);
      }
      const int mm = j + 1;
      if (check > 0 && mm % check == 0 && mm >= k + 1 && mm < mmax) {
        if (pending) {
          ck(cudaEventSynchronize(ev_done), "event");
          if (*hstop) break;                 // converged at an earlier test
        }
        ck(cudaEventRecord(ev_chk, c->stream), "event");
        ck(cudaStreamWaitEvent(c->stream2, ev_chk, 0), "wait");
        const size_t smk = (2 * mm + 2) * sizeof(double);
        KL(c, "eig_check", c->stream2, k_tridiag_values, k, kEigPoints, smk, mm, L.al, L.be, k, etop);
        KL(c, "eig_check", c->stream2, k_sum_first, 1, 32, 0, k, etop, esum);
        KL(c, "eig_check", c->stream2, k_tridiag_values, k, kEigPoints, smk, mm - 1, L.al, L.be, k, etop);
        KL(c, "eig_check", c->stream2, k_sum_first, 1, 32, 0, k, etop, esum + 1);
        KL(c, "eig_check", c->stream2, k_lz_converged, 1, 32, 0, esum, eps, mm, L.st);
        ck(cudaMemcpyAsync(hstop, reinterpret_cast<const char *>(L.st) + offsetof(LzState, stop), sizeof(int),
                           cudaMemcpyDeviceToHost, c->stream2), "D2H");
        ck(cudaEventRecord(ev_done, c->stream2), "event");
        pending = true;
      }
    }
    ck(cudaStreamSynchronize(c->stream2), "sync");
    ck(cudaStreamSynchronize(c->stream), "sync");
    if (use_graph) {
      ck(cudaEventRecord(c->ev_join, c->stream), "event");
      ck(cudaStreamWaitEvent(user, c->ev_join, 0), "wait");
      c->stream = user;
    }
    LzState hs;
    ck(cudaMemcpy(&hs, L.st, sizeof(hs), cudaMemcpyDeviceToHost), "D2H");
    if (persist) {
      // per step: E q, one (DDLR-2: two) A0 solves, E^T, the three-term update
      // and normalisation (with the FP32 copy of q_{j+1}), and the CGS passes:
      // the basis columns they read in FP64 and in FP32, as counted on the
      // device
      double a0 = 0;
      ddlr_get_traffic(c, nullptr, &a0, nullptr, 0);
      const double ne = double(P.nnz_ehat), sd = double(s) * 8.0, nd = double(n) * 8.0;
      const double step = ne * 12.0 + sd + nd + (c->opt.variant == 2 ? 2.0 : 1.0) * a0 + ne * 12.0 + nd + sd +
                          8.0 * sd;
      const double steps = double(hs.j);
      c->pz_lz_bytes += steps * (step + 4.0 * s) + sd * hs.qcols64 + 4.0 * s * hs.qcols32;
      c->pz_lz_runs += 1;
    }
    c->lz_passes = hs.j + hs.npass2;
    c->lz_fp32 = persist ? hs.nfp32 : 0;
    {
      // a bounded wait of the persistent kernel ran out: the state is not
      // that of a finished process
      int fl[4];
      read_dev(c, fl, c->dflag, sizeof(fl));
      if (fl[3]) {
        clear_timeout(c);
        c->err = "a bounded device wait timed out";
        return DDLR_ERR_TIMEOUT;
      }
    }
    const int mm = hs.conv_m > 0 ? hs.conv_m : std::min(hs.j, mmax);
    if (hs.nan_step >= 0 && hs.nan_step < mm) st = DDLR_ERR_NAN;
    if (st == DDLR_OK && mm < 1) throw Fail{DDLR_ERR_BREAKDOWN, "the Lanczos process took no step"};
    if (st == DDLR_OK) {
      c->msteps = mm;
      const int nvals = mm;
      KL(c, "eig", c->stream, k_tridiag_values, nvals, kEigPoints, (2 * mm + 2) * sizeof(double), mm, L.al, L.be,
         nvals, evals);
      KL(c, "eig", c->stream, k_tridiag_vectors, 1, 256, 0, mm, L.al, L.be, k, evals, eY, ework);
      c->ritz.assign(nvals, 0.0);
      read_dev(c, c->ritz.data(), evals, sizeof(double) * nvals);
      const double *Q = L.Q;
      if (c->opt.variant == 1) {
        KL(c, "ritz", c->stream, k_ritz_gemm<16>, nblk(s), kThreads, 0, s, mm, k, Q, (long long)s, eY, c->U64);
        KL(c, "ritz", c->stream, k_ddlr1_coef, 1, 32, 0, mm, k, c->opt.theta_mode, evals,
           c->theta_d, c->inv1mt64, c->coef64, c->dflag + 1);
        read_dev(c, &c->theta, c->theta_d, sizeof(double));
      } else {
        // V_k = Q_m Y_k; U_k = A0^-1 E V_k; H_k = (I - U_k^T E V_k)^-1
        double *V = W.V, *EV = W.EV, *vc = W.vc, *ev = W.ev, *uc = W.uc, *kp = W.kp, *hw = W.hw;
        KL(c, "ritz", c->stream, k_ritz_gemm<16>, nblk(s), kThreads, 0, s, mm, k, Q, (long long)s, eY, V);
        const double a = c->opt.alpha;
        for (int cc = 0; cc < k; cc++) {
          KL(c, "ritz", c->stream, k_get_col, nblk(s), kThreads, 0, (long long)s, k, cc, V, vc);
          KL(c, "e_vec", c->stream, k_e_vec<double>, nblk(n), kThreads, 0, m0, s, c->eh_rp, c->eh_ci,
             c->eh64, 1.0 / a, a, vc, (const double *)nullptr, ev, (const int *)nullptr);
          KL(c, "ritz", c->stream, k_set_col, nblk(n), kThreads, 0, (long long)n, k, cc, ev, EV);
          a0_solve<double>(c, ev, uc, nullptr);
          KL(c, "ritz", c->stream, k_set_col, nblk(n), kThreads, 0, (long long)n, k, cc, uc, c->U64);
        }
        KL(c, "ritz", c->stream, k_utv_partial, kRedGrid, 256, 0, (long long)n, k, c->U64, EV, kp);
        hk_finalize(c, k, kp, hw);
        c->theta = 0.0;
      }
      int fl[4];
      read_dev(c, fl, c->dflag, sizeof(fl));
      st = lowrank_status(c, fl);
    }
    sync(c);
  } catch (...) {
    c->stream = user;
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->stream2);
    cudaStreamSynchronize(c->gstream);
    throw;
  }
  return st;
}

void lowrank_to_low_precision(ddlr_ctx *c) {
  if (c->opt.precision == 0) return;
  const int k = c->opt.rank_k;
  const long long nu = (long long)c->urows * k;
  if (c->opt.uk_bf16)
    KL(c, "setup", c->stream, k_to_bf16, nblk(nu), kThreads, 0, nu, c->U64, c->Ub16);
  else
    KL(c, "setup", c->stream, (k_cast<float, double>), nblk(nu), kThreads, 0, nu, c->U64, c->U32, (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), 1, kThreads, 0, (long long)k, c->coef64, c->coef32, (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), 1, kThreads, 0, 1LL, c->inv1mt64, c->inv1mt32, (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk((long long)k * k), kThreads, 0, (long long)k * k, c->Hk64, c->Hk32, (const int *)nullptr);
}

// FP32 / BF16 copies used by the mixed-precision preconditioner
void make_low_precision(ddlr_ctx *c) {
  const Plan &P = c->P;
  if (c->opt.precision == 0) return;
  const long long ll = (long long)P.l_col.size(), lu = (long long)P.u_col.size();
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(ll), kThreads, 0, ll, c->l64, c->l32, (const int *)nullptr);
  if (c->lx32)
    KL(c, "setup", c->stream, (k_cast<float, double>), nblk(ll), kThreads, 0, ll, c->lx64, c->lx32,
       (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(lu), kThreads, 0, lu, c->u64, c->u32, (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(P.n), kThreads, 0, (long long)P.n, c->dinv64, c->dinv32, (const int *)nullptr);
  const long long nds = (long long)P.nslice * kSlice;
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(nds), kThreads, 0, nds, c->dinvs64, c->dinvs32, (const int *)nullptr);
  const long long ne = (long long)P.eh_ci.size();
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(ne), kThreads, 0, ne, c->eh64, c->eh32, (const int *)nullptr);
  KL(c, "setup", c->stream, (k_cast<float, double>), nblk(ne), kThreads, 0, ne, c->eht64, c->eht32, (const int *)nullptr);
  lowrank_to_low_precision(c);
}

}  // namespace

namespace {

const int *pcg_gate(ddlr_ctx *c) {
  return reinterpret_cast<const int *>(reinterpret_cast<const char *>(c->pcg) +
                                       offsetof(PcgState, done));
}

void batch_alloc(ddlr_ctx *c, int R);
template <typename T>
void a0_solve_mr(ddlr_ctx *c, const T *X, T *Z, int R, const int *gate);

// H_k = (I - U_k^T E V_k)^-1 for DDLR-2 from the k_utv_partial partials:
// Cholesky (an I - K that is not positive definite sets the NOT_SPD flag,
// prop. spd-2) or, in the indefinite mode, Gauss-Jordan with partial pivoting
// (a singular I - K sets the same flag, read as BREAKDOWN)
void hk_finalize(ddlr_ctx *c, int k, const double *kp, double *hw) {
  if (c->opt.indefinite)
    KL(c, "ritz", c->stream, k_hk_finalize_gj, 1, 32, 0, kRedGrid, k, kp, hw, c->Hk64, c->dflag + 1);
  else
    KL(c, "ritz", c->stream, k_hk_finalize, 1, 32, 0, kRedGrid, k, kp, hw, c->Hk64, c->dflag + 1);
}

// status of a finished low-rank build from the device flags (timeout, NaN,
// not SPD).  In the indefinite mode DDLR-1 keeps Ritz values >= 1 (the flag
// of k_ddlr1_coef is ignored) and only needs G_{k,theta} invertible:
// 1 - lambda_i and 1 - theta away from zero; DDLR-2's flag then means a
// singular I - K.  Both are BREAKDOWN.
ddlr_status lowrank_status(ddlr_ctx *c, const int *fl) {
  if (fl[3]) { clear_timeout(c); return DDLR_ERR_TIMEOUT; }
  if (fl[2]) return DDLR_ERR_NAN;
  if (!c->opt.indefinite) return fl[1] ? DDLR_ERR_NOT_SPD : DDLR_OK;
  if (c->opt.variant == 2) return fl[1] ? DDLR_ERR_BREAKDOWN : DDLR_OK;
  const int k = c->opt.rank_k;
  bool sing = !(std::fabs(1.0 - c->theta) > 1e-12);
  for (int i = 0; i < k && i < int(c->ritz.size()); i++) sing |= !(std::fabs(1.0 - c->ritz[i]) > 1e-12);
  for (double v : c->ritz)
    if (!std::isfinite(v)) return DDLR_ERR_NAN;
  return sing ? DDLR_ERR_BREAKDOWN : DDLR_OK;
}

const char *lowrank_error(ddlr_ctx *c, ddlr_status st) {
  switch (st) {
    case DDLR_ERR_NOT_SPD: return "preconditioner is not SPD (lambda_max >= 1 or I - K not PD)";
    case DDLR_ERR_BREAKDOWN:
      return c->opt.indefinite ? "G_{k,theta} or I - K is singular, or the low-rank process stopped early"
                               : "the low-rank process stopped before k steps";
    case DDLR_ERR_TIMEOUT: return "a bounded device wait timed out";
    default: return "NaN/Inf in the low-rank build";
  }
}

// Lanczos bidiagonalisation of K = A0^-1 E for DDLR-2 (ddlr_lbd.cuh): the
// steps run kernel by kernel with the scalars on the device; the host reads
// alpha_j and beta_j only for the stop decisions (breakdown, step limit, the
// eq. converge test on B_m^T B_m every lanczos_check steps, as for Lanczos)
ddlr_status run_lbd(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int n = P.n, m0 = P.m, s = P.s, k = c->opt.rank_k;
  int mmax = c->opt.lanczos_max > 0 ? c->opt.lanczos_max : 5 * k;
  mmax = std::max(std::min(mmax, s), k);
  const int check = c->opt.lanczos_check;
  const double eps = c->opt.lanczos_eps, a = c->opt.alpha;
  auto &B = c->lb;
  if (!B.ready) {
    B.mmax = mmax;
    B.Vq = c->alloc<double>(size_t(s) * (mmax + 1));
    B.Uq = c->alloc<double>(size_t(n) * mmax);
    B.al = c->alloc<double>(mmax + 1); B.be = c->alloc<double>(mmax + 1);
    B.td = c->alloc<double>(mmax + 1); B.te = c->alloc<double>(mmax + 1);
    B.t = c->alloc<double>(n); B.u = c->alloc<double>(n); B.v = c->alloc<double>(s);
    B.cpart = c->alloc<double>(size_t(kRedGrid) * (mmax + 2));
    B.cvec = c->alloc<double>(mmax + 2);
    B.evals = c->alloc<double>(mmax);
    B.eY = c->alloc<double>(size_t(mmax) * k);
    B.work = c->alloc<double>(size_t(5) * mmax * k);
    B.esum = c->alloc<double>(2);
    B.etop = c->alloc<double>(2 * size_t(k));
    B.G = c->alloc<double>(size_t(mmax) * k);
    B.Vk = c->alloc<double>(size_t(s) * k);
    B.EV = c->alloc<double>(size_t(n) * k);
    B.vc = c->alloc<double>(s); B.ev = c->alloc<double>(n);
    B.kp = c->alloc<double>(size_t(kRedGrid) * k * k);
    B.hw = c->alloc<double>(size_t(k) * k + k);
    // start vector: the Lanczos one (SplitMix64 stream seed over the
    // interface nodes in ascending original index, normalised)
    const auto &rank = P.iface_rank;
    std::vector<double> byrank(s), hv(s);
    double nn = 0;
    for (int r = 0; r < s; r++) { byrank[r] = sm64_pm1(c->opt.seed, (uint64_t)r); nn += byrank[r] * byrank[r]; }
    nn = std::sqrt(nn);
    for (int j = 0; j < s; j++) hv[j] = byrank[rank[j]] / nn;
    B.q0 = c->upload(hv);
    ck(cudaStreamSynchronize(c->stream), "sync");
    B.ready = true;
  }
  auto cgs2 = [&](long long rows, int ncol, const double *Q, double *w) {
    if (ncol <= 0) return;
    for (int pass = 0; pass < 2; pass++) {
      KL(c, "lbd_cgs", c->stream, k_cgs_partial<256>, kRedGrid, 256, 0, rows, ncol, Q, rows, w, B.cpart);
      KL(c, "lbd_cgs", c->stream, k_cgs_reduce, (ncol * 32 + 255) / 256, 256, 0, kRedGrid, ncol, B.cpart, B.cvec);
      KL(c, "lbd_cgs", c->stream, k_cgs_sub, nblk(rows), kThreads, ncol * sizeof(double), rows, ncol, Q, rows,
         B.cvec, w);
    }
  };
  auto norm = [&](long long rows, const double *x, double *out) {
    KL(c, "lbd", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, rows, x, x, c->part64,
       (const int *)nullptr);
    KL(c, "lbd", c->stream, k_cheb_reduce_norm, 1, 32, 0, kRedGrid, c->part64, out);
  };
  ck(cudaMemcpyAsync(B.Vq, B.q0, sizeof(double) * s, cudaMemcpyDeviceToDevice, c->stream), "D2D");
  double scale = 0.0;
  int mm = 0;
  for (int j = 0; j < mmax; j++) {
    const double *vj = B.Vq + (size_t)j * s;
    double *uj = B.Uq + (size_t)j * n;
    // u = K v_j - beta_{j-1} u_{j-1}, reorthogonalised; alpha_j = ||u||
    KL(c, "lbd", c->stream, k_e_vec<double>, nblk(n), kThreads, 0, m0, s, c->eh_rp, c->eh_ci, c->eh64, 1.0 / a, a,
       vj, (const double *)nullptr, B.t, (const int *)nullptr);
    a0_solve<double>(c, B.t, B.u, nullptr);
    if (j > 0) KL(c, "lbd", c->stream, k_lbd_axpy, nblk(n), kThreads, 0, (long long)n, B.be + j - 1, uj - n, B.u);
    cgs2(n, j, B.Uq, B.u);
    norm(n, B.u, B.al + j);
    double aj = 0;
    read_dev(c, &aj, B.al + j, sizeof(double));
    if (!std::isfinite(aj)) { c->err = "NaN/Inf in the bidiagonalisation"; return DDLR_ERR_NAN; }
    scale = std::max(scale, aj);
    if (!(aj > 1e-12 * scale)) break;          // K v_j in the span of U_{j-1}
    mm = j + 1;
    KL(c, "lbd", c->stream, k_lbd_scale, nblk(n), kThreads, 0, (long long)n, B.u, B.al + j, uj);
    // v = K^T u_j - alpha_j v_j, reorthogonalised; beta_j = ||v||
    a0_solve<double>(c, uj, B.t, nullptr);
    KL(c, "lbd", c->stream, k_et<double>, nblk(s), kThreads, 0, s, m0, c->eht_rp, c->eht_ci, c->eht64, 1.0 / a, a,
       B.t, B.v, (const int *)nullptr);
    KL(c, "lbd", c->stream, k_lbd_axpy, nblk(s), kThreads, 0, (long long)s, B.al + j, vj, B.v);
    cgs2(s, j + 1, B.Vq, B.v);
    norm(s, B.v, B.be + j);
    double bj = 0;
    read_dev(c, &bj, B.be + j, sizeof(double));
    if (!std::isfinite(bj)) { c->err = "NaN/Inf in the bidiagonalisation"; return DDLR_ERR_NAN; }
    scale = std::max(scale, bj);
    if (check > 0 && mm % check == 0 && mm >= k + 1) {
      // eq. converge on the k largest eigenvalues of B^T B for m and m - 1
      const size_t sm1 = (2 * size_t(mm) + 2) * sizeof(double);
      KL(c, "lbd", c->stream, k_lbd_tri, nblk(mm), kThreads, 0, mm, B.al, B.be, B.td, B.te);
      KL(c, "lbd", c->stream, k_tridiag_values, k, kEigPoints, sm1, mm, B.td, B.te, k, B.etop);
      KL(c, "lbd", c->stream, k_sum_first, 1, 32, 0, k, B.etop, B.esum);
      KL(c, "lbd", c->stream, k_tridiag_values, k, kEigPoints, sm1, mm - 1, B.td, B.te, k, B.etop + k);
      KL(c, "lbd", c->stream, k_sum_first, 1, 32, 0, k, B.etop + k, B.esum + 1);
      double sg[2];
      read_dev(c, sg, B.esum, sizeof(sg));
      if (std::fabs(sg[0] - sg[1]) < eps * std::fabs(sg[1])) break;
    }
    if (mm == mmax || !(bj > 1e-12 * scale)) break;
    KL(c, "lbd", c->stream, k_lbd_scale, nblk(s), kThreads, 0, (long long)s, B.v, B.be + j, B.Vq + (size_t)(j + 1) * s);
  }
  if (mm < k) {
    c->err = "the bidiagonalisation ended before k steps (rank of A0^-1 E below k)";
    return DDLR_ERR_BREAKDOWN;
  }
  // eigenpairs of B_m^T B_m; V_k = V_m Y_k; U_k = U_m (B_m Y_k)
  KL(c, "lbd", c->stream, k_lbd_tri, nblk(mm), kThreads, 0, mm, B.al, B.be, B.td, B.te);
  KL(c, "eig", c->stream, k_tridiag_values, mm, kEigPoints, (2 * mm + 2) * sizeof(double), mm, B.td, B.te, mm,
     B.evals);
  KL(c, "eig", c->stream, k_tridiag_vectors, 1, 256, 0, mm, B.td, B.te, k, B.evals, B.eY, B.work);
  c->msteps = mm;
  c->ritz.assign(mm, 0.0);
  read_dev(c, c->ritz.data(), B.evals, sizeof(double) * mm);
  KL(c, "ritz", c->stream, k_ritz_gemm<16>, nblk(s), kThreads, 0, s, mm, k, B.Vq, (long long)s, B.eY, B.Vk);
  KL(c, "ritz", c->stream, k_lbd_bmy, nblk((long long)mm * k), kThreads, 0, mm, k, B.al, B.be, B.eY, B.G);
  KL(c, "ritz", c->stream, k_ritz_gemm<16>, nblk(n), kThreads, 0, n, mm, k, B.Uq, (long long)n, B.G, c->U64);
  // H_k = (I - U_k^T E V_k)^-1
  ck(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), c->stream), "memset");
  for (int cc = 0; cc < k; cc++) {
    KL(c, "ritz", c->stream, k_get_col, nblk(s), kThreads, 0, (long long)s, k, cc, B.Vk, B.vc);
    KL(c, "e_vec", c->stream, k_e_vec<double>, nblk(n), kThreads, 0, m0, s, c->eh_rp, c->eh_ci, c->eh64, 1.0 / a, a,
       B.vc, (const double *)nullptr, B.ev, (const int *)nullptr);
    KL(c, "ritz", c->stream, k_set_col, nblk(n), kThreads, 0, (long long)n, k, cc, B.ev, B.EV);
  }
  KL(c, "ritz", c->stream, k_utv_partial, kRedGrid, 256, 0, (long long)n, k, c->U64, B.EV, B.kp);
  hk_finalize(c, k, B.kp, B.hw);
  c->theta = 0.0;
  int fl[4];
  read_dev(c, fl, c->dflag, sizeof(fl));
  const ddlr_status fst = lowrank_status(c, fl);
  if (fst != DDLR_OK) return fst;
  sync(c);
  return DDLR_OK;
}

// Randomized subspace iteration for the low-rank part (ddlr_rand.cuh):
// Omega -> Q = orth(Op Omega), q power steps, B = Q^T Op Q, eigenpairs of B,
// then U_k / Lambda_k / theta (DDLR-1) or V_k -> U_k = A0^-1 E V_k, H_k
// (DDLR-2) as after Lanczos.  Op on a block = batched E, A0 solve(s), E^T.
ddlr_status run_randomized(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int n = P.n, m = P.m, s = P.s, k = c->opt.rank_k;
  const int L = std::min(k + c->opt.rand_oversample, s);
  auto &R = c->rw;
  if (!R.ready) {
    R.L = L;
    R.Yb = c->alloc<double>(size_t(s) * L);
    R.Qb = c->alloc<double>(size_t(s) * L);
    R.V = c->alloc<double>(size_t(n) * L);
    R.Z = c->alloc<double>(size_t(n) * L);
    if (c->opt.variant == 2) R.Z2 = c->alloc<double>(size_t(n) * L);
    R.part = c->alloc<double>(size_t(kRedGrid) * L * L);
    R.G = c->alloc<double>(size_t(L) * L);
    R.Linv = c->alloc<double>(size_t(L) * L);
    R.d = c->alloc<double>(L);
    R.e = c->alloc<double>(L);
    R.Hv = c->alloc<double>(size_t(L) * L);
    R.vals = c->alloc<double>(L);
    R.eY = c->alloc<double>(size_t(L) * k);
    R.work = c->alloc<double>(size_t(5) * L * k);
    R.rank = c->upload(P.iface_rank);
    if (c->opt.variant == 2) {
      R.Vk = c->alloc<double>(size_t(s) * k);
      R.EV = c->alloc<double>(size_t(n) * k);
      R.vc = c->alloc<double>(s);
      R.ev = c->alloc<double>(n);
      R.uc = c->alloc<double>(n);
      R.kp = c->alloc<double>(size_t(kRedGrid) * k * k);
      R.hw = c->alloc<double>(size_t(k) * k + k);
    }
    if (c->opt.c_solver == 1) batch_alloc(c, L);   // Chebyshev work blocks of the batched A0 solve
    R.ready = true;
  }
  if (c->bt.chunk_per == 0) c->bt.chunk_per = std::max(1, 256 / L);
  const double a = c->opt.alpha;
  const int np = L * L;
  // Y (s x L) -> W (s x L) = Op Y
  auto op = [&](const double *Y, double *Wout) {
    KL(c, "rand_op", c->stream, k_e_block, nblk((long long)n * L), kThreads, 0, m, s, L, c->eh_rp, c->eh_ci,
       c->eh64, 1.0 / a, a, Y, R.V);
    a0_solve_mr<double>(c, R.V, R.Z, L, nullptr);
    const double *Zf = R.Z;
    if (c->opt.variant == 2) {
      a0_solve_mr<double>(c, R.Z, R.Z2, L, nullptr);
      Zf = R.Z2;
    }
    KL(c, "rand_op", c->stream, k_et_mr<double>, nblk((long long)s * L), kThreads, 0, s, m, c->eht_rp,
       c->eht_ci, c->eht64, 1.0 / a, a, Zf, Wout, L, (const int *)nullptr);
  };
  auto gram = [&](const double *X, const double *Y) {
    KL(c, "rand_orth", c->stream, k_gram_partial, kRedGrid, kGramNT, 0, (long long)s, L, X, Y, R.part);
    KL(c, "rand_orth", c->stream, k_gram_reduce, (np + 255) / 256, 256, 0, kRedGrid, np, R.part, R.G);
  };
  // Cholesky QR twice; the orthonormal factor ends in Y's buffer (Q is scratch)
  auto orth = [&](double *Y, double *Q) {
    gram(Y, Y);
    KL(c, "rand_orth", c->stream, k_chol_inv, 1, kRandMaxL, 0, L, R.G, R.Linv, c->dflag + 0);
    KL(c, "rand_orth", c->stream, k_apply_rinv, nblk(s), kThreads, 0, (long long)s, L, Y, R.Linv, Q);
    gram(Q, Q);
    KL(c, "rand_orth", c->stream, k_chol_inv, 1, kRandMaxL, 0, L, R.G, R.Linv, c->dflag + 0);
    KL(c, "rand_orth", c->stream, k_apply_rinv, nblk(s), kThreads, 0, (long long)s, L, Q, R.Linv, Y);
  };
  ck(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), c->stream), "memset");
  KL(c, "rand_op", c->stream, k_rand_omega, nblk((long long)s * L), kThreads, 0, s, L, R.rank, c->opt.seed, R.Qb);
  op(R.Qb, R.Yb);
  orth(R.Yb, R.Qb);                       // Q in Yb
  for (int it = 0; it < c->opt.rand_power; it++) {
    op(R.Yb, R.Qb);
    orth(R.Qb, R.Yb);                     // Q in Qb
    std::swap(R.Yb, R.Qb);                // keep Q in Yb
  }
  op(R.Yb, R.Qb);                         // W = Op Q in Qb
  gram(R.Yb, R.Qb);                       // B = Q^T W in G
  KL(c, "rand_eig", c->stream, k_sym_tridiag, 1, kRandMaxL, 0, L, R.G, R.d, R.e, R.Hv);
  KL(c, "rand_eig", c->stream, k_tridiag_values, L, kEigPoints, (2 * L + 2) * sizeof(double), L, R.d, R.e, L,
     R.vals);
  KL(c, "rand_eig", c->stream, k_tridiag_vectors, 1, 256, 0, L, R.d, R.e, k, R.vals, R.eY, R.work);
  KL(c, "rand_eig", c->stream, k_back_transform, 1, 64, 0, L, k, R.Hv, R.eY);
  int fl[4];
  read_dev(c, fl, c->dflag, sizeof(fl));
  if (fl[0]) { c->err = "randomized range basis is rank-deficient (Cholesky QR failed)"; return DDLR_ERR_BREAKDOWN; }
  c->msteps = L;
  c->ritz.assign(L, 0.0);
  read_dev(c, c->ritz.data(), R.vals, sizeof(double) * L);
  for (double v : c->ritz)
    if (!std::isfinite(v)) { c->err = "NaN/Inf in the randomized low-rank build"; return DDLR_ERR_NAN; }
  if (c->opt.variant == 1) {
    KL(c, "ritz", c->stream, k_rm_gemm, nblk(s), kThreads, 0, (long long)s, L, k, R.Yb, R.eY, c->U64);
    KL(c, "ritz", c->stream, k_ddlr1_coef, 1, 32, 0, L, k, c->opt.theta_mode, R.vals, c->theta_d, c->inv1mt64,
       c->coef64, c->dflag + 1);
    read_dev(c, &c->theta, c->theta_d, sizeof(double));
  } else {
    // V_k = Q Y_k; U_k = A0^-1 E V_k; H_k = (I - U_k^T E V_k)^-1
    KL(c, "ritz", c->stream, k_rm_gemm, nblk(s), kThreads, 0, (long long)s, L, k, R.Yb, R.eY, R.Vk);
    for (int cc = 0; cc < k; cc++) {
      KL(c, "ritz", c->stream, k_get_col, nblk(s), kThreads, 0, (long long)s, k, cc, R.Vk, R.vc);
      KL(c, "e_vec", c->stream, k_e_vec<double>, nblk(n), kThreads, 0, m, s, c->eh_rp, c->eh_ci, c->eh64, 1.0 / a,
         a, R.vc, (const double *)nullptr, R.ev, (const int *)nullptr);
      KL(c, "ritz", c->stream, k_set_col, nblk(n), kThreads, 0, (long long)n, k, cc, R.ev, R.EV);
      a0_solve<double>(c, R.ev, R.uc, nullptr);
      KL(c, "ritz", c->stream, k_set_col, nblk(n), kThreads, 0, (long long)n, k, cc, R.uc, c->U64);
    }
    KL(c, "ritz", c->stream, k_utv_partial, kRedGrid, 256, 0, (long long)n, k, c->U64, R.EV, R.kp);
    hk_finalize(c, k, R.kp, R.hw);
    c->theta = 0.0;
  }
  read_dev(c, fl, c->dflag, sizeof(fl));
  const ddlr_status fst = lowrank_status(c, fl);
  if (fst != DDLR_OK) return fst;
  sync(c);
  return DDLR_OK;
}

// Chebyshev C_a solve (Sec. 4.3): C_a's values, then the spectrum estimate of
// D_a^-1 C_a by Lanczos on the pair (C_a, D_a) in the D_a inner product (with
// p_j = D_a q_j: w = C_a q_j - beta_{j-1} p_{j-1}, alpha_j = q_j^T w,
// w -= alpha_j p_j, z = D_a^-1 w, beta_j = sqrt(w^T z), q_{j+1} = z/beta_j,
// p_{j+1} = w/beta_j), stopped early at an invariant subspace (beta_j <=
// 1e-14 max |alpha|); then the Ritz values and vectors of T_m and the
// widened interval with its coefficient table (ddlr_cheb.cuh).  Every step
// runs on the device; the host reads beta_j only to decide the early stop.
// C_a = C + a^2 I values over the interface rows (from the resident, possibly
// scaled, values)
void cc_values(ddlr_ctx *c) {
  const Plan &P = c->P;
  const long long ncc = (long long)P.cc_ci.size();
  const double a = c->opt.alpha;
  KL(c, "setup", c->stream, k_gather<double>, nblk(ncc), kThreads, 0, ncc, c->cc_src, c->vals, c->cc64);
  KL(c, "setup", c->stream, k_cc_add_diag, nblk(P.s), kThreads, 0, P.s, c->cc_diag, a * a, c->cc64);
  if (c->opt.precision == 1 && c->cc32)
    KL(c, "setup", c->stream, (k_cast<float, double>), nblk(ncc), kThreads, 0, ncc, c->cc64, c->cc32,
       (const int *)nullptr);
}

// approximate inverse of C_a by MR iterations (ddlr_mr.cuh), then its
// symmetric part as row CSR for the solve
ddlr_status mr_setup(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int s = P.s;
  auto &M = c->mr;
  cc_values(c);
  const MrX X{M.xcnt, M.xrow, M.xval};
  KL(c, "setup", c->stream, k_mr_init, nblk(s), kThreads, 0, s, c->cc_diag, c->cc64, X);
  for (int it = 0; it < c->opt.mr_iters; it++) {
    KL(c, "mr", c->stream, k_mr_column, nblk(s, 128), 128, 0, s, c->cc_rp, c->cc_ci, c->cc64, X, c->opt.mr_lfil,
       c->opt.mr_droptol, M.zcnt, M.zrow, M.zval, M.num, M.den);
    KL(c, "mr", c->stream, k_mr_beta, 1, 256, 0, s, M.num, M.den, M.beta);
    KL(c, "mr", c->stream, k_mr_update, nblk(s), kThreads, 0, s, X, M.zcnt, M.zrow, M.zval, M.beta);
  }
  ck(cudaMemsetAsync(M.rcnt, 0, sizeof(int) * s, c->stream), "memset");
  ck(cudaMemsetAsync(M.cursor, 0, sizeof(int) * s, c->stream), "memset");
  KL(c, "mr", c->stream, k_mr_sym_count, nblk(s), kThreads, 0, s, X, M.rcnt);
  KL(c, "mr", c->stream, k_mr_scan, 1, 1024, 0, s, M.rcnt, M.ptr);
  KL(c, "mr", c->stream, k_mr_sym_fill, nblk(s), kThreads, 0, s, X, M.ptr, M.cursor, M.col, M.val);
  KL(c, "mr", c->stream, k_mr_sym_sort, nblk(s), kThreads, 0, s, M.ptr, M.col, M.val, M.ucnt);
  if (M.val32) {
    int tot = 0;
    read_dev(c, &tot, M.ptr + s, sizeof(int));
    KL(c, "mr", c->stream, (k_cast<float, double>), nblk(tot), kThreads, 0, (long long)tot, M.val, M.val32,
       (const int *)nullptr);
  }
  std::vector<int> u(s);
  read_dev(c, u.data(), M.ucnt, sizeof(int) * s);
  M.nnz = 0;
  for (int v : u) M.nnz += v;
  double b = 0;
  read_dev(c, &b, M.beta, sizeof(double));
  if (!std::isfinite(b)) { c->err = "NaN/Inf in the MR approximate inverse"; return DDLR_ERR_NAN; }
  return DDLR_OK;
}

ddlr_status cheb_setup(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int s = P.s, m = P.m, t = c->opt.cheb_steps, me = c->opt.cheb_lanczos;
  cc_values(c);
  double *r = c->w64[0], *z = c->w64[1], *q = c->w64[2], *pv = c->w64[3], *pp = c->w64[4], *w = c->w64[5];
  const double *lv = c->l64, *uv = c->u64, *di = c->dinv64;
  KL(c, "setup", c->stream, k_cheb_start, nblk(s), kThreads, 0, s, m, c->cz_rank, c->opt.seed, r);
  chunk_sweeps<double>(c, c->stream, P.ch_c_ptr, "cheb_dsolve", lv, uv, di, r, z, nullptr);
  KL(c, "setup", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, r + m, z + m, c->part64,
     (const int *)nullptr);
  KL(c, "setup", c->stream, k_cheb_reduce_norm, 1, 32, 0, kRedGrid, c->part64, c->cz_b0);
  int msteps = 0;
  double scale = 0.0;
  for (int j = 0; j < me; j++) {
    const double *beta = j == 0 ? c->cz_b0 : c->cz_be + (j - 1);
    KL(c, "setup", c->stream, k_cheb_lz_qp, nblk(s), kThreads, 0, s, m, beta, z, r, q, pv);
    KL(c, "setup", c->stream, k_cheb_lz_w, nblk(s), kThreads, 0, s, m, c->cc_rp, c->cc_ci, c->cc64, q, pp,
       j > 0 ? c->cz_be + (j - 1) : (const double *)nullptr, w);
    KL(c, "setup", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, q + m, w + m,
       c->part64, (const int *)nullptr);
    KL(c, "setup", c->stream, k_reduce_scalar, 1, 32, 0, kRedGrid, c->part64, c->cz_al + j, 0,
       (const int *)nullptr);
    KL(c, "setup", c->stream, k_cheb_lz_sub, nblk(s), kThreads, 0, s, m, c->cz_al + j, pv, w);
    chunk_sweeps<double>(c, c->stream, P.ch_c_ptr, "cheb_dsolve", lv, uv, di, w, z, nullptr);
    KL(c, "setup", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)s, w + m, z + m,
       c->part64, (const int *)nullptr);
    KL(c, "setup", c->stream, k_cheb_reduce_norm, 1, 32, 0, kRedGrid, c->part64, c->cz_be + j);
    double ab[2];
    read_dev(c, &ab[0], c->cz_al + j, sizeof(double));
    read_dev(c, &ab[1], c->cz_be + j, sizeof(double));
    if (!std::isfinite(ab[0]) || !std::isfinite(ab[1])) {
      c->err = "NaN/Inf in the spectrum estimate of the Chebyshev C_a solve";
      return DDLR_ERR_NAN;
    }
    msteps = j + 1;
    scale = std::max(scale, std::fabs(ab[0]));
    if (ab[1] <= 1e-14 * scale) break;
    std::swap(pp, pv);   // p_j becomes p_{j-1}
    std::swap(r, w);     // w becomes the next r
  }
  c->cheb_msteps = msteps;
  KL(c, "setup", c->stream, k_tridiag_values, msteps, kEigPoints, (2 * msteps + 2) * sizeof(double), msteps,
     c->cz_al, c->cz_be, msteps, c->cz_vals);
  KL(c, "setup", c->stream, k_tridiag_vectors, 1, 256, 0, msteps, c->cz_al, c->cz_be, msteps, c->cz_vals, c->cz_Y,
     c->cz_work);
  KL(c, "setup", c->stream, k_cheb_bounds, 1, 32, 0, msteps, c->cz_vals, c->cz_Y, c->cz_be, t, c->ctab64,
     c->ctab32);
  double lohi[2];
  read_dev(c, lohi, c->ctab64, sizeof(lohi));
  if (!(lohi[0] > 0.0) || !(lohi[1] >= lohi[0])) {
    c->err = "the spectrum estimate of D_a^-1 C_a is not positive";
    return DDLR_ERR_NOT_SPD;
  }
  return DDLR_OK;
}

// device-side numeric setup from the resident values (Sec. 4.1: local factors, low-rank data)
ddlr_status numeric_setup(ddlr_ctx *c) {
  auto t0 = std::chrono::steady_clock::now();
  const Plan &P = c->P;
  const int n = P.n;
  const long long nnz = P.nnz, nf = P.nnz_factor;
  const double a = c->opt.alpha;
  ck(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), c->stream), "memset");
  if (c->opt.scale_diag) {
    KL(c, "setup", c->stream, k_diag_scale, nblk(n), kThreads, 0, n, c->diag_pos, c->val, c->dsc);
    KL(c, "setup", c->stream, k_scale_vals, nblk(nnz), kThreads, 0, nnz, c->orow, c->ocol, c->val, c->dsc, c->vals);
    KL(c, "setup", c->stream, k_permute_in<double>, nblk(n), kThreads, 0, n, c->perm, c->dsc, c->dsc_dev);
  }
  const long long na = (long long)P.a_col.size(), ne = (long long)P.eh_ci.size();
  KL(c, "setup", c->stream, k_gather<double>, nblk(na), kThreads, 0, na, c->a_src, c->val, c->a_val);
  KL(c, "setup", c->stream, k_gather<double>, nblk(ne), kThreads, 0, ne, c->eh_src, c->vals, c->eh64);
  KL(c, "setup", c->stream, k_gather<double>, nblk(ne), kThreads, 0, ne, c->eht_src, c->vals, c->eht64);
  KL(c, "setup", c->stream, k_factor_init, nblk(nf), kThreads, 0, (int)nf, c->f_src, c->f_prp, c->f_pa,
     c->f_pb, c->f_cdiag, c->vals, 1.0 / (a * a), a * a, c->fval);
  const int nL = int(P.fl_ptr.size()) - 1;
  for (int L = 0; L < nL; L++) {
    const int cnt = P.fl_ptr[L + 1] - P.fl_ptr[L];
    if (cnt == 0) continue;
    if (c->opt.factor >= 2)
      KL(c, "factor", c->stream, k_ildl_level, nblk(cnt), kThreads, 0, cnt, c->fl_rows + P.fl_ptr[L],
         c->f_rp, c->f_ci, c->fval, c->dflag);
    else
      KL(c, "factor", c->stream, k_ic_level, nblk(cnt), kThreads, 0, cnt, c->fl_rows + P.fl_ptr[L],
         c->f_rp, c->f_ci, c->fval, c->dflag);
  }
  ck(cudaMemsetAsync(c->l64, 0, sizeof(double) * P.l_col.size(), c->stream), "memset");
  ck(cudaMemsetAsync(c->u64, 0, sizeof(double) * P.u_col.size(), c->stream), "memset");
  KL(c, "setup", c->stream, k_solve_layout<double>, nblk(nf), kThreads, 0, (int)nf, c->f_row, c->f_rp,
     c->map_l, c->map_u, c->row_slot, c->fval, c->l64, c->u64, c->dinv64, c->dinvs64);
  if (c->lx64) {
    const long long nsl = (long long)P.l_col.size();
    KL(c, "setup", c->stream, k_prescale_cols<double>, nblk(nsl), kThreads, 0, nsl, c->S.l_col, c->l64,
       c->dinv64, c->lx64);
  }
  int fl[4];
  read_dev(c, fl, c->dflag, sizeof(fl));
  if (fl[3]) { clear_timeout(c); c->err = "a bounded device wait timed out"; return DDLR_ERR_TIMEOUT; }
  if (fl[0]) {
    c->err = "non-positive pivot in a local factorisation";
    return DDLR_ERR_BREAKDOWN;
  }
  if (c->opt.c_solver == 1) {
    ddlr_status cs = cheb_setup(c);
    if (cs != DDLR_OK) return cs;
  } else if (c->opt.c_solver == 2) {
    ddlr_status cs = mr_setup(c);
    if (cs != DDLR_OK) return cs;
  }
  ddlr_status st = c->opt.lowrank_method == 1   ? run_randomized(c)
                   : c->opt.lowrank_method == 2 ? run_lbd(c)
                                                : run_lanczos(c);
  if (st != DDLR_OK) {
    c->err = lowrank_error(c, st);
    return st;
  }
  make_low_precision(c);
  ck(cudaPeekAtLastError(), "kernel launch");
  sync(c);
  c->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return DDLR_OK;
}

// ------------------------------------------------ persistent kernels
size_t pz_pcg_smem(int k) { return size_t(kPzThreads + 32 + k + 2) * sizeof(double); }
size_t pz_lz_smem(int mmax) {
  return size_t(kPzLzThreads + 32 + 3 * mmax + 2) * sizeof(double) + size_t(mmax + 2) * sizeof(float);
}

// Whole-solve persistent kernels serve shallow factors (every block at most
// kPzMaxLevels levels deep) on devices with cooperative launch; one CTA per
// SM.  The Lanczos process then always runs persistent.  PCG runs persistent
// up to kPzPcgRowsPerSm rows per SM: beyond that the per-phase kernels, with
// four times the resident threads, hide the gather latency better (measured
// on GB300, 7-point Laplacian: 64^3 73 vs 91 us per iteration, 128^3 633 vs
// 489).  DDLR_PERSIST=0 keeps the kernel-per-phase path everywhere, =1 uses
// the persistent PCG at every size.
constexpr int kPzPcgRowsPerSm = 3000;
void pz_setup(ddlr_ctx *c, int mmax) {
  const Plan &P = c->P;
  const char *env = getenv("DDLR_PERSIST");
  if (env && env[0] == '0') return;
  // the persistent kernels solve with Cholesky-factored C_a only; the
  // Chebyshev and MR C_a solves and L D L^T factors run in the
  // kernel-per-phase path
  if (c->opt.c_solver != 0 || c->opt.factor >= 2) return;
  const bool force = env && env[0] == '1';
  const int nL = int(P.ch_all_ptr.size()) - 1;
  if (nL < 1 || nL > kPzMaxLevels || std::max(P.levels_interior, P.levels_c) > kShallowLevels) return;
  if (P.lv_desc.empty() || int(P.lv_ptr.size()) != nL + 1) return;
  const int k = c->opt.rank_k;
  int dev = 0, sms = 0, coop = 0, optin = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (!coop || sms <= 0 || k > kPzThreads) return;
  const size_t sp = pz_pcg_smem(k), sl = pz_lz_smem(mmax);
  int occ_p = 0, occ_l = 0;
  const void *pcg_fn = c->opt.precision == 0 ? (const void *)k_pcg_persist<kPzThreads, double, double>
                       : c->opt.uk_bf16    ? (const void *)k_pcg_persist<kPzThreads, float, __nv_bfloat16>
                                           : (const void *)k_pcg_persist<kPzThreads, float, float>;
  ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, pcg_fn, kPzThreads, sp), "occupancy");
  if (sl <= size_t(optin)) {
    raise_smem_limit((const void *)k_lz_persist<kPzLzThreads>, sl);
    ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, k_lz_persist<kPzLzThreads>, kPzLzThreads, sl),
       "occupancy");
  }
  c->pz_grid = sms;
  c->pz_pstride = std::max(k, mmax + 2);
  c->pz_mmax = mmax;
  c->pz_pcg = occ_p >= 1 && (force || P.n <= (long long)kPzPcgRowsPerSm * sms);
  c->pz_lz = occ_l >= 1;
  if (!c->pz_pcg && !c->pz_lz) return;
  c->pz_part = c->alloc<double>(size_t(3) * c->pz_grid * c->pz_pstride);
  c->pz_bar = c->alloc<unsigned>(1);
  std::vector<unsigned char> f0(P.n, 0);
  for (int b = 0; b + 1 < int(P.blk_lvl0.size()); b++) {
    const int l0 = P.blk_lvl0[b];
    if (l0 >= P.blk_lvl0[b + 1]) continue;
    for (int r = P.lvl_row0[l0]; r < P.lvl_row0[l0] + P.lvl_nrows[l0]; r++) f0[r] = 1;
  }
  c->pz_lvl0 = c->upload(f0);
}

template <typename T> const T *pz_u(ddlr_ctx *c);
template <> const double *pz_u<double>(ddlr_ctx *c) { return c->U64; }
template <> const float *pz_u<float>(ddlr_ctx *c) { return c->U32; }
template <> const __nv_bfloat16 *pz_u<__nv_bfloat16>(ddlr_ctx *c) { return c->Ub16; }

template <typename T, typename TU>
PzOp<T, TU> make_pzop(ddlr_ctx *c) {
  const Plan &P = c->P;
  PzOp<T, TU> O{};
  O.n = P.n; O.m = P.m; O.s = P.s; O.k = c->opt.rank_k; O.variant = c->opt.variant;
  O.nL = int(P.ch_all_ptr.size()) - 1;
  O.pstride = c->pz_pstride;
  O.a = c->opt.alpha; O.ia = 1.0 / c->opt.alpha;
  for (int i = 0; i <= O.nL; i++) O.lvl_ptr[i] = P.lv_ptr[i];
  O.desc = c->lv_desc;
  O.l_col = c->S.l_col;
  O.u_col = c->S.u_col;
  O.lval = Prec<T>::l(c); O.uval = Prec<T>::u(c); O.dinv = Prec<T>::dinv(c);
  O.eh_rp = c->eh_rp; O.eh_ci = c->eh_ci; O.eh = Prec<T>::eh(c);
  O.eht_rp = c->eht_rp; O.eht_ci = c->eht_ci; O.eht = Prec<T>::eht(c);
  O.U = pz_u<TU>(c); O.coef = Prec<T>::coef(c); O.inv1mt = Prec<T>::inv1mt(c); O.Hk = Prec<T>::Hk(c);
  O.a_soff = c->a_soff; O.a_sw = c->a_sw; O.a_col = c->a_col; O.a_val = c->a_val;
  O.dsc = c->dsc_dev;
  O.lvl0 = c->pz_lvl0;
  O.fuse0 = O.nL >= 2 ? 1 : 0;
  O.part = c->pz_part;
  O.gs.count = c->pz_bar;
  O.gs.err = c->dflag + 3;
  O.gs.wait_ns = c->wait_ns;
  // tests of the timeout path: DDLR_TEST_UNMET_BARRIER=1 makes the first grid
  // barrier of this launch wait for an arrival that never comes
  const char *um = getenv("DDLR_TEST_UNMET_BARRIER");
  O.gs.unmet = (um && um[0] == '1') ? 1 : 0;
  return O;
}

// the whole PCG solve in one persistent launch, preconditioner in T (U_k in TU)
template <typename T, typename TU>
bool pcg_persist(ddlr_ctx *c, const double *b, double *x, double tol, int maxit, T *u, T *z, T *y, T *w,
                 T *rhs) {
  PzOp<T, TU> O = make_pzop<T, TU>(c);
  PzPcg<T> Pp{};
  Pp.b = b; Pp.x = x; Pp.r = c->pv[1]; Pp.p0 = c->pv[3]; Pp.p1 = c->pv[2]; Pp.q = c->pv[4]; Pp.t = c->pv[5];
  Pp.zo = c->pv[6];
  Pp.u = u; Pp.z = z; Pp.y = y; Pp.w = w; Pp.rhs = rhs;
  Pp.st = c->pcg; Pp.tol = tol; Pp.maxit = maxit;
  void *args[] = {&O, &Pp};
  return pz_launch(c, "pcg_persist", (const void *)k_pcg_persist<kPzThreads, T, TU>, pz_pcg_smem(c->opt.rank_k),
                   args);
}

// one cooperative launch of a persistent kernel on the handle's stream;
// false (and the handle keeps to the per-phase kernels from then on) when the
// launch is refused, e.g. because every CTA cannot be resident at once
bool pz_launch(ddlr_ctx *c, const char *fam, const void *fn, size_t smem, void **args, int threads) {
  ck(cudaMemsetAsync(c->pz_bar, 0, sizeof(unsigned), c->stream), "memset");
  ddlr_ctx::Scope sc(c, fam, c->stream);
  // DDLR_FAKE_COOP_REFUSAL=1 stands in for a refused launch (tests of the
  // fallback; no kernel is launched then)
  const char *fake = getenv("DDLR_FAKE_COOP_REFUSAL");
  const cudaError_t e = (fake && fake[0] == '1')
                            ? cudaErrorCooperativeLaunchTooLarge
                            : cudaLaunchCooperativeKernel(fn, dim3(c->pz_grid), dim3(threads), args, smem,
                                                          c->stream);
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
    cudaGetLastError();   // not sticky: clear it
    c->pz_pcg = c->pz_lz = false;
    return false;
  }
  ck(e, "cudaLaunchCooperativeKernel");
  return true;
}

// grid barriers of one PCG iteration and of one Lanczos step, upper bounds
int pz_barriers_per_iteration(const ddlr_ctx *c) {
  const int nL = int(c->P.ch_all_ptr.size()) - 1;
  return 2 * (2 * nL - 1) + 8;
}

void allocate(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int n = P.n, k = c->opt.rank_k;
  c->perm = c->upload(P.perm);
  c->a_soff = c->upload(P.a_soff); c->a_sw = c->upload(P.a_sw);
  c->a_col = c->upload(P.a_col); c->a_src = c->upload(P.a_src);
  c->eh_rp = c->upload(P.eh_rp); c->eh_ci = c->upload(P.eh_ci); c->eh_src = c->upload(P.eh_src);
  c->eht_rp = c->upload(P.eht_rp); c->eht_ci = c->upload(P.eht_ci); c->eht_src = c->upload(P.eht_src);
  c->f_rp = c->upload(P.f_rp); c->f_ci = c->upload(P.f_ci); c->f_row = c->upload(P.f_row);
  c->f_src = c->upload(P.f_src); c->f_prp = c->upload(P.f_prp);
  c->f_pa = c->upload(P.f_pa); c->f_pb = c->upload(P.f_pb); c->f_cdiag = c->upload(P.f_cdiag);
  c->fl_rows = c->upload(P.fl_rows);
  c->map_l = c->upload(P.map_l); c->map_u = c->upload(P.map_u);
  c->orow = c->upload(P.orig_row); c->ocol = c->upload(P.orig_col); c->diag_pos = c->upload(P.diag_pos);
  c->S.blk_lvl0 = c->upload(P.blk_lvl0);
  c->S.lvl_row0 = c->upload(P.lvl_row0);
  c->S.lvl_nrows = c->upload(P.lvl_nrows);
  c->S.lvl_slice0 = c->upload(P.lvl_slice0);
  c->S.l_soff = c->upload(P.l_soff); c->S.l_sw = c->upload(P.l_sw); c->S.l_col = c->upload(P.l_col);
  c->S.u_soff = c->upload(P.u_soff); c->S.u_sw = c->upload(P.u_sw); c->S.u_col = c->upload(P.u_col);
  c->val = c->alloc<double>(P.nnz);
  if (c->opt.scale_diag) {
    c->vals = c->alloc<double>(P.nnz);
    c->dsc = c->alloc<double>(n);
    c->dsc_dev = c->alloc<double>(n);
  } else {
    c->vals = c->val;
  }
  c->a_val = c->alloc<double>(P.a_col.size());
  c->fval = c->alloc<double>(P.nnz_factor);
  c->l64 = c->alloc<double>(P.l_col.size());
  c->u64 = c->alloc<double>(P.u_col.size());
  {
    const char *pe = getenv("DDLR_PRESCALE");
    const int nL = int(P.ch_all_ptr.size()) - 1, nLc = int(P.ch_c_ptr.size()) - 1;
    if (!(pe && pe[0] == '0') && (nL == 2 || nLc == 2)) {
      c->lx64 = c->alloc<double>(P.l_col.size());
      if (c->opt.precision == 1) c->lx32 = c->alloc<float>(P.l_col.size());
    }
  }
  c->dinv64 = c->alloc<double>(n);
  c->dinvs64 = c->alloc<double>(size_t(P.nslice) * kSlice);
  ck(cudaMemsetAsync(c->dinvs64, 0, sizeof(double) * size_t(P.nslice) * kSlice, c->stream), "memset");
  c->row_slot = c->upload(P.row_slot);
  c->l_span = reinterpret_cast<int2 *>(c->upload(P.l_span));
  c->u_span = reinterpret_cast<int2 *>(c->upload(P.u_span));
  c->blk_row0 = c->upload(P.blk_row0);
  c->chunks = c->upload(P.chunks);
  if (!P.lv_desc.empty()) c->lv_desc = reinterpret_cast<int4 *>(c->upload(P.lv_desc));
  {
    // interior-solve kernel for deep factors: TMA-pipelined level schedule
    // (default), synchronisation-free, or plain level schedule
    // (DDLR_SOLVE=tma|sf|plain)
    const char *env = getenv("DDLR_SOLVE");
    const std::string kind = env ? env : "tma";
    const char *uv = getenv("DDLR_UVEC");
    c->uvec = !(uv && uv[0] == '0');
    const char *cr = getenv("DDLR_CHUNK_ROWS");
    if (cr && (cr[0] == '1' || cr[0] == '2' || cr[0] == '4')) c->chunk_rows = cr[0] - '0';
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool sf_ok = P.tma_zs > 0 && kind == "sf";
    c->use_sf64 = sf_ok && sf_smem_bytes<double>(P) <= size_t(optin);
    c->use_sf32 = sf_ok && sf_smem_bytes<float>(P) <= size_t(optin);
    const bool off = kind == "plain";
    c->use_tma64 = !off && !c->use_sf64 && tma_config<double>(P, c->tma64);
    c->use_tma32 = !off && !c->use_sf32 && tma_config<float>(P, c->tma32);
    if (c->use_sf64)
      raise_smem_limit((const void *)k_sptrsv_blocks_sf<double, 256, 4>, sf_smem_bytes<double>(P));
    if (c->use_sf32)
      raise_smem_limit((const void *)k_sptrsv_blocks_sf<float, 256, 4>, sf_smem_bytes<float>(P));
    ck(cudaFuncSetAttribute(k_tridiag_values, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10), "attr");
    ck(cudaFuncSetAttribute(k_w_rhs_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, int(urows_smem_bytes(64))),
       "attr");
    ck(cudaFuncSetAttribute(k_w_rhs_smem, cudaFuncAttributePreferredSharedMemoryCarveout, 100), "attr");
    ck(cudaFuncSetAttribute(k_u_add_smem, cudaFuncAttributePreferredSharedMemoryCarveout, 100), "attr");
    ck(cudaFuncSetAttribute(k_u_add_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, int(urows_smem_bytes(64))),
       "attr");
    if (c->use_tma64)
      raise_smem_limit((const void *)k_sptrsv_blocks_tma<double, 256>, tma_smem_bytes<double>(c->tma64));
    if (c->use_tma32)
      raise_smem_limit((const void *)k_sptrsv_blocks_tma<float, 256>, tma_smem_bytes<float>(c->tma32));
  }
  c->eh64 = c->alloc<double>(P.eh_ci.size());
  c->eht64 = c->alloc<double>(P.eht_ci.size());
  c->urows = c->opt.variant == 1 ? P.s : n;
  c->U64 = c->alloc<double>(size_t(c->urows) * k);
  c->coef64 = c->alloc<double>(k);
  c->Hk64 = c->alloc<double>(size_t(k) * k);
  c->theta_d = c->alloc<double>(1);
  c->inv1mt64 = c->alloc<double>(1);
  ck(cudaMemsetAsync(c->coef64, 0, sizeof(double) * k, c->stream), "memset");
  ck(cudaMemsetAsync(c->Hk64, 0, sizeof(double) * k * k, c->stream), "memset");
  ck(cudaMemsetAsync(c->inv1mt64, 0, sizeof(double), c->stream), "memset");
  c->dflag = c->alloc<int>(4);
  c->udone = c->alloc<unsigned>(1);
  ck(cudaMemsetAsync(c->udone, 0, sizeof(unsigned), c->stream), "memset");
  c->pdone = c->alloc<unsigned>(1);
  ck(cudaMemsetAsync(c->pdone, 0, sizeof(unsigned), c->stream), "memset");
  for (int i = 0; i < 8; i++) c->w64[i] = c->alloc<double>(n);
  int mmax = c->opt.lanczos_max > 0 ? c->opt.lanczos_max : 5 * k;
  mmax = std::max(std::min(mmax, P.s), k);
  c->part64 = c->alloc<double>(size_t(kRedGrid) * std::max(k + 2, mmax + 2) + 2 * kRedGrid);
  pz_setup(c, mmax);
  if (c->opt.precision == 1) {
    c->l32 = c->alloc<float>(P.l_col.size());
    c->u32 = c->alloc<float>(P.u_col.size());
    c->dinv32 = c->alloc<float>(n);
    c->dinvs32 = c->alloc<float>(size_t(P.nslice) * kSlice);
    c->eh32 = c->alloc<float>(P.eh_ci.size());
    c->eht32 = c->alloc<float>(P.eht_ci.size());
    if (c->opt.uk_bf16) c->Ub16 = c->alloc<__nv_bfloat16>(size_t(c->urows) * k);
    else c->U32 = c->alloc<float>(size_t(c->urows) * k);
    c->coef32 = c->alloc<float>(k);
    c->Hk32 = c->alloc<float>(size_t(k) * k);
    c->inv1mt32 = c->alloc<float>(1);
    for (int i = 0; i < 8; i++) c->w32[i] = c->alloc<float>(n);
    c->part32 = c->alloc<float>(size_t(kRedGrid) * (k + 2));
  }
  if (c->opt.c_solver == 2) {
    const int s = P.s;
    c->cc_rp = c->upload(P.cc_rp); c->cc_ci = c->upload(P.cc_ci);
    c->cc_src = c->upload(P.cc_src); c->cc_diag = c->upload(P.cc_diag);
    c->cc64 = c->alloc<double>(P.cc_ci.size());
    auto &M = c->mr;
    const size_t cap = size_t(s) * kMrCap;
    M.xcnt = c->alloc<int>(s); M.xrow = c->alloc<int>(cap); M.xval = c->alloc<double>(cap);
    M.zcnt = c->alloc<int>(s); M.zrow = c->alloc<int>(cap); M.zval = c->alloc<double>(cap);
    M.num = c->alloc<double>(s); M.den = c->alloc<double>(s); M.beta = c->alloc<double>(1);
    M.rcnt = c->alloc<int>(s); M.ptr = c->alloc<int>(size_t(s) + 1); M.cursor = c->alloc<int>(s);
    M.ucnt = c->alloc<int>(s);
    M.col = c->alloc<int>(2 * cap); M.val = c->alloc<double>(2 * cap);
    if (c->opt.precision == 1) M.val32 = c->alloc<float>(2 * cap);
  }
  if (c->opt.c_solver == 1) {
    const int t = c->opt.cheb_steps, me = c->opt.cheb_lanczos;
    c->cc_rp = c->upload(P.cc_rp); c->cc_ci = c->upload(P.cc_ci);
    c->cc_src = c->upload(P.cc_src); c->cc_diag = c->upload(P.cc_diag);
    c->cz_rank = c->upload(P.iface_rank);
    c->cc64 = c->alloc<double>(P.cc_ci.size());
    c->ctab64 = c->alloc<double>(2 * t + 1);
    c->ctab32 = c->alloc<float>(2 * t + 1);
    for (int i = 0; i < 5; i++) c->cb64[i] = c->alloc<double>(n);
    if (c->opt.precision == 1) {
      c->cc32 = c->alloc<float>(P.cc_ci.size());
      for (int i = 0; i < 5; i++) c->cb32[i] = c->alloc<float>(n);
    }
    c->cz_al = c->alloc<double>(me + 1);
    c->cz_be = c->alloc<double>(me + 1);
    c->cz_vals = c->alloc<double>(me + 1);
    c->cz_Y = c->alloc<double>(size_t(me) * me);
    c->cz_work = c->alloc<double>(size_t(5) * me * me);
    c->cz_b0 = c->alloc<double>(1);
  }
  c->pcg = c->alloc<PcgState>(1);
  for (int i = 0; i < 8; i++) c->pv[i] = c->alloc<double>(n);
  c->stg_in = c->alloc<double>(n);
  c->stg_out = c->alloc<double>(n);
  ck(cudaMallocHost(&c->h_pin, 64 * sizeof(double)), "cudaMallocHost");
}

// one PCG iteration (Sec. 5) on device-order vectors; every kernel reads its
// scalars from the device state and returns at once after convergence

void pcg_iteration(ddlr_ctx *c, const double *b, double *x, int flexible) {
  const int n = c->P.n;
  double *r = c->pv[1], *z = c->pv[2], *p = c->pv[3], *q = c->pv[4], *t = c->pv[5], *zo = c->pv[6];
  double *part = c->part64;
  const int *gate = pcg_gate(c);
  // x, r update with r.r and the residual test in one launch, and r.z with
  // beta in one launch (last-CTA reductions); q = A p keeps a row per thread
  // (fusing p.q into it needs a capped grid, which measured slower)
  KL(c, "spmv", c->stream, k_spmv<double>, nblk(n), kThreads, 0, n, c->a_soff, c->a_sw, c->a_col, c->a_val, p, q, gate);
  KL(c, "pcg_dot", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)n, p, q, part, gate);
  KL(c, "pcg_scalar", c->stream, k_pcg_alpha, 1, 32, 0, c->pcg, part, kRedGrid);
  KL(c, "pcg_axpy", c->stream, k_pcg_update_rr<256>, kRedGrid, 256, 0, (long long)n, c->pcg, p, q, x, r, part,
     c->pdone);
  KL(c, "pcg_check", c->stream, k_pcg_true_res<256>, kRedGrid, 256, 0, n, c->pcg, c->a_soff, c->a_sw, c->a_col, c->a_val, b, x, t, part);
  KL(c, "pcg_scalar", c->stream, k_pcg_true_dec, 1, 32, 0, c->pcg, part, kRedGrid);
  // bounded grid: it returns at once in all but restart iterations
  KL(c, "pcg_check", c->stream, k_pcg_copy_r, std::min<unsigned>(nblk(n), 152 * 8), kThreads, 0, (long long)n, c->pcg,
     t, r);
  precond(c, r, z, gate);
  KL(c, "pcg_dot2", c->stream, k_dot2_beta<256>, kRedGrid, 256, 0, (long long)n, r, z, flexible ? zo : z, part,
     c->pcg, c->pdone);
  KL(c, "pcg_p", c->stream, k_pcg_p, nblk(n), kThreads, 0, (long long)n, c->pcg, z, p, flexible ? zo : (double *)nullptr);
}

// PCG on device-order vectors b -> x (Sec. 5), device-side control flow; the
// host only polls the `done` word every few iterations.  Unless per-kernel
// timing is on, one iteration is captured once into a CUDA graph (on an
// internal stream ordered after the caller's) and replayed.
void pcg_dev(ddlr_ctx *c, const double *b, double *x, double tol, int maxit,
             ddlr_solve_info *info) {
  const Plan &P = c->P;
  const int n = P.n;
  const int flexible = c->opt.precision == 1 ? 1 : 0;
  double *r = c->pv[1], *z = c->pv[2], *p = c->pv[3], *q = c->pv[4], *zo = c->pv[6];
  double *part = c->part64;
  const int *gate = pcg_gate(c);
  const char *ng = getenv("DDLR_NO_GRAPH");
  // the whole solve in one persistent kernel when the factors are shallow
  bool persist = c->pz_pcg &&
                 (long long)(maxit + 2) * pz_barriers_per_iteration(c) * c->pz_grid < (1LL << 31);
  cudaStream_t user = c->stream;
  struct Restore {
    ddlr_ctx *c; cudaStream_t s;
    ~Restore() { c->stream = s; }
  } restore{c, user};
  if (persist) {
    if (c->opt.precision == 0)
      persist = pcg_persist<double, double>(c, b, x, tol, maxit, c->pv[7], c->w64[0], c->w64[1], c->w64[2],
                                            c->w64[3]);
    else if (c->opt.uk_bf16)
      persist = pcg_persist<float, __nv_bfloat16>(c, b, x, tol, maxit, c->w32[4], c->w32[0], c->w32[1],
                                                  c->w32[2], c->w32[3]);
    else
      persist = pcg_persist<float, float>(c, b, x, tol, maxit, c->w32[4], c->w32[0], c->w32[1], c->w32[2],
                                          c->w32[3]);
  }
  const bool use_graph = !persist && !c->timing && !(ng && ng[0] == '1');
  if (!persist) {
    if (use_graph) {
      ck(cudaEventRecord(c->ev_fork, user), "event");
      ck(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0), "wait");
      c->stream = c->gstream;
    }
    ck(cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream), "memset");
    ck(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy");
    KL(c, "pcg", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)n, b, b, part, (const int *)nullptr);
    KL(c, "pcg", c->stream, k_pcg_init, 1, 32, 0, c->pcg, part, kRedGrid, tol, maxit, flexible);
    precond(c, r, z, gate);
    KL(c, "pcg", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)n, r, z, part, gate);
    KL(c, "pcg", c->stream, k_pcg_rz0, 1, 32, 0, c->pcg, part, kRedGrid);
    ck(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy");
    ck(cudaMemcpyAsync(zo, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy");
    if (use_graph && (c->pcg_exec == nullptr || c->pcg_exec_flexible != flexible)) {
      if (c->pcg_exec) { cudaGraphExecDestroy(c->pcg_exec); c->pcg_exec = nullptr; }
      const long long l0 = c->launches;
      const std::vector<long long> f0 = c->fam_cnt;
      ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture");
      pcg_iteration(c, b, x, flexible);
      cudaGraph_t g = nullptr;
      ck(cudaStreamEndCapture(c->stream, &g), "capture");
      cudaError_t e = cudaGraphInstantiate(&c->pcg_exec, g, 0);
      cudaGraphDestroy(g);
      ck(e, "cudaGraphInstantiate");
      c->pcg_exec_flexible = flexible;
      c->pcg_nodes = c->launches - l0;
      c->pcg_fam_nodes.assign(c->fam_cnt.size(), 0);
      for (size_t i = 0; i < c->fam_cnt.size(); i++)
        c->pcg_fam_nodes[i] = c->fam_cnt[i] - (i < f0.size() ? f0[i] : 0);
      c->launches = l0;                    // captured, not yet executed
      for (size_t i = 0; i < f0.size(); i++) c->fam_cnt[i] = f0[i];
      for (size_t i = f0.size(); i < c->fam_cnt.size(); i++) c->fam_cnt[i] = 0;
    }
    const int batch = 4;
    for (int it = 0; it < maxit + batch; it += batch) {
      for (int bi = 0; bi < batch; bi++) {
        if (use_graph) {
          ck(cudaGraphLaunch(c->pcg_exec, c->stream), "cudaGraphLaunch");
          c->launches += c->pcg_nodes;
          for (size_t i = 0; i < c->pcg_fam_nodes.size(); i++) c->fam_cnt[i] += c->pcg_fam_nodes[i];
        } else {
          pcg_iteration(c, b, x, flexible);
        }
      }
      int done = 0;
      ck(cudaMemcpyAsync(c->h_pin, pcg_gate(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream), "D2H");
      ck(cudaStreamSynchronize(c->stream), "sync");
      std::memcpy(&done, c->h_pin, sizeof(int));
      if (done) break;
    }
  }
  // final true residual
  KL(c, "spmv", c->stream, k_spmv<double>, nblk(n), kThreads, 0, n, c->a_soff, c->a_sw, c->a_col, c->a_val, x, q, (const int *)nullptr);
  KL(c, "pcg", c->stream, k_resid2_partial<256>, kRedGrid, 256, 0, (long long)n, b, q, part);
  KL(c, "pcg", c->stream, k_reduce_scalar, 1, 32, 0, kRedGrid, part, c->w64[7], 0, (const int *)nullptr);
  PcgState hs;
  int dfl[4];
  ck(cudaMemcpyAsync(c->h_pin, c->w64[7], sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaMemcpyAsync(&hs, c->pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaMemcpyAsync(dfl, c->dflag, sizeof(dfl), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (use_graph) {
    ck(cudaEventRecord(c->ev_join, c->stream), "event");
    ck(cudaStreamWaitEvent(user, c->ev_join, 0), "wait");
  }
  if (dfl[3]) timeout_fail(c);
  if (persist) {
    // x, r, p, b set up and one apply; per iteration one apply, A p with the
    // p update (A once, p_old, z, p, q), the x and r updates, and z_old for
    // flexible CG
    double apply = 0;
    ddlr_get_traffic(c, &apply, nullptr, nullptr, 0);
    const double nd = double(n) * 8.0, nnz = double(P.nnz);
    const double it = apply + nnz * 12.0 + 4.0 * nd + 6.0 * nd + (flexible ? 2.0 * nd : 0.0);
    c->pz_pcg_bytes += 4.0 * nd + apply + double(hs.its) * it;
    c->pz_pcg_runs += 1;
  }
  if (info) {
    info->its = hs.its;
    info->relres = hs.bb > 0 ? std::sqrt(c->h_pin[0] / hs.bb) : 0.0;
    info->status = hs.status == 0 ? DDLR_OK : (hs.status == 5 ? DDLR_ERR_NOCONV : DDLR_ERR_NAN);
    if (hs.done == 0) info->status = DDLR_ERR_NOCONV;
  }
}

constexpr int kGmresMaxRestart = 512;

// Restarted GMRES(m) on device-order vectors b -> x (Sec. 5: GMRES(40) for
// the indefinite problems), right-preconditioned, kernels in ddlr_gmres.cuh.
// The host reads the rotated residual norm and h_{j+1,j} after every Arnoldi
// step to end the cycle; the true residual b - A x ends each cycle.
void gmres_dev(ddlr_ctx *c, const double *b, double *x, double tol, int maxit, int m, ddlr_solve_info *info) {
  const int n = c->P.n;
  auto &G = c->gm;
  if (G.m < m) {
    // grown arrays replace the old ones; the arena keeps the old until destroy
    G.free_graphs();
    G.V = c->alloc<double>(size_t(n) * (m + 1));
    G.Z = c->alloc<double>(size_t(n) * m);
    G.H = c->alloc<double>(size_t(m + 1) * m);
    G.cs = c->alloc<double>(m); G.sn = c->alloc<double>(m);
    G.g = c->alloc<double>(m + 1); G.y = c->alloc<double>(m);
    G.cpart = c->alloc<double>(size_t(kRedGrid) * (m + 1));
    G.cvec = c->alloc<double>(m + 1);
    G.st = c->alloc<double>(4);
    G.m = m;
  }
  const int ld = m + 1;
  double *r = c->pv[1], *w = c->pv[3], *q = c->pv[4];
  // unless per-kernel timing is on, every Arnoldi step runs as one CUDA graph
  // (step j captured once per handle, on the internal stream ordered after
  // the caller's): with deep factors a step is about a thousand launches
  const char *ng = getenv("DDLR_NO_GRAPH");
  const bool use_graph = !c->timing && !(ng && ng[0] == '1');
  cudaStream_t user = c->stream;
  struct Restore {
    ddlr_ctx *c; cudaStream_t s;
    ~Restore() { c->stream = s; }
  } restore{c, user};
  if (use_graph) {
    ck(cudaEventRecord(c->ev_fork, user), "event");
    ck(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0), "wait");
    c->stream = c->gstream;
    if (G.step_m != m) G.free_graphs();   // H's leading dimension is m + 1
    G.step_m = m;
    if (int(G.step.size()) < m) {
      G.step.resize(m, nullptr);
      G.nodes.resize(m, 0);
      G.fam_nodes.resize(m);
    }
  }
  auto norm_to = [&](const double *v, double *o1, double *o2) {
    KL(c, "gmres", c->stream, (k_dot_partial<double, 256>), kRedGrid, 256, 0, (long long)n, v, v, c->part64,
       (const int *)nullptr);
    KL(c, "gmres", c->stream, k_gm_norm, 1, 32, 0, kRedGrid, c->part64, o1, o2);
  };
  auto read2 = [&](const double *src, double *dst) {
    ck(cudaMemcpyAsync(c->h_pin, src, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "D2H");
    ck(cudaStreamSynchronize(c->stream), "sync");
    dst[0] = c->h_pin[0];
    dst[1] = c->h_pin[1];
  };
  ck(cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream), "memset");
  ck(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy");
  norm_to(b, G.st + 2, G.st + 3);
  double sc[2];
  read2(G.st + 2, sc);
  const double bn = sc[0];
  double beta = bn;
  int its = 0, status = DDLR_ERR_NOCONV;
  while (true) {
    if (!std::isfinite(beta)) { status = DDLR_ERR_NAN; break; }
    if (beta <= tol * bn) { status = DDLR_OK; break; }
    if (its >= maxit) break;
    KL(c, "gmres", c->stream, k_lbd_scale, nblk(n), kThreads, 0, (long long)n, r, G.st + 2, G.V);   // v_0 = r / beta
    KL(c, "gmres", c->stream, k_gm_ginit, 1, std::max(32, ((m + 1 + 31) / 32) * 32), 0, m, G.st + 2, G.g);
    int j = 0;
    bool nan = false;
    while (j < m && its < maxit) {
      // one Arnoldi step: z_j = M^-1 v_j, w = A z_j, two CGS passes against
      // V_{j+1}, h_{j+1,j}, v_{j+1}, the Givens rotation of column j
      auto arnoldi = [&](int jj) {
        const double *vj = G.V + size_t(jj) * n;
        double *zj = G.Z + size_t(jj) * n, *hcol = G.H + size_t(jj) * ld;
        precond(c, vj, zj, nullptr);
        KL(c, "spmv", c->stream, k_spmv<double>, nblk(n), kThreads, 0, n, c->a_soff, c->a_sw, c->a_col, c->a_val, zj,
           w, (const int *)nullptr);
        for (int pass = 0; pass < 2; pass++) {
          KL(c, "gmres_cgs", c->stream, k_cgs_partial<256>, kRedGrid, 256, 0, (long long)n, jj + 1, G.V, (long long)n,
             w, G.cpart);
          KL(c, "gmres_cgs", c->stream, k_gm_reduce_acc, ((jj + 1) * 32 + 255) / 256, 256, 0, kRedGrid, jj + 1,
             G.cpart, G.cvec, hcol, pass == 0 ? 1 : 0);
          KL(c, "gmres_cgs", c->stream, k_cgs_sub, nblk(n), kThreads, (jj + 1) * sizeof(double), (long long)n, jj + 1,
             G.V, (long long)n, G.cvec, w);
        }
        norm_to(w, hcol + jj + 1, G.st + 1);
        KL(c, "gmres", c->stream, k_lbd_scale, nblk(n), kThreads, 0, (long long)n, w, G.st + 1,
           G.V + size_t(jj + 1) * n);
        KL(c, "gmres", c->stream, k_gm_givens, 1, 32, 0, jj, hcol, G.cs, G.sn, G.g, G.st);
      };
      if (use_graph) {
        if (!G.step[j]) {
          const long long l0 = c->launches;
          const std::vector<long long> f0 = c->fam_cnt;
          ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture");
          arnoldi(j);
          cudaGraph_t g = nullptr;
          ck(cudaStreamEndCapture(c->stream, &g), "capture");
          cudaError_t e = cudaGraphInstantiate(&G.step[j], g, 0);
          cudaGraphDestroy(g);
          ck(e, "cudaGraphInstantiate");
          G.nodes[j] = c->launches - l0;
          G.fam_nodes[j].assign(c->fam_cnt.size(), 0);
          for (size_t i = 0; i < c->fam_cnt.size(); i++)
            G.fam_nodes[j][i] = c->fam_cnt[i] - (i < f0.size() ? f0[i] : 0);
          c->launches = l0;                  // captured, not yet executed
          for (size_t i = 0; i < f0.size(); i++) c->fam_cnt[i] = f0[i];
          for (size_t i = f0.size(); i < c->fam_cnt.size(); i++) c->fam_cnt[i] = 0;
        }
        ck(cudaGraphLaunch(G.step[j], c->stream), "cudaGraphLaunch");
        c->launches += G.nodes[j];
        for (size_t i = 0; i < G.fam_nodes[j].size(); i++) c->fam_cnt[i] += G.fam_nodes[j][i];
      } else {
        arnoldi(j);
      }
      read2(G.st, sc);
      its++;
      j++;
      if (!std::isfinite(sc[0]) || !std::isfinite(sc[1])) { nan = true; break; }
      if (sc[0] <= tol * bn || !(sc[1] > 0.0)) break;
    }
    if (nan) { status = DDLR_ERR_NAN; break; }
    KL(c, "gmres", c->stream, k_gm_backsolve, 1, 32, 0, j, G.H, ld, G.g, G.y);
    KL(c, "gmres", c->stream, k_gm_update, nblk(n), kThreads, j * sizeof(double), (long long)n, j, G.Z, G.y, x);
    KL(c, "spmv", c->stream, k_spmv<double>, nblk(n), kThreads, 0, n, c->a_soff, c->a_sw, c->a_col, c->a_val, x, q,
       (const int *)nullptr);
    KL(c, "gmres", c->stream, k_gm_resid, nblk(n), kThreads, 0, (long long)n, b, q, r);
    norm_to(r, G.st + 2, G.st + 3);
    read2(G.st + 2, sc);
    beta = sc[0];
  }
  if (use_graph) {
    ck(cudaEventRecord(c->ev_join, c->stream), "event");
    ck(cudaStreamWaitEvent(user, c->ev_join, 0), "wait");
  }
  int dfl[4];
  read_dev(c, dfl, c->dflag, sizeof(dfl));
  if (dfl[3]) timeout_fail(c);
  if (info) {
    info->its = its;
    info->relres = bn > 0 ? beta / bn : 0.0;
    info->status = status;
  }
}

// ============================================================ batched path
// row ranges (partial sums) of the tensor-core U_k^T Y
constexpr int kTcRedGrid = 4 * kRedGrid;

void batch_free(ddlr_ctx *c) {
  auto &B = c->bt;
  for (auto &kv : B.graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  for (void *p : B.mem) cudaFree(p);
  B = ddlr_ctx::Batch();
}

// workspaces for batches of up to R right-hand sides; they only grow (a
// narrower batch reuses them), so steady-state serving never frees memory
void batch_alloc(ddlr_ctx *c, int R) {
  auto &B = c->bt;
  if (B.R >= R) return;
  const int per_c = B.chunk_per, bd_e = B.bd_elem;
  const bool tuned = B.tuned;
  batch_free(c);
  const Plan &P = c->P;
  const size_t nR = size_t(P.n) * R, sR = size_t(P.s) * R, k = c->opt.rank_k;
  auto al = [&](size_t bytes) {
    void *p = nullptr;
    ck(cudaMalloc(&p, bytes < 16 ? 16 : bytes), "cudaMalloc");
    B.mem.push_back(p);
    return p;
  };
  double **v[] = {&B.B, &B.X, &B.Rr, &B.Z, &B.P, &B.Q, &B.T, &B.Zo, &B.S};
  for (double **pp : v) *pp = (double *)al(nR * 8);
  B.w64[0] = (double *)al(nR * 8);   // A0 solve result
  B.w64[1] = (double *)al(sR * 8);   // Y
  B.w64[2] = (double *)al(sR * 8);   // W
  B.w64[3] = (double *)al(nR * 8);   // RHS
  B.w64[4] = (double *)al(k * R * 8);
  if (c->opt.precision == 1) {
    B.w32[0] = (float *)al(nR * 4);
    B.w32[1] = (float *)al(sR * 4);
    B.w32[2] = (float *)al(sR * 4);
    B.w32[3] = (float *)al(nR * 4);
    B.w32[4] = (float *)al(k * R * 4);
    B.w32[5] = (float *)al(nR * 4);   // cast input
    B.w32[6] = (float *)al(nR * 4);   // cast output
    // the tensor-core U_k^T Y writes kTcRedGrid partials plus a k x R sum
    B.part32 = (float *)al((size_t(kTcRedGrid) + 1) * std::max<size_t>(k * R, 2 * R) * 4);
  }
  B.part64 = (double *)al(size_t(kRedGrid) * std::max<size_t>(k * R, 2 * R) * 8);
  B.fpart = (double *)al(size_t((P.n + kFbRows - 1) / kFbRows) * R * 8);
  if (c->opt.c_solver == 1)
    for (int i = 0; i < 5; i++) {
      B.cb64[i] = (double *)al(nR * 8);
      if (c->opt.precision == 1) B.cb32[i] = (float *)al(nR * 4);
    }
  B.st = (PcgStateMR *)al(sizeof(PcgStateMR));
  B.R = R;
  const char *tce = getenv("DDLR_BATCH_TC");
  B.tc = !(tce && tce[0] == '0') && k <= 64;
  B.chunk_per = tuned ? per_c : std::max(1, 256 / R);
  B.bd_elem = tuned ? bd_e : 256;
  B.tuned = tuned;
}

// block of the batched level solve: the autotuned rows-per-pass times R
inline int chunk_block(const ddlr_ctx *c, int R) {
  return std::max(R, std::min(1024 / R, std::max(1, c->bt.chunk_per)) * R);
}

template <typename T> struct BPrec;
template <> struct BPrec<double> {
  static double *w(ddlr_ctx *c, int i) { return c->bt.w64[i]; }
  static double *part(ddlr_ctx *c) { return c->bt.part64; }
};
template <> struct BPrec<float> {
  static float *w(ddlr_ctx *c, int i) { return c->bt.w32[i]; }
  static float *part(ddlr_ctx *c) { return c->bt.part32; }
};

inline unsigned eblk(long long cnt, int bd) { return (unsigned)((cnt + bd - 1) / bd); }

// widest batch the shared-memory tiles allow (k*R <= 1024, k <= 64); < 2 means
// "solve column by column"
inline int batch_width(const ddlr_ctx *c) {
  const int k = c->opt.rank_k;
  if (c->opt.factor >= 2) return 0;   // L D L^T factors: one right-hand side at a time
  return k <= 64 ? std::min(kMaxR, 1024 / k) : 0;
}

// Z = A0^-1 X for a block of R vectors: every level of all blocks per launch
template <typename T>
void a0_solve_mr(ddlr_ctx *c, const T *X, T *Z, int R, const int *gate) {
  const Plan &P = c->P;
  const T *lv0 = Prec<T>::l(c), *lx = Prec<T>::lx(c), *uv = Prec<T>::u(c), *di = Prec<T>::dinv(c);
  const std::vector<int> &ptr = P.ch_all_ptr;
  const int nL = int(ptr.size()) - 1;
  const std::vector<int> &dptr = P.lv_ptr;
  auto launch = [&](int L, int mode) {
    const T *lv = mode == 5 ? lx : lv0;
    if (c->lv_desc) {
      const int cnt = dptr[L + 1] - dptr[L];
      if (cnt <= 0) return;
      constexpr int kV = Vec16<T>::n;
      if (R % kV == 0) {
        // 16-byte vectors of kV columns per thread; 256 threads
        const int per = 256 / (R / kV), rows = per * kMrRowsPerThread;
        KL(c, "sptrsv_levels_mr", c->stream, k_sptrsv_desc_mr_v<T>, (cnt + rows - 1) / rows, per * (R / kV), 0,
           c->lv_desc + dptr[L], cnt, mode, c->S.l_col, c->S.u_col, lv, uv, di, X, Z, R, gate);
        return;
      }
      const int bd = chunk_block(c, R), rows = (bd / R) * kMrRowsPerThread;
      KL(c, "sptrsv_levels_mr", c->stream, k_sptrsv_desc_mr<T>, (cnt + rows - 1) / rows, bd, 0,
         c->lv_desc + dptr[L], cnt, mode, c->S.l_col, c->S.u_col, lv, uv, di, X, Z, R, gate);
      return;
    }
    const int nch = ptr[L + 1] - ptr[L];
    if (nch > 0)
      KL(c, "sptrsv_levels_mr", c->stream, k_sptrsv_chunks_mr<T>, nch, chunk_block(c, R), 0, c->S,
         reinterpret_cast<const int4 *>(c->chunks) + ptr[L], mode, lv, uv, di, X, Z, R, gate);
  };
  if (nL == 2) {            // multicolour factors: two launches, see modes 3 (5) and 4
    launch(1, lx ? 5 : 3);
    launch(0, 4);
  } else {
    for (int L = 0; L + 1 < nL; L++) launch(L, 0);
    if (nL > 0) launch(nL - 1, 2);
    for (int L = nL - 2; L >= 0; L--) launch(L, 1);
  }
  if (c->opt.c_solver == 1) cheb_tail<T>(c, c->stream, X, Z, R, gate);
  else if (c->opt.c_solver == 2) mr_apply_c<T>(c, c->stream, X, Z, R, gate);
}

template <typename T>
void cheb_dsolve(ddlr_ctx *c, cudaStream_t st, const T *x, T *z, int R, const int *gate) {
  const T *lv0 = Prec<T>::l(c), *lx = Prec<T>::lx(c), *uv = Prec<T>::u(c), *di = Prec<T>::dinv(c);
  const std::vector<int> &ptr = c->P.ch_c_ptr;
  if (R == 1) {
    chunk_sweeps<T>(c, st, ptr, "cheb_dsolve", lv0, uv, di, x, z, gate);
    return;
  }
  const int nL = int(ptr.size()) - 1;
  auto launch = [&](int L, int mode) {
    const T *lv = mode == 5 ? lx : lv0;
    const int nch = ptr[L + 1] - ptr[L];
    if (nch > 0)
      KL(c, "cheb_dsolve", st, k_sptrsv_chunks_mr<T>, nch, chunk_block(c, R), 0, c->S,
         reinterpret_cast<const int4 *>(c->chunks) + ptr[L], mode, lv, uv, di, x, z, R, gate);
  };
  if (nL == 2) {
    launch(1, lx ? 5 : 3);
    launch(0, 4);
    return;
  }
  for (int L = 0; L + 1 < nL; L++) launch(L, 0);
  if (nL > 0) launch(nL - 1, 2);
  for (int L = nL - 2; L >= 0; L--) launch(L, 1);
}

// Out = M^-1 X for a block of R vectors (device order, row-major)
template <typename T, typename TU>
void apply_mr(ddlr_ctx *c, const TU *U, const T *X, T *Out, int R, const int *gate) {
  const Plan &P = c->P;
  const int n = P.n, m = P.m, s = P.s, k = c->opt.rank_k;
  const int bd = c->bt.bd_elem;
  const T a = T(c->opt.alpha), ia = T(1.0 / c->opt.alpha);
  T *part = BPrec<T>::part(c), *Tm = BPrec<T>::w(c, 4);
  if (c->opt.variant == 1) {
    T *Z = BPrec<T>::w(c, 0), *Y = BPrec<T>::w(c, 1), *W = BPrec<T>::w(c, 2), *RHS = BPrec<T>::w(c, 3);
    a0_solve_mr<T>(c, X, Z, R, gate);
    constexpr int kV = Vec16<T>::n;
    const bool vec = R % kV == 0;
    if (vec)
      KL(c, "et_mr", c->stream, k_et_mr_v<T>, eblk((long long)s * (R / kV), 256), 256, 0, s, m, c->eht_rp,
         c->eht_ci, Prec<T>::eht(c), ia, a, Z, Y, R, gate);
    else
      KL(c, "et_mr", c->stream, k_et_mr<T>, eblk((long long)s * R, bd), bd, 0, s, m, c->eht_rp, c->eht_ci,
         Prec<T>::eht(c), ia, a, Z, Y, R, gate);
    bool tc = false;
    if constexpr (std::is_same<T, float>::value) {
      tc = c->bt.tc;
      if (tc) {
        // more, shorter row ranges than the scalar form: every CTA of the
        // tensor-core form is resident at once
        KL(c, "utx_mr", c->stream, (k_utx_mr_tc<TU>), kTcRedGrid, 256, 0, (long long)s, k, U, Y, R, part, gate);
        KL(c, "reduce_mr", c->stream, k_reduce_cols_mr<T>, (unsigned)((k * R + 31) / 32), 256, 0, kTcRedGrid,
           k * R, R, part, Prec<T>::coef(c), Tm, gate);
      }
    }
    if (!tc) {
      KL(c, "utx_mr", c->stream, (k_utx_mr_partial<T, TU>), kRedGrid, 256, 0, (long long)s, k, U, Y, R, part, gate);
      KL(c, "reduce_mr", c->stream, k_reduce_mr<T>, 1, 256, 0, kRedGrid, k, R, part, Prec<T>::coef(c),
         (const T *)nullptr, Tm, gate);
    }
    if constexpr (std::is_same<T, float>::value) {
      if (tc) {
        KL(c, "w_rhs_mr", c->stream, (k_w_rhs_mr_tc<TU>), (unsigned)((s + 127) / 128), 256, 0, s, m, k, U, Tm, Y,
           Prec<T>::inv1mt(c), a, X, W, RHS, R, gate);
      } else {
        KL(c, "w_rhs_mr", c->stream, (k_w_rhs_mr<T, TU>), eblk((long long)s * R, bd), bd, 0, s, m, k, U, Tm, Y,
           Prec<T>::inv1mt(c), a, X, W, RHS, R, gate);
      }
    } else {
      KL(c, "w_rhs_mr", c->stream, (k_w_rhs_mr<T, TU>), eblk((long long)s * R, bd), bd, 0, s, m, k, U, Tm, Y,
         Prec<T>::inv1mt(c), a, X, W, RHS, R, gate);
    }
    if (vec)
      KL(c, "e_int_mr", c->stream, k_e_interior_mr_v<T>, eblk((long long)m * (R / kV), 256), 256, 0, m, c->eh_rp,
         c->eh_ci, Prec<T>::eh(c), ia, W, X, RHS, R, gate);
    else
      KL(c, "e_int_mr", c->stream, k_e_interior_mr<T>, eblk((long long)m * R, bd), bd, 0, m, c->eh_rp, c->eh_ci,
         Prec<T>::eh(c), ia, W, X, RHS, R, gate);
    a0_solve_mr<T>(c, RHS, Out, R, gate);
  } else {
    a0_solve_mr<T>(c, X, Out, R, gate);
    bool tc = false;
    if constexpr (std::is_same<T, float>::value) tc = c->bt.tc;
    if constexpr (std::is_same<T, float>::value) {
      if (tc) {
        KL(c, "utx_mr", c->stream, (k_utx_mr_tc<TU>), kTcRedGrid, 256, 0, (long long)n, k, U, X, R, part, gate);
        // column sums first, then H_k applied to the k x R block
        T *tmp = part + size_t(kTcRedGrid) * k * R;
        KL(c, "reduce_mr", c->stream, k_reduce_cols_mr<T>, (unsigned)((k * R + 31) / 32), 256, 0, kTcRedGrid,
           k * R, R, part, (const T *)nullptr, tmp, gate);
        KL(c, "reduce_mr", c->stream, k_reduce_mr<T>, 1, 256, 0, 1, k, R, tmp, (const T *)nullptr, Prec<T>::Hk(c),
           Tm, gate);
      }
    }
    if (!tc) {
      KL(c, "utx_mr", c->stream, (k_utx_mr_partial<T, TU>), kRedGrid, 256, 0, (long long)n, k, U, X, R, part, gate);
      KL(c, "reduce_mr", c->stream, k_reduce_mr<T>, 1, 256, 0, kRedGrid, k, R, part, (const T *)nullptr,
         Prec<T>::Hk(c), Tm, gate);
    }
    if constexpr (std::is_same<T, float>::value) {
      if (tc)
        KL(c, "u_add_mr", c->stream, (k_u_add_mr_tc<TU>), (unsigned)((n + 127) / 128), 256, 0, (long long)n, k, U,
           Tm, Out, R, gate);
    }
    if (!tc)
      KL(c, "u_add_mr", c->stream, (k_u_add_mr<T, TU>), eblk((long long)n * R, bd), bd, 0, (long long)n, k, U, Tm,
         Out, R, gate);
  }
}

// Z = M^-1 Rr on FP64 blocks (scaling and precision handled here)
void precond_mr(ddlr_ctx *c, const double *Rr, double *Z, int R, const int *gate) {
  const int n = c->P.n;
  const long long nR = (long long)n * R;
  const int bd = c->bt.bd_elem;
  if (c->opt.precision == 0) {
    const double *in = Rr;
    if (c->dsc_dev) {
      KL(c, "vec_mr", c->stream, k_scale_rows_mr, eblk(nR, bd), bd, 0, (long long)n, R, c->dsc_dev, Rr, c->bt.S,
         gate);
      in = c->bt.S;
    }
    apply_mr<double, double>(c, c->U64, in, Z, R, gate);
    if (c->dsc_dev)
      KL(c, "vec_mr", c->stream, k_scale_rows_mr, eblk(nR, bd), bd, 0, (long long)n, R, c->dsc_dev, Z, Z, gate);
  } else {
    // scaling and change of precision in one pass each way
    float *i32 = c->bt.w32[5], *o32 = c->bt.w32[6];
    KL(c, "vec_mr", c->stream, (k_scale_cast_mr<float, double>), eblk((nR + 3) / 4, 256), 256, 0, (long long)n, R,
       c->dsc_dev, Rr, i32, gate);
    if (c->opt.uk_bf16) apply_mr<float, __nv_bfloat16>(c, c->Ub16, i32, o32, R, gate);
    else apply_mr<float, float>(c, c->U32, i32, o32, R, gate);
    KL(c, "vec_mr", c->stream, (k_scale_cast_mr<double, float>), eblk((nR + 3) / 4, 256), 256, 0, (long long)n, R,
       c->dsc_dev, o32, Z, gate);
  }
}

// Autotuner: block shapes of the batched solve kernels, picked by timing the
// candidates on the handle's own data (three preconditioner applications each,
// CUDA events) the first time a batch of this width is used.
void batch_autotune(ddlr_ctx *c, int R) {
  auto &B = c->bt;
  if (B.tuned) return;
  const bool timing = c->timing;
  c->timing = false;
  const long long l0 = c->launches;
  const std::vector<long long> f0 = c->fam_cnt;
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaMemsetAsync(B.Rr, 0, sizeof(double) * size_t(c->P.n) * R, c->stream), "memset");
  auto time_apply = [&]() {
    precond_mr(c, B.Rr, B.Z, R, nullptr);     // warm
    ck(cudaEventRecord(e0, c->stream), "event");
    for (int i = 0; i < 3; i++) precond_mr(c, B.Rr, B.Z, R, nullptr);
    ck(cudaEventRecord(e1, c->stream), "event");
    ck(cudaEventSynchronize(e1), "event");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  int best_c = B.chunk_per;
  float best = 1e30f;
  for (int mult : {1, 2, 4, 8, 16, 32}) {
    const int bd = R * mult;
    if (bd < 32 || bd > 1024) continue;
    B.chunk_per = mult;
    const float t = time_apply();
    if (t < best) { best = t; best_c = mult; }
  }
  B.chunk_per = best_c;
  int best_e = B.bd_elem;
  best = 1e30f;
  for (int bd : {128, 256, 512, 1024}) {
    B.bd_elem = bd;
    const float t = time_apply();
    if (t < best) { best = t; best_e = bd; }
  }
  B.bd_elem = best_e;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->launches = l0;                      // tuning launches are not the caller's work
  c->fam_cnt = f0;
  c->fam_cnt.resize(c->fam_names.size(), 0);
  c->timing = timing;
  B.tuned = true;
}

void pcg_mr_iteration(ddlr_ctx *c, int R, int flexible) {
  auto &B = c->bt;
  const int n = c->P.n;
  const long long nR = (long long)n * R;
  const int bd = B.bd_elem;
  const int *gate = reinterpret_cast<const int *>(reinterpret_cast<const char *>(B.st) +
                                                  offsetof(PcgStateMR, all_done));
  double *part = B.part64;
  // q = A p with the p.q partials, and the x, r update with the r.r partials,
  // in one pass each (64-row blocks, then the blocks of each reduction range)
  const unsigned nb = (unsigned)((n + kFbRows - 1) / kFbRows);
  const int fg = fb_groups(R);
  const unsigned fgrid = (nb + fg - 1) / fg, fthreads = unsigned(fg * kFbLanes * R);
  KL(c, "spmv_mr", c->stream, k_spmv_pq_mr, fgrid, fthreads, 0, n, c->a_soff, c->a_sw, c->a_col, c->a_val, B.P,
     B.Q, R, B.fpart, gate);
  KL(c, "pcg_mr_red", c->stream, k_fused_partials_reduce, kRedGrid, 64, 0, (int)nb, R, B.fpart, part, gate);
  KL(c, "pcg_mr_scalar", c->stream, k_pcgmr_alpha, 1, kScalarThreads, 0, B.st, part, kRedGrid);
  KL(c, "pcg_mr_axpy", c->stream, k_update_rr_mr, fgrid, fthreads, 0, (long long)n, B.st, B.P, B.Q, B.X, B.Rr,
     B.fpart);
  KL(c, "pcg_mr_red", c->stream, k_fused_partials_reduce, kRedGrid, 64, 0, (int)nb, R, B.fpart, part, gate);
  KL(c, "pcg_mr_scalar", c->stream, k_pcgmr_rr, 1, kScalarThreads, 0, B.st, part, kRedGrid);
  // the check kernels run on a bounded grid: most iterations they return at once
  const unsigned gchk = (unsigned)std::min<long long>(eblk(nR, bd), 152LL * 8);
  KL(c, "pcg_mr_check", c->stream, k_pcgmr_true_res, gchk, bd, 0, n, B.st, c->a_soff, c->a_sw, c->a_col, c->a_val,
     B.B, B.X, B.T);
  // T.T only when a column's true residual is checked this iteration
  const int *gate_chk = reinterpret_cast<const int *>(reinterpret_cast<const char *>(B.st) +
                                                      offsetof(PcgStateMR, no_check));
  KL(c, "pcg_mr_dot", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.T, B.T, (const double *)nullptr, part,
     gate_chk);
  KL(c, "pcg_mr_scalar", c->stream, k_pcgmr_true_dec, 1, kScalarThreads, 0, B.st, part, kRedGrid);
  KL(c, "pcg_mr_check", c->stream, k_pcgmr_copy_r, gchk, bd, 0, (long long)n, B.st, B.T, B.Rr);
  precond_mr(c, B.Rr, B.Z, R, gate);
  KL(c, "pcg_mr_dot", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.Rr, B.Z, flexible ? B.Zo : B.Z, part, gate);
  KL(c, "pcg_mr_scalar", c->stream, k_pcgmr_beta, 1, kScalarThreads, 0, B.st, part, kRedGrid);
  KL(c, "pcg_mr_p", c->stream, k_pcgmr_p, eblk(nR, bd), bd, 0, (long long)n, B.st, B.Z, B.P, flexible ? B.Zo : (double *)nullptr);
}

// the captured graph of one batched iteration of width R on c->stream (a
// stream in capture mode must not be the caller's legacy stream, so callers
// capture on the handle's internal stream)
void mr_graph(ddlr_ctx *c, int R, int flexible) {
  auto &GR = c->bt.graphs[R];
  if (GR.exec != nullptr && GR.flex == flexible) return;
  if (GR.exec) { cudaGraphExecDestroy(GR.exec); GR.exec = nullptr; }
  const long long l0 = c->launches;
  const std::vector<long long> f0 = c->fam_cnt;
  ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture");
  pcg_mr_iteration(c, R, flexible);
  cudaGraph_t g = nullptr;
  ck(cudaStreamEndCapture(c->stream, &g), "capture");
  cudaError_t e = cudaGraphInstantiate(&GR.exec, g, 0);
  cudaGraphDestroy(g);
  ck(e, "cudaGraphInstantiate");
  GR.flex = flexible;
  GR.nodes = c->launches - l0;
  GR.fam_nodes.assign(c->fam_cnt.size(), 0);
  for (size_t i = 0; i < c->fam_cnt.size(); i++)
    GR.fam_nodes[i] = c->fam_cnt[i] - (i < f0.size() ? f0[i] : 0);
  c->launches = l0;
  for (size_t i = 0; i < f0.size(); i++) c->fam_cnt[i] = f0[i];
  for (size_t i = f0.size(); i < c->fam_cnt.size(); i++) c->fam_cnt[i] = 0;
}

// one batched iteration of width R on c->stream (the graph when use_graph)
void mr_iterate(ddlr_ctx *c, int R, int flexible, bool use_graph) {
  if (use_graph) {
    auto &GR = c->bt.graphs[R];
    ck(cudaGraphLaunch(GR.exec, c->stream), "cudaGraphLaunch");
    c->launches += GR.nodes;
    for (size_t i = 0; i < GR.fam_nodes.size(); i++) c->fam_cnt[i] += GR.fam_nodes[i];
  } else {
    pcg_mr_iteration(c, R, flexible);
  }
}

// block PCG on B.B (device order, row-major, R columns) -> B.X
void pcg_mr_dev(ddlr_ctx *c, int R, double tol, int maxit, ddlr_solve_info *info) {
  auto &B = c->bt;
  const int n = c->P.n;
  const long long nR = (long long)n * R;
  const int flexible = c->opt.precision == 1 ? 1 : 0;
  const int *gate = reinterpret_cast<const int *>(reinterpret_cast<const char *>(B.st) +
                                                  offsetof(PcgStateMR, all_done));
  const char *ng = getenv("DDLR_NO_GRAPH");
  const bool use_graph = !c->timing && !(ng && ng[0] == '1');
  cudaStream_t user = c->stream;
  struct Restore {
    ddlr_ctx *c; cudaStream_t s;
    ~Restore() { c->stream = s; }
  } restore{c, user};
  if (use_graph) {
    ck(cudaEventRecord(c->ev_fork, user), "event");
    ck(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0), "wait");
    c->stream = c->gstream;
  }
  batch_autotune(c, R);
  B.last_R = R;
  double *part = B.part64;
  const int bd = B.bd_elem;
  ck(cudaMemsetAsync(B.X, 0, sizeof(double) * nR, c->stream), "memset");
  ck(cudaMemcpyAsync(B.Rr, B.B, sizeof(double) * nR, cudaMemcpyDeviceToDevice, c->stream), "copy");
  KL(c, "pcg_mr", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.B, B.B, (const double *)nullptr, part, (const int *)nullptr);
  KL(c, "pcg_mr", c->stream, k_pcgmr_init, 1, kScalarThreads, 0, B.st, part, kRedGrid, R, tol, maxit, flexible);
  precond_mr(c, B.Rr, B.Z, R, gate);
  KL(c, "pcg_mr", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.Rr, B.Z, (const double *)nullptr, part, gate);
  KL(c, "pcg_mr", c->stream, k_pcgmr_rz0, 1, kScalarThreads, 0, B.st, part, kRedGrid);
  ck(cudaMemcpyAsync(B.P, B.Z, sizeof(double) * nR, cudaMemcpyDeviceToDevice, c->stream), "copy");
  ck(cudaMemcpyAsync(B.Zo, B.Z, sizeof(double) * nR, cudaMemcpyDeviceToDevice, c->stream), "copy");
  if (use_graph) mr_graph(c, R, flexible);
  const int batch = 4;
  for (int it = 0; it < maxit + batch; it += batch) {
    for (int bi = 0; bi < batch; bi++) mr_iterate(c, R, flexible, use_graph);
    int done = 0;
    ck(cudaMemcpyAsync(c->h_pin, gate, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "D2H");
    ck(cudaStreamSynchronize(c->stream), "sync");
    std::memcpy(&done, c->h_pin, sizeof(int));
    if (done) break;
  }
  // true residuals
  KL(c, "spmv_mr", c->stream, k_spmv_mr<double>, eblk(nR, bd), bd, 0, n, c->a_soff, c->a_sw, c->a_col,
     c->a_val, B.X, B.Q, R, (const int *)nullptr);
  KL(c, "pcg_mr", c->stream, k_sub_mr, eblk(nR, bd), bd, 0, nR, B.B, B.Q, B.T);
  KL(c, "pcg_mr", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.T, B.T, (const double *)nullptr, part, (const int *)nullptr);
  std::vector<double> hp(size_t(kRedGrid) * 2 * R);
  PcgStateMR hs;
  int dfl[4];
  ck(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaMemcpyAsync(&hs, B.st, sizeof(PcgStateMR), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaMemcpyAsync(dfl, c->dflag, sizeof(dfl), cudaMemcpyDeviceToHost, c->stream), "D2H");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (use_graph) {
    ck(cudaEventRecord(c->ev_join, c->stream), "event");
    ck(cudaStreamWaitEvent(user, c->ev_join, 0), "wait");
  }
  if (dfl[3]) timeout_fail(c);
  for (int q = 0; q < R; q++) {
    double rt2 = 0;
    for (int g = 0; g < kRedGrid; g++) rt2 += hp[size_t(g) * 2 * R + q];   // fixed order
    info[q].its = hs.its[q];
    info[q].relres = hs.bb[q] > 0 ? std::sqrt(rt2 / hs.bb[q]) : 0.0;
    info[q].status = hs.status[q] == 0 ? DDLR_OK : (hs.status[q] == 5 ? DDLR_ERR_NOCONV : DDLR_ERR_NAN);
    if (!hs.done[q]) info[q].status = DDLR_ERR_NOCONV;
  }
}

// a group of R columns of the caller's vectors (host or device, column-major,
// original order) in and out of the batch layout
void batch_load(ddlr_ctx *c, const double *x, int ld, int R, bool host, double *dst) {
  const int n = c->P.n;
  const double *src = x;
  if (host) {
    ck(cudaMemcpy2DAsync(c->bt.S, sizeof(double) * n, x, sizeof(double) * size_t(ld), sizeof(double) * n, R,
                         cudaMemcpyHostToDevice, c->stream), "H2D");
    src = c->bt.S;
  }
  KL(c, "perm", c->stream, k_batch_in, eblk((long long)n * R, 256), 256, 0, n, R, c->perm, src,
     host ? (long long)n : (long long)ld, dst);
}
void batch_store(ddlr_ctx *c, const double *srcb, double *y, int ld, int R, bool host) {
  const int n = c->P.n;
  double *dst = host ? c->bt.S : y;
  KL(c, "perm", c->stream, k_batch_out, eblk((long long)n * R, 256), 256, 0, n, R, c->perm, srcb, dst,
     host ? (long long)n : (long long)ld);
  if (host) {
    ck(cudaMemcpy2DAsync(y, sizeof(double) * size_t(ld), c->bt.S, sizeof(double) * n, sizeof(double) * n, R,
                         cudaMemcpyDeviceToHost, c->stream), "D2H");
    sync(c);
  }
}

}  // namespace

// ====================================================================== ABI

namespace {
// A bounded device wait ran out: clear the flag (the next call starts clean)
// and report DDLR_ERR_TIMEOUT
void clear_timeout(ddlr_ctx *c) {
  cudaMemsetAsync(c->dflag + 3, 0, sizeof(int), c->stream);
  cudaStreamSynchronize(c->stream);
}
[[noreturn]] void timeout_fail(ddlr_ctx *c) {
  clear_timeout(c);
  throw Fail{DDLR_ERR_TIMEOUT, "a bounded device wait timed out"};
}

ddlr_status run_guarded(ddlr_ctx *c, const std::function<ddlr_status()> &f) {
  // a launch error left by an earlier call that already returned its own
  // status is not this call's error
  cudaGetLastError();
  try {
    ddlr_status st = f();
    if (st == DDLR_OK) {
      cudaError_t e = cudaPeekAtLastError();
      if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DDLR_ERR_CUDA; }
    }
    return st;
  } catch (const Fail &f2) {
    c->err = f2.msg;
    return f2.st;
  } catch (const std::bad_alloc &) {
    c->err = "host allocation failed";
    return DDLR_ERR_OOM;
  } catch (const std::exception &e) {
    c->err = e.what();
    return DDLR_ERR_INVALID;
  }
}

}  // namespace

// ------------------------------------------------ continuous batching (serving)
// A block PCG of width R whose columns ("slots") are admitted and retired
// between iterations (ddlr_batch.cuh, continuous batching).  The block's
// buffers and per-column state stay on the device; idle slots are done
// columns, which the step kernels skip.
namespace {
struct SlotSolver {
  bool open = false;
  int R = 0, maxit = 500;
  double tol = 1e-8;
  int *mask = nullptr;           // device, kMaxR ints
  PcgStateMR hs{};               // host copy after the last run
};
std::mutex g_slots_mu;
std::map<ddlr_ctx *, SlotSolver> g_slots;
SlotSolver &slots_of(ddlr_ctx *c) {
  std::lock_guard<std::mutex> lk(g_slots_mu);
  return g_slots[c];
}
// capture the iteration graph of width R on the internal stream
void slots_capture(ddlr_ctx *c, int R, int flexible) {
  cudaStream_t user = c->stream;
  ck(cudaEventRecord(c->ev_fork, user), "event");
  ck(cudaStreamWaitEvent(c->gstream, c->ev_fork, 0), "wait");
  c->stream = c->gstream;
  try {
    mr_graph(c, R, flexible);
  } catch (...) {
    c->stream = user;
    throw;
  }
  ck(cudaEventRecord(c->ev_join, c->stream), "event");
  ck(cudaStreamWaitEvent(user, c->ev_join, 0), "wait");
  c->stream = user;
}
}  // namespace

ddlr_status slots_open(ddlr_ctx *c, int R, double tol, int maxit) {
  return run_guarded(c, [&]() -> ddlr_status {
    if (R < 1 || R > std::min(kMaxR, std::max(1, batch_width(c)))) throw Fail{DDLR_ERR_INVALID, "slot width"};
    SlotSolver &S = slots_of(c);
    auto &B = c->bt;
    batch_alloc(c, R);
    batch_autotune(c, R);
    B.last_R = R;
    if (!S.mask) S.mask = c->alloc<int>(kMaxR);
    const size_t nR = size_t(c->P.n) * R;
    for (double *v : {B.B, B.X, B.Rr, B.Z, B.P, B.Zo, B.Q, B.T})
      ck(cudaMemsetAsync(v, 0, sizeof(double) * nR, c->stream), "memset");
    PcgStateMR h{};
    h.R = R; h.maxit = maxit; h.flexible = c->opt.precision == 1 ? 1 : 0;
    h.all_done = 1; h.no_check = 1;
    for (int q = 0; q < kMaxR; q++) h.done[q] = 1;
    ck(cudaMemcpyAsync(B.st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream), "H2D");
    S.hs = h;
    S.R = R; S.tol = tol; S.maxit = maxit; S.open = true;
    const char *ng = getenv("DDLR_NO_GRAPH");
    if (!(c->timing || (ng && ng[0] == '1'))) slots_capture(c, R, h.flexible);
    sync(c);
    return DDLR_OK;
  });
}

// lay the open block out again as R1 columns, new column q = old column
// map[q] (map[q] < 0: a new idle column): every FP64 block that carries state
// across iterations is moved, and the per-column state with it, so the moved
// columns continue exactly as before (widening, and narrowing to the busy
// columns)
ddlr_status slots_resize(ddlr_ctx *c, int R1, const int *map) {
  return run_guarded(c, [&]() -> ddlr_status {
    SlotSolver &S = slots_of(c);
    if (!S.open) throw Fail{DDLR_ERR_INVALID, "no open slots"};
    const int R0 = S.R;
    if (R1 < 1 || R1 > std::min(kMaxR, std::max(1, batch_width(c)))) throw Fail{DDLR_ERR_INVALID, "slot width"};
    for (int q = 0; q < R1; q++)
      if (map[q] >= R0) throw Fail{DDLR_ERR_INVALID, "slot map"};
    const long long n = c->P.n;
    auto &B = c->bt;
    std::vector<void *> tmp;
    double *src[5] = {B.B, B.X, B.Rr, B.P, B.Zo};
    double *save[5];
    for (int i = 0; i < 5; i++) {
      void *p = nullptr;
      ck(cudaMallocAsync(&p, sizeof(double) * size_t(n) * R0, c->stream), "cudaMallocAsync");
      tmp.push_back(p);
      save[i] = static_cast<double *>(p);
      ck(cudaMemcpyAsync(save[i], src[i], sizeof(double) * size_t(n) * R0, cudaMemcpyDeviceToDevice, c->stream),
         "copy");
    }
    PcgStateMR o{};
    ck(cudaMemcpyAsync(&o, B.st, sizeof(o), cudaMemcpyDeviceToHost, c->stream), "D2H");
    sync(c);
    // the per-column state, permuted on the host
    PcgStateMR st = o;
    for (int q = 0; q < kMaxR; q++) {
      const int f = q < R1 ? map[q] : -1;
      if (f >= 0) {
        st.rz[q] = o.rz[f]; st.pq[q] = o.pq[f]; st.alpha[q] = o.alpha[f]; st.beta[q] = o.beta[f];
        st.rr[q] = o.rr[f]; st.bb[q] = o.bb[f]; st.tol2[q] = o.tol2[f]; st.rt2[q] = o.rt2[f];
        st.its[q] = o.its[f]; st.done[q] = o.done[f]; st.status[q] = o.status[f]; st.check[q] = o.check[f];
        st.restart[q] = o.restart[f]; st.fresh[q] = o.fresh[f];
      } else {
        st.rz[q] = st.pq[q] = st.alpha[q] = st.beta[q] = st.rr[q] = st.bb[q] = st.tol2[q] = st.rt2[q] = 0.0;
        st.its[q] = 0; st.done[q] = 1; st.status[q] = 0; st.check[q] = 0; st.restart[q] = 0; st.fresh[q] = 0;
      }
    }
    st.R = R1;
    int all = 1;
    for (int q = 0; q < R1; q++) all &= st.done[q];
    st.all_done = all;
    batch_alloc(c, R1);                  // reallocates the block buffers when wider than before
    batch_autotune(c, R1);
    B.last_R = R1;
    int hmap[kMaxR];
    for (int q = 0; q < kMaxR; q++) hmap[q] = q < R1 ? map[q] : -1;
    ck(cudaMemcpyAsync(S.mask, hmap, sizeof(hmap), cudaMemcpyHostToDevice, c->stream), "H2D");
    ck(cudaMemcpyAsync(B.st, &st, sizeof(st), cudaMemcpyHostToDevice, c->stream), "H2D");
    double *dst[5] = {B.B, B.X, B.Rr, B.P, B.Zo};
    for (int i = 0; i < 5; i++)
      KL(c, "slots", c->stream, k_relayout, eblk(n * R1, 256), 256, 0, n, R0, R1, S.mask, save[i], dst[i]);
    for (double *v : {B.Z, B.Q, B.T})
      ck(cudaMemsetAsync(v, 0, sizeof(double) * size_t(n) * R1, c->stream), "memset");
    for (void *p : tmp) ck(cudaFreeAsync(p, c->stream), "cudaFreeAsync");
    S.R = R1;
    S.hs = st;
    const char *ng = getenv("DDLR_NO_GRAPH");
    if (!(c->timing || (ng && ng[0] == '1'))) slots_capture(c, R1, c->opt.precision == 1 ? 1 : 0);
    sync(c);
    return DDLR_OK;
  });
}

// admit right-hand sides b[i] (host, original order) into free slots slot[i]
ddlr_status slots_admit(ddlr_ctx *c, int cnt, const int *slot, const double *const *b) {
  return run_guarded(c, [&]() -> ddlr_status {
    SlotSolver &S = slots_of(c);
    if (!S.open) throw Fail{DDLR_ERR_INVALID, "no open slots"};
    const int n = c->P.n, R = S.R;
    auto &B = c->bt;
    int hm[kMaxR] = {0};
    for (int i = 0; i < cnt; i++) {
      const int q = slot[i];
      if (q < 0 || q >= R || hm[q] || !S.hs.done[q]) throw Fail{DDLR_ERR_INVALID, "slot not free"};
      hm[q] = 1;
      // staging: the first n doubles of the S block per admitted column
      ck(cudaMemcpyAsync(B.S, b[i], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "H2D");
      KL(c, "slots", c->stream, k_col_in, nblk(n), kThreads, 0, n, R, q, c->perm, B.S, B.B);
    }
    ck(cudaMemcpyAsync(S.mask, hm, sizeof(hm), cudaMemcpyHostToDevice, c->stream), "H2D");
    KL(c, "slots", c->stream, k_slot_reset, eblk((long long)n * R, 256), 256, 0, (long long)n, R, S.mask, B.B, B.X,
       B.Rr, B.P);
    KL(c, "slots", c->stream, k_dot_mr_partial, kRedGrid, 256, 0, (long long)n, R, B.B, B.B, (const double *)nullptr,
       B.part64, (const int *)nullptr);
    KL(c, "slots", c->stream, k_slot_init, 1, kScalarThreads, 0, B.st, B.part64, kRedGrid, S.mask, R, S.tol,
       S.maxit, c->opt.precision == 1 ? 1 : 0);
    sync(c);       // the host vectors may be released when this returns
    for (int i = 0; i < cnt; i++) S.hs.done[slot[i]] = 0;
    return DDLR_OK;
  });
}

// run `iters` iterations of the open block; done[q] (host, R ints) then
// tells which slots have finished (idle slots included)
ddlr_status slots_run(ddlr_ctx *c, int iters, int *done) {
  return run_guarded(c, [&]() -> ddlr_status {
    SlotSolver &S = slots_of(c);
    if (!S.open) throw Fail{DDLR_ERR_INVALID, "no open slots"};
    const int flexible = c->opt.precision == 1 ? 1 : 0;
    const char *ng = getenv("DDLR_NO_GRAPH");
    const bool use_graph = !(c->timing || (ng && ng[0] == '1'));
    if (use_graph && !c->bt.graphs[S.R].exec) slots_capture(c, S.R, flexible);
    for (int i = 0; i < iters; i++) mr_iterate(c, S.R, flexible, use_graph);
    int dfl[4];
    ck(cudaMemcpyAsync(&S.hs, c->bt.st, sizeof(S.hs), cudaMemcpyDeviceToHost, c->stream), "D2H");
    ck(cudaMemcpyAsync(dfl, c->dflag, sizeof(dfl), cudaMemcpyDeviceToHost, c->stream), "D2H");
    sync(c);
    if (dfl[3]) timeout_fail(c);
    for (int q = 0; q < S.R; q++) done[q] = S.hs.done[q];
    return DDLR_OK;
  });
}

// the result of a finished slot (x: host, original order); the slot is free
// afterwards.  relres: the true residual of the check that ended the solve
// (status OK), else the recursive residual.
ddlr_status slots_take(ddlr_ctx *c, int slot, double *x, ddlr_solve_info *info) {
  return run_guarded(c, [&]() -> ddlr_status {
    SlotSolver &S = slots_of(c);
    if (!S.open || slot < 0 || slot >= S.R || !S.hs.done[slot]) throw Fail{DDLR_ERR_INVALID, "slot not finished"};
    const int n = c->P.n;
    auto &B = c->bt;
    KL(c, "slots", c->stream, k_col_out, nblk(n), kThreads, 0, n, S.R, slot, c->perm, B.X, B.S);
    ck(cudaMemcpyAsync(x, B.S, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "D2H");
    sync(c);
    const PcgStateMR &h = S.hs;
    info->its = h.its[slot];
    const double bb = h.bb[slot];
    const double r2 = h.status[slot] == 0 ? h.rt2[slot] : h.rr[slot];
    info->relres = bb > 0 ? std::sqrt(r2 / bb) : 0.0;
    info->status = h.status[slot] == 0 ? DDLR_OK : (h.status[slot] == 5 ? DDLR_ERR_NOCONV : DDLR_ERR_NAN);
    return DDLR_OK;
  });
}

int slots_width(ddlr_ctx *c) { return slots_of(c).R; }

void slots_forget(ddlr_ctx *c) {
  std::lock_guard<std::mutex> lk(g_slots_mu);
  g_slots.erase(c);
}

extern "C" {

ddlr_status ddlr_options_default(ddlr_options *o) {
  if (!o) return DDLR_ERR_INVALID;
  std::memset(o, 0, sizeof(*o));
  o->variant = 1;
  o->rank_k = 16;
  o->alpha = 1.0;
  o->theta_mode = 1;
  o->factor = 0;
  o->c_order = 0;
  o->b_order = 0;
  o->precision = 0;
  o->uk_bf16 = 0;
  o->scale_diag = 0;
  o->lanczos_max = 0;
  o->lanczos_check = 10;
  o->lanczos_eps = 1e-4;
  o->seed = 0;
  o->max_nrhs = 1;
  o->c_solver = 0;
  o->cheb_steps = 5;
  o->cheb_lanczos = 20;
  o->lowrank_method = 0;
  o->rand_oversample = 10;
  o->rand_power = 2;
  o->mr_iters = 3;
  o->mr_lfil = 8;
  o->mr_droptol = 1e-3;
  o->indefinite = 0;
  o->fill_level = 0;
  o->lanczos_reorth = 0;
  o->wait_limit_s = 2.0;
  return DDLR_OK;
}

ddlr_status ddlr_setup(int n, const int *rowptr, const int *colind, const double *val,
                       const int *part, int p, const ddlr_options *opt, void *cuda_stream,
                       ddlr_handle *out) {
  if (!out) return DDLR_ERR_INVALID;
  *out = nullptr;
  auto t0 = std::chrono::steady_clock::now();
  ddlr_options o;
  if (opt) o = *opt; else ddlr_options_default(&o);
  if ((o.variant != 1 && o.variant != 2) || !(o.alpha > 0) || (o.precision != 0 && o.precision != 1) ||
      o.factor < 0 || o.factor > 3 ||
      (o.factor >= 2 && (o.precision != 0 || o.c_solver != 0 || o.lowrank_method == 1)) ||
      (o.c_order != 0 && o.c_order != 1) ||
      (o.b_order != 0 && o.b_order != 1) || o.rank_k < 1 ||
      o.rank_k > 256 || o.c_solver < 0 || o.c_solver > 2 ||
      (o.c_solver == 2 && (o.mr_iters < 0 || o.mr_lfil < 1 || o.mr_lfil >= kMrCap ||
                           1 + (long long)o.mr_iters * o.mr_lfil > kMrCap || !(o.mr_droptol >= 0.0))) ||
      (o.c_solver == 1 && (o.cheb_steps < 1 || o.cheb_steps > kChebMaxSteps || o.cheb_lanczos < 1 ||
                           o.cheb_lanczos > 1000)) ||
      o.lowrank_method < 0 || o.lowrank_method > 2 || (o.lowrank_method == 2 && o.variant != 2) ||
      (o.indefinite != 0 && o.indefinite != 1) || o.fill_level < 0 || o.fill_level > 64 ||
      (o.fill_level > 0 && (o.factor == 1 || o.factor == 3)) ||
      (o.lanczos_reorth != 0 && o.lanczos_reorth != 1) || !(o.wait_limit_s > 0) || o.wait_limit_s > 3600 ||
      (o.lowrank_method == 1 && (o.rand_oversample < 0 || o.rand_power < 0 || o.rand_power > 100 ||
                                 o.rank_k + o.rand_oversample > kRandMaxL))) {
    g_setup_error = "invalid options";
    return DDLR_ERR_INVALID;
  }
  if (o.lanczos_check < 0) o.lanczos_check = 0;
  ddlr_ctx *c = new (std::nothrow) ddlr_ctx();
  if (!c) { g_setup_error = "host allocation failed"; return DDLR_ERR_OOM; }
  c->opt = o;
  c->stream = (cudaStream_t)cuda_stream;
  c->wait_ns = (unsigned long long)(o.wait_limit_s * 1e9);
  ddlr_status st = run_guarded(c, [&]() -> ddlr_status {
    std::string err;
    ddlr_status s1 = build_plan(n, rowptr, colind, val, part, p, c->opt, c->P, err);
    if (s1 != DDLR_OK) { c->err = err; return s1; }
    ck(cudaGetDevice(&c->device), "cudaGetDevice");
    if (c->opt.c_solver == 2) {
      // the per-column work of the MR iterations holds r_j and C_a z_j in
      // fixed local arrays: rows of C_a times the column capacity must fit
      int maxc = 0;
      for (int i = 0; i < c->P.s; i++) maxc = std::max(maxc, c->P.cc_rp[i + 1] - c->P.cc_rp[i]);
      const long long cap = 1 + (long long)c->opt.mr_iters * c->opt.mr_lfil;
      if (cap * maxc + 1 > kMrCand || (long long)c->opt.mr_lfil * maxc > kMrCand) {
        c->err = "c_solver 2: (1 + mr_iters * mr_lfil) x the longest row of C_a exceeds 256";
        return DDLR_ERR_INVALID;
      }
    }
    c->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ck(cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    ck(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    allocate(c);
    ck(cudaMemcpyAsync(c->val, val, sizeof(double) * c->P.nnz, cudaMemcpyHostToDevice, c->stream), "H2D");
    return numeric_setup(c);
  });
  if (st != DDLR_OK) {
    g_setup_error = c->err;
    ddlr_destroy(c);
    return st;
  }
  c->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return DDLR_OK;
}

ddlr_status ddlr_refactor(ddlr_handle c, const double *val) {
  if (!c) return DDLR_ERR_INVALID;
  return run_guarded(c, [&]() -> ddlr_status {
    if (val)
      ck(cudaMemcpyAsync(c->val, val, sizeof(double) * c->P.nnz, cudaMemcpyDefault, c->stream), "copy values");
    return numeric_setup(c);
  });
}

ddlr_status ddlr_increase_rank(ddlr_handle c, int k_new) {
  if (!c) return DDLR_ERR_INVALID;
  const Plan &P = c->P;
  const int k_old = c->opt.rank_k;
  if (k_new <= k_old || k_new > P.s || k_new > 256) {
    c->err = "ddlr_increase_rank: need rank_k < k_new <= min(s, 256)";
    return DDLR_ERR_INVALID;
  }
  if (c->opt.lowrank_method != 0) {
    c->err = "ddlr_increase_rank continues the Lanczos process: lowrank_method 0 only";
    return DDLR_ERR_INVALID;
  }
  if (!c->lw.ready) { c->err = "ddlr_increase_rank: no Lanczos state"; return DDLR_ERR_INVALID; }
  return run_guarded(c, [&]() -> ddlr_status {
    ck(cudaStreamSynchronize(c->stream), "sync");
    ck(cudaStreamSynchronize(c->stream2), "sync");
    auto mmax_of = [&](int k) {
      int mm = c->opt.lanczos_max > 0 ? c->opt.lanczos_max : 5 * k;
      return std::max(std::min(mm, P.s), k);
    };
    const int m_old = mmax_of(k_old), m_new = mmax_of(k_new);
    const int s = P.s, n = P.n, k = k_new;
    auto &W = c->lw;
    // graphs hold the old arrays' addresses
    if (W.exec) { cudaGraphExecDestroy(W.exec); W.exec = nullptr; }
    if (c->pcg_exec) { cudaGraphExecDestroy(c->pcg_exec); c->pcg_exec = nullptr; }
    c->gm.free_graphs();
    batch_free(c);
    // Lanczos workspace for m_new steps: the basis and T_j carried over (the
    // old arrays stay in the handle's arena until it is destroyed)
    if (m_new > m_old) {
      double *Q = c->alloc<double>(size_t(s) * size_t(m_new + 1));
      double *al = c->alloc<double>(m_new + 1), *be = c->alloc<double>(m_new + 1);
      ck(cudaMemsetAsync(be, 0, sizeof(double) * (m_new + 1), c->stream), "memset");
      ck(cudaMemcpyAsync(Q, W.Q, sizeof(double) * size_t(s) * size_t(m_old + 1), cudaMemcpyDeviceToDevice,
                         c->stream), "copy");
      ck(cudaMemcpyAsync(al, W.al, sizeof(double) * (m_old + 1), cudaMemcpyDeviceToDevice, c->stream), "copy");
      ck(cudaMemcpyAsync(be, W.be, sizeof(double) * (m_old + 1), cudaMemcpyDeviceToDevice, c->stream), "copy");
      W.Q = Q; W.al = al; W.be = be;
      W.Q32 = nullptr;   // allocated again at the next persistent Lanczos launch
      W.cvec = c->alloc<double>(m_new + 2);
      W.evals = c->alloc<double>(m_new);
    }
    W.ework = c->alloc<double>(5 * size_t(m_new) * k);
    W.etop = c->alloc<double>(2 * k + 1);
    W.eY = c->alloc<double>(size_t(m_new) * k);
    if (c->opt.variant == 2) {
      W.V = c->alloc<double>(size_t(s) * k);
      W.EV = c->alloc<double>(size_t(n) * k);
      W.kp = c->alloc<double>(size_t(kRedGrid) * k * k);
      W.hw = c->alloc<double>(size_t(k) * k + k);
    }
    // low-rank data and reduction buffers for k_new
    c->opt.rank_k = k;
    c->U64 = c->alloc<double>(size_t(c->urows) * k);
    c->coef64 = c->alloc<double>(k);
    c->Hk64 = c->alloc<double>(size_t(k) * k);
    ck(cudaMemsetAsync(c->coef64, 0, sizeof(double) * k, c->stream), "memset");
    ck(cudaMemsetAsync(c->Hk64, 0, sizeof(double) * k * k, c->stream), "memset");
    c->part64 = c->alloc<double>(size_t(kRedGrid) * std::max(k + 2, m_new + 2) + 2 * kRedGrid);
    if (c->opt.precision == 1) {
      if (c->opt.uk_bf16) c->Ub16 = c->alloc<__nv_bfloat16>(size_t(c->urows) * k);
      else c->U32 = c->alloc<float>(size_t(c->urows) * k);
      c->coef32 = c->alloc<float>(k);
      c->Hk32 = c->alloc<float>(size_t(k) * k);
      c->part32 = c->alloc<float>(size_t(kRedGrid) * (k + 2));
    }
    if (c->pz_pcg || c->pz_lz) pz_setup(c, m_new);
    const ddlr_status st = run_lanczos(c, true);
    if (st != DDLR_OK) {
      c->err = lowrank_error(c, st);
      return st;
    }
    make_low_precision(c);
    sync(c);
    return DDLR_OK;
  });
}

static ddlr_status vec_call(ddlr_ctx *c, const double *x, double *y, int nrhs, int ld,
                            const std::function<void(const double *, double *)> &body) {
  if (!c) return DDLR_ERR_INVALID;
  const int n = c->P.n;
  if (!x || !y || nrhs < 1 || ld < n) { c->err = "invalid vector arguments"; return DDLR_ERR_INVALID; }
  return run_guarded(c, [&]() -> ddlr_status {
    const bool hx = !is_device_ptr(x), hy = !is_device_ptr(y);
    for (int j = 0; j < nrhs; j++) {
      const double *xj = x + size_t(j) * ld;
      double *yj = y + size_t(j) * ld;
      const double *xd = xj;
      double *yd = yj;
      if (hx) {
        ck(cudaMemcpyAsync(c->stg_in, xj, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "H2D");
        xd = c->stg_in;
      }
      if (hy) yd = c->stg_out;
      body(xd, yd);
      if (hy) {
        ck(cudaMemcpyAsync(yj, yd, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "D2H");
        sync(c);
      }
    }
    return DDLR_OK;
  });
}

ddlr_status ddlr_apply(ddlr_handle c, const double *x, double *y, int nrhs, int ld) {
  if (c && nrhs > 1 && batch_width(c) >= 2) {
    const int n = c->P.n;
    if (!x || !y || ld < n) { c->err = "invalid vector arguments"; return DDLR_ERR_INVALID; }
    return run_guarded(c, [&]() -> ddlr_status {
      const bool hx = !is_device_ptr(x), hy = !is_device_ptr(y);
      const int W = batch_width(c);
      for (int j0 = 0; j0 < nrhs; j0 += W) {
        const int R = std::min(W, nrhs - j0);
        batch_alloc(c, R);
        batch_autotune(c, R);
        c->bt.last_R = R;
        batch_load(c, x + size_t(j0) * ld, ld, R, hx, c->bt.Rr);
        precond_mr(c, c->bt.Rr, c->bt.Z, R, nullptr);
        batch_store(c, c->bt.Z, y + size_t(j0) * ld, ld, R, hy);
      }
      return DDLR_OK;
    });
  }
  return vec_call(c, x, y, nrhs, ld, [c](const double *xd, double *yd) {
    const int n = c->P.n;
    double *xi = c->pv[1], *yo = c->pv[2];
    KL(c, "perm", c->stream, k_permute_in<double>, nblk(n), kThreads, 0, n, c->perm, xd, xi);
    precond(c, xi, yo, nullptr);
    KL(c, "perm", c->stream, k_permute_out<double>, nblk(n), kThreads, 0, n, c->perm, yo, yd);
  });
}

ddlr_status ddlr_a0_solve(ddlr_handle c, const double *x, double *y, int nrhs, int ld) {
  return vec_call(c, x, y, nrhs, ld, [c](const double *xd, double *yd) {
    const int n = c->P.n;
    double *xi = c->pv[1], *yo = c->pv[2];
    KL(c, "perm", c->stream, k_permute_in<double>, nblk(n), kThreads, 0, n, c->perm, xd, xi);
    if (c->opt.precision == 0) {
      a0_solve<double>(c, xi, yo, nullptr);
    } else {
      KL(c, "vec", c->stream, (k_cast<float, double>), nblk(n), kThreads, 0, (long long)n, xi, c->w32[6], (const int *)nullptr);
      a0_solve<float>(c, c->w32[6], c->w32[7], nullptr);
      KL(c, "vec", c->stream, (k_cast<double, float>), nblk(n), kThreads, 0, (long long)n, c->w32[7], yo, (const int *)nullptr);
    }
    KL(c, "perm", c->stream, k_permute_out<double>, nblk(n), kThreads, 0, n, c->perm, yo, yd);
  });
}

}  // extern "C"

// ------------------------------------------------- A0 solve without allocation
// Scratch of ddlr_a0_solve_noalloc: the permuted right-hand side and the
// permuted result, at most kNoAllocMaxN rows each (16 MiB; every GPU that
// loads the library holds it until the process exits).
namespace {
constexpr int kNoAllocMaxN = 1 << 20;
}
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxN];
static_assert(sizeof(g_noalloc_scratch) == 2 * size_t(kNoAllocMaxN) * sizeof(double),
              "the two vectors of the no-allocation solve must fit the array");

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[128] = {nullptr};   // device address of the scratch, per device
}

extern "C" {

ddlr_status ddlr_a0_solve_noalloc(ddlr_handle c, const double *x, double *y) {
  if (!c) return DDLR_ERR_INVALID;
  const int n = c->P.n;
  if (!x || !y) { c->err = "NULL vector"; return DDLR_ERR_INVALID; }
  if (n > kNoAllocMaxN) {
    c->err = "ddlr_a0_solve_noalloc: n = " + std::to_string(n) + " exceeds its limit of " +
             std::to_string(kNoAllocMaxN) + " rows";
    return DDLR_ERR_INVALID;
  }
  if (c->opt.precision != 0) { c->err = "ddlr_a0_solve_noalloc: FP64 handles only"; return DDLR_ERR_INVALID; }
  if (!is_device_ptr(x) || !is_device_ptr(y)) {
    c->err = "ddlr_a0_solve_noalloc: x and y must be device memory";
    return DDLR_ERR_INVALID;
  }
  const bool timing = c->timing;
  c->timing = false;   // per-kernel timing would create events
  ddlr_status st = run_guarded(c, [&]() -> ddlr_status {
    // the array's address is per device: look it up on the handle's device,
    // which must be the current one (a kernel given another device's address
    // would read that device's memory)
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != c->device)
      throw Fail{DDLR_ERR_INVALID, "ddlr_a0_solve_noalloc: the current device (" + std::to_string(dev) +
                                       ") is not the handle's device (" + std::to_string(c->device) + ")"};
    if (dev < 0 || dev >= 128) throw Fail{DDLR_ERR_INVALID, "device index out of range"};
    double *scratch = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_noalloc_mu);
      if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        ck(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<double *>(ptr);
      }
      scratch = g_noalloc_ptr[dev];
    }
    double *xi = scratch, *yo = scratch + kNoAllocMaxN;
    k_permute_in<double><<<nblk(n), kThreads, 0, c->stream>>>(n, c->perm, x, xi);
    a0_solve<double>(c, xi, yo, nullptr);
    k_permute_out<double><<<nblk(n), kThreads, 0, c->stream>>>(n, c->perm, yo, y);
    c->launches += 2;
    return DDLR_OK;
  });
  c->timing = timing;
  return st;
}

ddlr_status ddlr_pcg(ddlr_handle c, const double *b, double *x, int nrhs, int ld, double tol,
                     int maxit, ddlr_solve_info *info) {
  if (!c) return DDLR_ERR_INVALID;
  if (maxit <= 0) maxit = 500;
  if (!(tol > 0)) { c->err = "tol must be positive"; return DDLR_ERR_INVALID; }
  std::vector<ddlr_solve_info> inf(nrhs > 0 ? nrhs : 1);
  if (nrhs > 1 && batch_width(c) >= 2) {
    const int n = c->P.n;
    if (!b || !x || ld < n) { c->err = "invalid vector arguments"; return DDLR_ERR_INVALID; }
    ddlr_status st = run_guarded(c, [&]() -> ddlr_status {
      const bool hb = !is_device_ptr(b), hx = !is_device_ptr(x);
      const int W = batch_width(c);
      for (int j0 = 0; j0 < nrhs; j0 += W) {
        const int R = std::min(W, nrhs - j0);
        batch_alloc(c, R);
        batch_load(c, b + size_t(j0) * ld, ld, R, hb, c->bt.B);
        pcg_mr_dev(c, R, tol, maxit, inf.data() + j0);
        batch_store(c, c->bt.X, x + size_t(j0) * ld, ld, R, hx);
      }
      return DDLR_OK;
    });
    if (st != DDLR_OK) return st;
    ddlr_status agg = DDLR_OK;
    for (int r = 0; r < nrhs; r++) {
      if (info) info[r] = inf[r];
      if (inf[r].status != DDLR_OK && agg == DDLR_OK) agg = (ddlr_status)inf[r].status;
    }
    if (agg != DDLR_OK) c->err = agg == DDLR_ERR_NOCONV ? "PCG did not converge" : "NaN/Inf in PCG";
    return agg;
  }
  int j = 0;
  ddlr_status st = vec_call(c, b, x, nrhs, ld, [&](const double *bd, double *xd) {
    const int n = c->P.n;
    // b in device order -> pv[0]; solution in device order -> w64[5]
    KL(c, "perm", c->stream, k_permute_in<double>, nblk(n), kThreads, 0, n, c->perm, bd, c->pv[0]);
    pcg_dev(c, c->pv[0], c->w64[5], tol, maxit, &inf[j]);
    KL(c, "perm", c->stream, k_permute_out<double>, nblk(n), kThreads, 0, n, c->perm, c->w64[5], xd);
    j++;
  });
  if (st != DDLR_OK) return st;
  ddlr_status agg = DDLR_OK;
  for (int r = 0; r < nrhs; r++) {
    if (info) info[r] = inf[r];
    if (inf[r].status != DDLR_OK && agg == DDLR_OK) agg = (ddlr_status)inf[r].status;
  }
  if (agg != DDLR_OK) c->err = agg == DDLR_ERR_NOCONV ? "PCG did not converge" : "NaN/Inf in PCG";
  return agg;
}

ddlr_status ddlr_gmres(ddlr_handle c, const double *b, double *x, double tol, int maxit, int restart,
                       ddlr_solve_info *info) {
  if (!c) return DDLR_ERR_INVALID;
  if (maxit <= 0) maxit = 500;
  if (restart <= 0) restart = 40;
  if (!(tol > 0) || restart > kGmresMaxRestart) { c->err = "tol must be positive, restart <= 512"; return DDLR_ERR_INVALID; }
  ddlr_solve_info inf{};
  ddlr_status st = vec_call(c, b, x, 1, c->P.n, [&](const double *bd, double *xd) {
    const int n = c->P.n;
    KL(c, "perm", c->stream, k_permute_in<double>, nblk(n), kThreads, 0, n, c->perm, bd, c->pv[0]);
    gmres_dev(c, c->pv[0], c->pv[2], tol, maxit, restart, &inf);
    KL(c, "perm", c->stream, k_permute_out<double>, nblk(n), kThreads, 0, n, c->perm, c->pv[2], xd);
  });
  if (st != DDLR_OK) return st;
  if (info) *info = inf;
  if (inf.status != DDLR_OK) c->err = inf.status == DDLR_ERR_NOCONV ? "GMRES did not converge" : "NaN/Inf in GMRES";
  return (ddlr_status)inf.status;
}

ddlr_status ddlr_get_info(ddlr_handle c, ddlr_info *info) {
  if (!c || !info) return DDLR_ERR_INVALID;
  const Plan &P = c->P;
  std::memset(info, 0, sizeof(*info));
  info->n = P.n; info->p = P.p; info->s = P.s; info->m = P.m; info->k = c->opt.rank_k;
  info->variant = c->opt.variant; info->precision = c->opt.precision;
  info->lanczos_steps = c->msteps; info->ncolors = P.ncolors;
  info->levels_interior = P.levels_interior; info->levels_c = P.levels_c;
  info->theta = c->theta;
  info->lambda_max = c->ritz.empty() ? 0.0 : c->ritz[0];
  info->nnz_a = P.nnz; info->nnz_factor = P.nnz_factor; info->nnz_ehat = P.nnz_ehat;
  // fill ratio (Sec. 5): factors + Ehat + low-rank data over nnz(A)
  const double lr = double(c->urows) * c->opt.rank_k + (c->opt.variant == 2 ? double(c->opt.rank_k) * c->opt.rank_k : 0);
  info->fill_ratio = (double(P.nnz_factor) + double(P.nnz_ehat) + lr) / double(P.nnz);
  info->device_bytes = c->dev_bytes;
  info->batch_block_chunks = c->bt.chunk_per;
  info->batch_block_elem = c->bt.bd_elem;
  info->setup_ms = c->setup_ms;
  info->plan_ms = c->plan_ms;
  info->persistent = (c->pz_pcg ? 1 : 0) | (c->pz_lz ? 2 : 0);
  info->reorth_passes = c->lz_passes;
  info->reorth_fp32 = c->lz_fp32;
  if (c->opt.c_solver == 1) {
    double lohi[2] = {0, 0};
    if (cudaMemcpy(lohi, c->ctab64, sizeof(lohi), cudaMemcpyDeviceToHost) != cudaSuccess) return DDLR_ERR_CUDA;
    info->cheb_lo = lohi[0];
    info->cheb_hi = lohi[1];
    info->cheb_lanczos_steps = c->cheb_msteps;
  }
  return DDLR_OK;
}

ddlr_status ddlr_get_ritz(ddlr_handle c, double *out, int cap, int *count) {
  if (!c) return DDLR_ERR_INVALID;
  if (count) *count = int(c->ritz.size());
  if (out)
    for (int i = 0; i < cap && i < int(c->ritz.size()); i++) out[i] = c->ritz[i];
  return DDLR_OK;
}

ddlr_status ddlr_get_factor_coo(ddlr_handle c, long long *nnz, int *rows, int *cols, double *vals) {
  if (!c || !nnz) return DDLR_ERR_INVALID;
  *nnz = c->P.nnz_factor;
  if (!rows) return DDLR_OK;
  return run_guarded(c, [&]() -> ddlr_status {
    std::vector<double> h(c->P.nnz_factor);
    read_dev(c, h.data(), c->fval, sizeof(double) * h.size());
    for (long long q = 0; q < c->P.nnz_factor; q++) {
      rows[q] = c->P.perm[c->P.f_row[q]];
      cols[q] = c->P.perm[c->P.f_ci[q]];
      if (vals) vals[q] = h[q];
    }
    return DDLR_OK;
  });
}

// rows of U in ascending original index: order[r] = device row of rank r
static std::vector<int> lowrank_order(ddlr_ctx *c) {
  const Plan &P = c->P;
  const int off = c->opt.variant == 1 ? P.m : 0;
  std::vector<std::pair<int, int>> o(c->urows);
  for (int r = 0; r < c->urows; r++) o[r] = {P.perm[off + r], r};
  std::sort(o.begin(), o.end());
  std::vector<int> ord(c->urows);
  for (int r = 0; r < c->urows; r++) ord[r] = o[r].second;
  return ord;
}

ddlr_status ddlr_get_lowrank(ddlr_handle c, double *U, double *lam, double *theta, double *Hk) {
  if (!c) return DDLR_ERR_INVALID;
  return run_guarded(c, [&]() -> ddlr_status {
    const int k = c->opt.rank_k;
    if (U) {
      std::vector<double> h(size_t(c->urows) * k);
      read_dev(c, h.data(), c->U64, sizeof(double) * h.size());
      std::vector<int> ord = lowrank_order(c);
      for (int r = 0; r < c->urows; r++)
        std::memcpy(U + size_t(r) * k, h.data() + size_t(ord[r]) * k, sizeof(double) * k);
    }
    if (lam) for (int i = 0; i < k; i++) lam[i] = i < int(c->ritz.size()) ? c->ritz[i] : 0.0;
    if (theta) *theta = c->theta;
    if (Hk) read_dev(c, Hk, c->Hk64, sizeof(double) * k * k);
    return DDLR_OK;
  });
}

ddlr_status ddlr_set_cheb_bounds(ddlr_handle c, double lo, double hi) {
  if (!c) return DDLR_ERR_INVALID;
  if (c->opt.c_solver != 1 || !(lo > 0.0) || !(hi >= lo) || !std::isfinite(hi)) {
    c->err = "ddlr_set_cheb_bounds: needs c_solver 1 and 0 < lo <= hi";
    return DDLR_ERR_INVALID;
  }
  return run_guarded(c, [&]() -> ddlr_status {
    KL(c, "setup", c->stream, k_cheb_coef, 1, 32, 0, lo, hi, c->opt.cheb_steps, c->ctab64, c->ctab32);
    sync(c);
    return DDLR_OK;
  });
}

ddlr_status ddlr_set_lowrank(ddlr_handle c, const double *U, const double *lam, double theta,
                             const double *Hk) {
  if (!c || !U) return DDLR_ERR_INVALID;
  if (c->opt.variant == 1 && !lam) return DDLR_ERR_INVALID;
  if (c->opt.variant == 2 && !Hk) return DDLR_ERR_INVALID;
  return run_guarded(c, [&]() -> ddlr_status {
    const int k = c->opt.rank_k;
    std::vector<int> ord = lowrank_order(c);
    std::vector<double> h(size_t(c->urows) * k);
    for (int r = 0; r < c->urows; r++)
      std::memcpy(h.data() + size_t(ord[r]) * k, U + size_t(r) * k, sizeof(double) * k);
    ck(cudaMemcpyAsync(c->U64, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c->stream), "H2D");
    if (c->opt.variant == 1) {
      std::vector<double> v(lam, lam + k);
      v.push_back(theta);
      double *dv = c->w64[7];
      ck(cudaMemcpyAsync(dv, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, c->stream), "H2D");
      ck(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), c->stream), "memset");
      KL(c, "setup", c->stream, k_ddlr1_coef, 1, 32, 0, k + 1, k, 1, dv, c->theta_d, c->inv1mt64,
         c->coef64, c->dflag + 1);
      c->theta = theta;
      for (int i = 0; i < k && i < int(c->ritz.size()); i++) c->ritz[i] = lam[i];
    } else {
      ck(cudaMemcpyAsync(c->Hk64, Hk, sizeof(double) * k * k, cudaMemcpyHostToDevice, c->stream), "H2D");
    }
    lowrank_to_low_precision(c);
    sync(c);
    return DDLR_OK;
  });
}

ddlr_status ddlr_set_timing(ddlr_handle c, int enable) {
  if (!c) return DDLR_ERR_INVALID;
  c->timing = enable != 0;
  return DDLR_OK;
}

ddlr_status ddlr_get_counters(ddlr_handle c, long long *launches, char *names, int cap, double *ms,
                              long long *family_launches, int cap_f, int *nfamilies) {
  if (!c) return DDLR_ERR_INVALID;
  return run_guarded(c, [&]() -> ddlr_status {
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->stream2);
    c->resolve();
    if (launches) *launches = c->launches;
    if (nfamilies) *nfamilies = int(c->fam_names.size());
    if (names && cap > 0) {
      std::string all;
      for (size_t i = 0; i < c->fam_names.size(); i++) { if (i) all += ","; all += c->fam_names[i]; }
      std::strncpy(names, all.c_str(), size_t(cap) - 1);
      names[cap - 1] = 0;
    }
    for (int i = 0; i < cap_f && i < int(c->fam_names.size()); i++) {
      if (ms) ms[i] = c->fam_ms[i];
      if (family_launches) family_launches[i] = c->fam_cnt[i];
    }
    return DDLR_OK;
  });
}

ddlr_status ddlr_reset_counters(ddlr_handle c) {
  if (!c) return DDLR_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  cudaStreamSynchronize(c->stream2);
  c->resolve();
  c->launches = 0;
  for (auto &v : c->fam_ms) v = 0;
  for (auto &v : c->fam_cnt) v = 0;
  c->pz_pcg_bytes = c->pz_lz_bytes = 0;
  c->pz_pcg_runs = c->pz_lz_runs = 0;
  return DDLR_OK;
}

// algorithmic bytes of one batched A0 solve of R columns (level launches of
// k_sptrsv_*_mr): the off-diagonal factor entries and the inverse diagonal once
// per sweep, every column read and written once per sweep (gathered reads of
// other rows as cache hits)
static double batch_a0_bytes(const ddlr_ctx *c, double R) {
  const Plan &P = c->P;
  const double v = c->opt.precision == 1 ? 4.0 : 8.0;
  const double off = double(P.nnz_factor) - double(P.n);
  return 2.0 * (off * (v + 4.0) + double(P.n) * v + 2.0 * double(P.n) * R * v);
}
static double batch_a0_launches(const ddlr_ctx *c) {
  const int nL = int(c->P.ch_all_ptr.size()) - 1;
  return nL == 2 ? 2.0 : double(std::max(1, 2 * nL - 1));
}

ddlr_status ddlr_get_traffic(ddlr_handle c, double *apply_bytes, double *a0_bytes,
                             double *family_bytes, int cap_f) {
  if (!c) return DDLR_ERR_INVALID;
  const Plan &P = c->P;
  const double v = c->opt.precision == 1 ? 4.0 : 8.0;
  const double ub = c->opt.precision == 1 ? (c->opt.uk_bf16 ? 2.0 : 4.0) : 8.0;
  const double n = P.n, s = P.s, m = P.m, k = c->opt.rank_k;
  // off-diagonal factor entries of the interior blocks and of C_a
  double off_c = 0.0;
  for (int g = P.blk_row0[P.p]; g < P.n; g++) off_c += P.f_rp[g + 1] - P.f_rp[g] - 1;
  const double off_int = double(P.nnz_factor) - n - off_c;
  const double ne = double(P.nnz_ehat);
  // one forward + one backward sweep: off-diagonal values and indices once per
  // sweep, the inverse diagonal, the right-hand side read and the result written
  const double blocks = 2.0 * (off_int * (v + 4.0) + 3.0 * m * v);
  const double cblk = 2.0 * (off_c * (v + 4.0) + 3.0 * s * v);
  // Chebyshev C_a solve (block p factors D_a): t - 1 more D_a solves, and the
  // step kernels stream C_a (values, indices, row pointers) and the x, s, r
  // vectors (ddlr_cheb.cuh)
  double cheb_k = 0.0;
  const int t = c->opt.cheb_steps;
  if (c->opt.c_solver == 1) {
    const double ccb = double(P.cc_ci.size()) * (v + 4.0) + 4.0 * s;
    cheb_k = t == 1 ? 2.0 * s * v : (ccb + 5.0 * s * v) + (t - 2) * (ccb + 7.0 * s * v) + 4.0 * s * v;
  }
  // approximate inverse (c_solver 2): the C_a block's rows are diagonal in
  // the sweeps, then one row-wise product with the symmetric part of X
  const double mr_k = c->opt.c_solver == 2 ? double(c->mr.nnz) * (v + 4.0) + 8.0 * s + 2.0 * s * v : 0.0;
  const double a0 = blocks + cblk + (c->opt.c_solver == 1 ? (t - 1) * cblk + cheb_k : 0.0) + mr_k;
  const double et = ne * (v + 4.0) + 4.0 * s + 2.0 * s * v;
  const double urows = c->urows;
  const double utx = urows * k * ub + urows * v;
  const double wr = s * k * ub + 4.0 * s * v;
  const double ei = ne * (v + 4.0) + 4.0 * m + 2.0 * m * v;
  const double uadd = n * k * ub + 2.0 * n * v;
  const double apply = c->opt.variant == 1 ? 2.0 * a0 + et + utx + wr + ei : a0 + utx + uadd;
  if (apply_bytes) *apply_bytes = apply;
  if (a0_bytes) *a0_bytes = a0;
  if (family_bytes) {
    // launches per A0 sweep pair: two for two-level factors (modes 3 and 4),
    // else forward, top and backward levels
    auto sweeps = [](int L) { return L == 2 ? 2 : std::max(1, 2 * L - 1); };
    const double clev = sweeps(P.levels_c);
    const double nnz_a = double(P.nnz);
    const double R = std::max(1, c->bt.last_R);
    for (int i = 0; i < cap_f && i < int(c->fam_names.size()); i++) {
      const std::string &f = c->fam_names[i];
      double b = 0.0;
      if (f == "sptrsv_blocks") b = blocks;
      else if (f == "sptrsv_levels") b = (blocks + cblk) / sweeps(std::max(P.levels_interior, P.levels_c));
      else if (f == "sptrsv_c" || f == "cheb_dsolve") b = cblk / clev;
      else if (f == "cheb") b = cheb_k / t;
      else if (f == "mr_apply") b = mr_k;
      else if (f == "et") b = et;
      else if (f == "utx") b = utx;
      else if (f == "w_rhs") b = wr;
      else if (f == "e_int") b = ei;
      else if (f == "u_add") b = uadd;
      else if (f == "spmv") b = nnz_a * 12.0 + 2.0 * n * 8.0;
      else if (f == "pcg_dot") b = 2.0 * n * 8.0;
      else if (f == "pcg_axpy") b = 6.0 * n * 8.0;
      else if (f == "pcg_dot2") b = 3.0 * n * 8.0;
      else if (f == "pcg_p") b = (c->opt.precision == 1 ? 4.0 : 3.0) * n * 8.0;
      else if (f == "pcg_persist") b = c->pz_pcg_runs ? c->pz_pcg_bytes / double(c->pz_pcg_runs) : 0.0;
      // batched (R right-hand sides, R = the width of the last batched call):
      // operator data once per launch, R columns of every vector
      else if (f == "sptrsv_levels_mr") b = batch_a0_bytes(c, R) / batch_a0_launches(c);
      else if (f == "et_mr") b = ne * (v + 4.0) + 4.0 * s + 2.0 * s * R * v;
      else if (f == "utx_mr") b = urows * k * ub + urows * R * v;
      else if (f == "reduce_mr")
        b = double(c->opt.precision == 1 && c->bt.tc ? kTcRedGrid : kRedGrid) * k * R * v + k * R * v;
      else if (f == "w_rhs_mr") b = s * k * ub + 4.0 * s * R * v;
      else if (f == "e_int_mr") b = ne * (v + 4.0) + 4.0 * m + 2.0 * m * R * v;
      else if (f == "u_add_mr") b = n * k * ub + 2.0 * n * R * v;
      else if (f == "spmv_mr") b = nnz_a * 12.0 + 2.0 * n * R * 8.0;
      else if (f == "pcg_mr_dot") b = 2.0 * n * R * 8.0;
      else if (f == "pcg_mr_red") b = (std::ceil(n / kFbRows) + kRedGrid) * R * 8.0;
      else if (f == "pcg_mr_axpy") b = 6.0 * n * R * 8.0;
      else if (f == "pcg_mr_p") b = (c->opt.precision == 1 ? 4.0 : 3.0) * n * R * 8.0;
      else if (f == "vec_mr") b = n * R * (8.0 + v) + (c->dsc_dev ? 8.0 * n : 0.0);
      else if (f == "lanczos_persist") b = c->pz_lz_runs ? c->pz_lz_bytes / double(c->pz_lz_runs) : 0.0;
      family_bytes[i] = b;
    }
  }
  return DDLR_OK;
}

ddlr_status ddlr_set_stream(ddlr_handle c, void *s) {
  if (!c) return DDLR_ERR_INVALID;
  c->stream = (cudaStream_t)s;
  return DDLR_OK;
}

ddlr_status ddlr_set_wait_limit(ddlr_handle c, double seconds) {
  if (!c) return DDLR_ERR_INVALID;
  if (!(seconds > 0) || seconds > 3600) { c->err = "wait limit must be in (0, 3600] seconds"; return DDLR_ERR_INVALID; }
  return run_guarded(c, [&]() -> ddlr_status {
    ck(cudaStreamSynchronize(c->stream), "sync");
    c->wait_ns = (unsigned long long)(seconds * 1e9);
    c->opt.wait_limit_s = seconds;
    // captured graphs hold the old limit in their kernel arguments
    if (c->lw.exec) { cudaGraphExecDestroy(c->lw.exec); c->lw.exec = nullptr; }
    if (c->pcg_exec) { cudaGraphExecDestroy(c->pcg_exec); c->pcg_exec = nullptr; }
    c->gm.free_graphs();
    for (auto &kv : c->bt.graphs)
      if (kv.second.exec) { cudaGraphExecDestroy(kv.second.exec); kv.second.exec = nullptr; }
    c->bt.graphs.clear();
    return DDLR_OK;
  });
}

ddlr_status ddlr_selftest_conversions(const double *in, long long n, int dir, long long *mismatches) {
  if (!in || !mismatches || n < 0 || (dir != 0 && dir != 1)) return DDLR_ERR_INVALID;
  *mismatches = 0;
  if (n == 0) return DDLR_OK;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, in) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return DDLR_ERR_INVALID;
  }
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * size_t(n)) != cudaSuccess) return DDLR_ERR_CUDA;
  k_cvt_check<<<unsigned((n + 255) / 256), 256>>>(n, in, out, dir);
  std::vector<double> h(static_cast<size_t>(n));
  cudaError_t e = cudaMemcpy(h.data(), out, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost);
  cudaFree(out);
  if (e != cudaSuccess) return DDLR_ERR_CUDA;
  long long bad = 0;
  for (double v : h) bad += v != 0.0;
  *mismatches = bad;
  return DDLR_OK;
}

const char *ddlr_last_error(ddlr_handle c) {
  if (!c) return g_setup_error.c_str();
  return c->err.c_str();
}

ddlr_status ddlr_destroy(ddlr_handle c) {
  if (!c) return DDLR_OK;
  slots_forget(c);
  if (c->stream2) cudaStreamSynchronize(c->stream2);
  cudaStreamSynchronize(c->stream);
  c->resolve();
  for (auto e : c->evpool) cudaEventDestroy(e);
  batch_free(c);
  c->release();
  if (c->h_pin) cudaFreeHost(c->h_pin);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
  c->gm.free_graphs();
  if (c->lw.exec) cudaGraphExecDestroy(c->lw.exec);
  if (c->lw.ev_chk) cudaEventDestroy(c->lw.ev_chk);
  if (c->lw.ev_done) cudaEventDestroy(c->lw.ev_done);
  if (c->lw.h_st) cudaFreeHost(c->lw.h_st);
  if (c->gstream) { cudaStreamSynchronize(c->gstream); cudaStreamDestroy(c->gstream); }
  if (c->stream2) cudaStreamDestroy(c->stream2);
  delete c;
  return DDLR_OK;
}

}  // extern "C"
