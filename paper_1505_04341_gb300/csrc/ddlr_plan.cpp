// ddlr_plan.cpp -- host-side symbolic analysis (pattern and partition only).
//
//  * Sec. 2.1: a node is an interface node when it couples to a node of
//    another subdomain, else an interior node.
//  * eq. (Bmat): interiors of subdomains 0..p-1 first, then all interface
//    nodes; within each group ascending original index.
//  * eq. (split) / Proposition (locality of Ehat Ehat^T): block b < p of A0 is
//    B_{b,a} = B_b + a^-2 E_b E_b^T, block p is C_a = C + a^2 I.
//  * Local solvers (Sec. 5): incomplete Cholesky with zero fill on the block
//    pattern, or exact Cholesky on the symbolic fill pattern.  The elimination
//    order is ascending original index (b_order 0) or multicolour (b_order
//    1: the two colour classes of a bipartite block graph, else greedy
//    colouring) for interior blocks, and likewise (c_order) for C_a.
//  * Device order: inside every block the rows are sorted by (dependency
//    level, elimination position).  This is a topological order of the
//    factor's dependency graph, so it leaves the factor unchanged and lets
//    every level be solved in parallel.
//
// The analysis runs on all host cores: rows, slices and blocks are
// independent, and every flat CSR output is built in two passes (count per
// row, prefix sum, fill), so the plan does not depend on the thread count.
#include "ddlr_plan.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <numeric>
#include <thread>

namespace ddlr {

namespace {

// position of column c in row r of the original CSR, -1 if absent
inline int find_pos(const int *rp, const int *ci, int r, int c) {
  const int *b = ci + rp[r], *e = ci + rp[r + 1];
  const int *it = std::lower_bound(b, e, c);
  return (it != e && *it == c) ? int(it - ci) : -1;
}

// A fixed set of worker threads for the lifetime of one analysis.  run(n, f)
// calls f(lo, hi) on disjoint ranges covering [0, n) (static split, one per
// worker) and returns when all are done; run_dynamic(n, f) hands out single
// indices in order to whichever worker is free.
class Pool {
 public:
  explicit Pool(int nt) : nt_(std::max(1, nt)) {
    for (int t = 1; t < nt_; t++) th_.emplace_back([this, t] { loop(t); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
      gen_++;
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }
  int size() const { return nt_; }
  void run(long long n, const std::function<void(long long, long long)> &f, long long min_chunk = 2048) {
    if (n <= 0) return;
    const int parts = int(std::min<long long>(nt_, std::max<long long>(1, n / min_chunk)));
    if (parts <= 1) { f(0, n); return; }
    job_ = [&f, n, parts](int t) {
      if (t >= parts) return;
      f(n * t / parts, n * (t + 1) / parts);
    };
    dispatch();
  }
  void run_dynamic(int n, const std::function<void(int)> &f) {
    if (n <= 0) return;
    std::atomic<int> next(0);
    job_ = [&f, &next, n](int) {
      for (int i = next++; i < n; i = next++) f(i);
    };
    dispatch();
  }

 private:
  void dispatch() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      pending_ = nt_ - 1;
      gen_++;
    }
    cv_.notify_all();
    job_(0);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [this] { return pending_ == 0; });
  }
  void loop(int t) {
    unsigned long long seen = 0;
    while (true) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
      }
      job_(t);
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_cv_.notify_one();
    }
  }
  int nt_;
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::function<void(int)> job_;
  unsigned long long gen_ = 0;
  int pending_ = 0;
  bool stop_ = false;
};

int plan_threads(long long work) {
  const int hw = int(std::thread::hardware_concurrency());
  const int by_size = int(std::min<long long>(64, std::max<long long>(1, work / 20000)));
  return std::max(1, std::min({hw > 0 ? hw : 1, 32, by_size}));
}

// exclusive prefix sum of counts[0..n) into offsets[0..n]
template <typename C, typename D>
void prefix(const C &counts, D &offsets) {
  offsets.assign(counts.size() + 1, 0);
  for (size_t i = 0; i < counts.size(); i++) offsets[i + 1] = offsets[i] + counts[i];
}

}  // namespace

ddlr_status build_plan(int n, const int *rp, const int *ci, const double *val,
                       const int *part, int p, const ddlr_options &opt, Plan &P,
                       std::string &err) {
  if (n <= 0 || p <= 0 || !rp || !ci || !val || !part) {
    err = "invalid sizes or NULL array";
    return DDLR_ERR_INVALID;
  }
  if (rp[0] != 0) { err = "rowptr[0] != 0"; return DDLR_ERR_INVALID; }
  for (int i = 0; i < n; i++)
    if (rp[i + 1] < rp[i]) { err = "rowptr not monotone"; return DDLR_ERR_INVALID; }
  const long long nnz = rp[n];
  Pool pool(plan_threads(nnz));

  // ---- input checks: the first offending row (in row order) names the error
  {
    std::vector<int> bad_row(pool.size(), n);
    std::vector<const char *> bad_msg(pool.size(), nullptr);
    std::atomic<int> slot(0);
    pool.run(n, [&](long long lo, long long hi) {
      const int me = slot++;
      for (int i = int(lo); i < int(hi); i++) {
        const char *msg = nullptr;
        if (part[i] < 0 || part[i] >= p) msg = "part out of range";
        bool diag = false;
        for (int q = rp[i]; q < rp[i + 1] && !msg; q++) {
          if (ci[q] < 0 || ci[q] >= n) { msg = "column index out of range"; break; }
          if (q > rp[i] && ci[q] <= ci[q - 1]) { msg = "columns not strictly ascending"; break; }
          if (ci[q] == i) diag = true;
        }
        if (!msg && !diag) msg = "missing diagonal entry";
        if (msg) { bad_row[me] = i; bad_msg[me] = msg; return; }
      }
    });
    int first = n;
    const char *msg = nullptr;
    for (int t = 0; t < pool.size(); t++)
      if (bad_msg[t] && bad_row[t] < first) { first = bad_row[t]; msg = bad_msg[t]; }
    if (msg) { err = msg; return DDLR_ERR_INVALID; }
    std::atomic<int> asym(0);
    pool.run(n, [&](long long lo, long long hi) {
      for (int i = int(lo); i < int(hi) && !asym.load(std::memory_order_relaxed); i++)
        for (int q = rp[i]; q < rp[i + 1]; q++) {
          const int t = find_pos(rp, ci, ci[q], i);
          if (t < 0 || val[t] != val[q]) { asym = 1; return; }
        }
    });
    if (asym) { err = "matrix is not symmetric"; return DDLR_ERR_INVALID; }
  }
  P = Plan();
  P.n = n; P.p = p; P.nnz = nnz;
  P.orig_row.resize(nnz); P.orig_col.resize(nnz); P.diag_pos.resize(n);
  pool.run(n, [&](long long lo, long long hi) {
    for (int i = int(lo); i < int(hi); i++)
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        P.orig_row[q] = i; P.orig_col[q] = ci[q];
        if (ci[q] == i) P.diag_pos[i] = q;
      }
  });

  // ---- Sec. 2.1 classification and eq. (Bmat) order
  std::vector<char> iface(n, 0);
  pool.run(n, [&](long long lo, long long hi) {
    for (int i = int(lo); i < int(hi); i++)
      for (int q = rp[i]; q < rp[i + 1]; q++)
        if (part[ci[q]] != part[i]) { iface[i] = 1; break; }
  });
  // members of every block in ascending index: a counting sort over fixed
  // row ranges (per-range counts, offsets, parallel fill)
  std::vector<std::vector<int>> members(p + 1);
  {
    const int nr = pool.size();
    std::vector<int> rcnt(size_t(nr) * (p + 1), 0);
    pool.run_dynamic(nr, [&](int t) {
      int *c = rcnt.data() + size_t(t) * (p + 1);
      for (long long i = n * (long long)t / nr; i < n * (long long)(t + 1) / nr; i++) c[iface[i] ? p : part[i]]++;
    });
    for (int b = 0; b <= p; b++) {
      int tot = 0;
      for (int t = 0; t < nr; t++) { const int c = rcnt[size_t(t) * (p + 1) + b]; rcnt[size_t(t) * (p + 1) + b] = tot; tot += c; }
      members[b].resize(tot);
    }
    pool.run_dynamic(nr, [&](int t) {
      int *c = rcnt.data() + size_t(t) * (p + 1);
      for (long long i = n * (long long)t / nr; i < n * (long long)(t + 1) / nr; i++) {
        const int b = iface[i] ? p : part[i];
        members[b][c[b]++] = int(i);
      }
    });
  }
  int s = int(members[p].size());
  if (s == 0) { err = "no interface nodes (p = 1?)"; return DDLR_ERR_INVALID; }
  if (opt.rank_k < 1 || opt.rank_k > s) { err = "rank_k must be in [1, s]"; return DDLR_ERR_INVALID; }
  P.s = s; P.m = n - s;
  std::vector<int> blk_of(n);
  std::vector<int> loc(n, -1);   // index of a node inside its own block
  for (int b = 0; b <= p; b++)
    for (int t = 0; t < int(members[b].size()); t++) { blk_of[members[b][t]] = b; loc[members[b][t]] = t; }

  const bool exact = opt.factor == 1 || opt.factor == 3;   // symbolic fill pattern
  P.perm.resize(n); P.iperm.resize(n);
  P.blk_row0.assign(p + 2, 0);
  for (int b = 0; b <= p; b++) P.blk_row0[b + 1] = P.blk_row0[b] + int(members[b].size());
  // per node: level in its block's factor; lower factor pattern per device
  // row as device-order columns (per block, joined afterwards)
  std::vector<int> level_of(n, 0);
  std::vector<int> low_cnt(n, 0);
  std::vector<std::vector<int>> low_blk(p + 1);
  std::vector<int> blk_levels(p + 1, 0), blk_colors(p + 1, 0);
  std::vector<const char *> blk_err(p + 1, nullptr);
  // blocks in decreasing size, so the largest (usually C_a) starts first
  std::vector<int> border(p + 1);
  std::iota(border.begin(), border.end(), 0);
  std::stable_sort(border.begin(), border.end(),
                   [&](int a, int b) { return members[a].size() > members[b].size(); });
  pool.run_dynamic(p + 1, [&](int bi) {
    const int b = border[bi];
    const std::vector<int> &mem = members[b];
    const int nb = int(mem.size());
    const int row_w = P.blk_row0[b];
    std::vector<int> arp(nb + 1, 0), aci, ord(nb), epos(nb), lrp, lci, lev, dev, col, used, cnt;
    // block graph (local indices, flat CSR): A restricted to the block, plus,
    // for interior blocks, the pattern of Ehat Ehat^T
    for (int t = 0; t < nb; t++) {
      const int i = mem[t];
      const size_t a0 = aci.size();
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        const int j = ci[q];
        // Chebyshev mode (Sec. 4.3): block p is the block Jacobi matrix D_a,
        // the couplings of C_a between interface nodes of one subdomain; with
        // the approximate inverse (c_solver 2) block p is left diagonal (the
        // A0 sweeps' C_a rows are then replaced by the product with X)
        if (j != i && blk_of[j] == b &&
            (b < p || opt.c_solver == 0 || (opt.c_solver == 1 && part[j] == part[i])))
          aci.push_back(loc[j]);
        if (b < p && iface[j]) {
          for (int q2 = rp[j]; q2 < rp[j + 1]; q2++) {
            const int r = ci[q2];
            if (r != i && !iface[r]) {
              if (blk_of[r] != b) { blk_err[b] = "Ehat Ehat^T couples two subdomains"; return; }
              aci.push_back(loc[r]);
            }
          }
        }
      }
      std::sort(aci.begin() + a0, aci.end());
      aci.erase(std::unique(aci.begin() + a0, aci.end()), aci.end());
      arp[t + 1] = int(aci.size());
    }
    // elimination order
    std::iota(ord.begin(), ord.end(), 0);
    if ((b == p && opt.c_order == 1) || (b < p && opt.b_order == 1)) {
      // a bipartite block graph takes its two-colouring: breadth-first from
      // the lowest unvisited node of each component, which gets colour 0
      // (unique, and the same colouring the greedy rule finds whenever that
      // one needs only two colours); otherwise greedy: ascending index, the
      // smallest colour no lower-indexed neighbour has
      col.assign(nb, -1);
      int nc = 0;
      bool bip = true;
      {
        std::vector<int> queue(nb);
        for (int t0 = 0; t0 < nb && bip; t0++) {
          if (col[t0] >= 0) continue;
          col[t0] = 0;
          int head = 0, tail = 0;
          queue[tail++] = t0;
          while (head < tail && bip) {
            const int u = queue[head++];
            for (int q = arp[u]; q < arp[u + 1]; q++) {
              const int v = aci[q];
              if (col[v] < 0) { col[v] = 1 - col[u]; queue[tail++] = v; }
              else if (col[v] == col[u]) { bip = false; break; }
            }
          }
        }
        if (bip) for (int t = 0; t < nb; t++) nc = std::max(nc, col[t] + 1);
      }
      if (!bip) {
        col.assign(nb, -1);
        used.assign(nb + 2, -1);
        nc = 0;
        for (int t = 0; t < nb; t++) {
          for (int q = arp[t]; q < arp[t + 1]; q++) if (aci[q] < t) used[col[aci[q]]] = t;
          int c = 0;
          while (used[c] == t) c++;
          col[t] = c;
          nc = std::max(nc, c + 1);
        }
      }
      blk_colors[b] = nc;
      // stable counting sort by colour
      cnt.assign(nc + 1, 0);
      for (int t = 0; t < nb; t++) cnt[col[t] + 1]++;
      for (int c = 0; c < nc; c++) cnt[c + 1] += cnt[c];
      for (int t = 0; t < nb; t++) ord[cnt[col[t]]++] = t;
    }
    for (int e = 0; e < nb; e++) epos[ord[e]] = e;
    // lower pattern in elimination positions (flat CSR lrp/lci)
    lrp.assign(nb + 1, 0);
    for (int e = 0; e < nb; e++) {
      const int t = ord[e];
      const size_t l0 = lci.size();
      for (int q = arp[t]; q < arp[t + 1]; q++) if (epos[aci[q]] < e) lci.push_back(epos[aci[q]]);
      std::sort(lci.begin() + l0, lci.end());
      lrp[e + 1] = int(lci.size());
    }
    if (!exact && opt.fill_level > 0) {
      // level-of-fill pattern: the block's entries have level 0, and
      // eliminating pivot t gives entry (i, j) of two later neighbours of t
      // the level lev(i,t) + lev(j,t) + 1; entries of level <= fill_level
      // are kept (only kept entries produce fill).  Column lists of
      // (row, level), complete when their pivot is reached.
      const int kf = opt.fill_level;
      std::vector<std::vector<std::pair<int, int>>> colv(nb);
      for (int e = 0; e < nb; e++)
        for (int q = lrp[e]; q < lrp[e + 1]; q++) colv[lci[q]].push_back({e, 0});
      long long total = 0;
      for (int t = 0; t < nb; t++) {
        std::vector<std::pair<int, int>> &c = colv[t];
        std::sort(c.begin(), c.end());
        size_t w = 0;   // one entry per row, its smallest level
        for (size_t a = 0; a < c.size(); a++) {
          if (w > 0 && c[w - 1].first == c[a].first) continue;
          c[w++] = c[a];
        }
        c.resize(w);
        total += (long long)w;
        if (total > 60000000LL) { blk_err[b] = "fill pattern too large"; return; }
        for (size_t x = 1; x < c.size(); x++)
          for (size_t y = 0; y < x; y++) {
            const int lv = c[x].second + c[y].second + 1;
            if (lv <= kf) colv[c[y].first].push_back({c[x].first, lv});
          }
      }
      std::vector<int> rc(nb + 1, 0);
      for (int j = 0; j < nb; j++) for (const auto &pr : colv[j]) rc[pr.first + 1]++;
      for (int e = 0; e < nb; e++) rc[e + 1] += rc[e];
      lrp = rc;
      lci.assign(rc[nb], 0);
      for (int j = 0; j < nb; j++) for (const auto &pr : colv[j]) lci[rc[pr.first]++] = j;   // ascending j per row
    }
    if (exact) {
      // symbolic Cholesky: struct(L_{*j}) = struct(A_{*j}) U struct of the
      // children of j in the elimination tree, minus j
      std::vector<std::vector<int>> cols(nb);
      for (int e = 0; e < nb; e++) for (int q = lrp[e]; q < lrp[e + 1]; q++) cols[lci[q]].push_back(e);
      long long total = 0;
      for (int j = 0; j < nb; j++) {
        std::vector<int> &c = cols[j];
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        total += (long long)c.size();
        if (total > 60000000LL) { blk_err[b] = "exact factor too large"; return; }
        if (!c.empty()) {
          int par = c[0];
          for (size_t t = 1; t < c.size(); t++) cols[par].push_back(c[t]);
        }
      }
      std::vector<int> rc(nb + 1, 0);
      for (int j = 0; j < nb; j++) for (int e : cols[j]) rc[e + 1]++;
      for (int e = 0; e < nb; e++) rc[e + 1] += rc[e];
      lrp = rc;
      lci.assign(rc[nb], 0);
      for (int j = 0; j < nb; j++) for (int e : cols[j]) lci[rc[e]++] = j;   // ascending j per row
    }
    // levels
    lev.assign(nb, 0);
    int maxlev = 0;
    for (int e = 0; e < nb; e++) {
      int l = 0;
      for (int q = lrp[e]; q < lrp[e + 1]; q++) l = std::max(l, lev[lci[q]] + 1);
      lev[e] = l;
      maxlev = std::max(maxlev, l);
    }
    blk_levels[b] = nb ? maxlev + 1 : 0;
    // device order: (level, elimination position), stable counting sort
    cnt.assign(maxlev + 2, 0);
    for (int e = 0; e < nb; e++) cnt[lev[e] + 1]++;
    for (int l = 0; l <= maxlev; l++) cnt[l + 1] += cnt[l];
    dev.resize(nb);
    for (int e = 0; e < nb; e++) dev[cnt[lev[e]]++] = e;
    std::vector<int> drow(nb);   // elimination position -> device row
    for (int d = 0; d < nb; d++) drow[dev[d]] = row_w + d;
    std::vector<int> &lowb = low_blk[b];
    lowb.reserve(lci.size());
    for (int d = 0; d < nb; d++) {
      const int e = dev[d];
      const int i = mem[ord[e]];
      P.perm[row_w + d] = i;
      level_of[i] = lev[e];
      for (int q = lrp[e]; q < lrp[e + 1]; q++) lowb.push_back(drow[lci[q]]);
      low_cnt[row_w + d] = lrp[e + 1] - lrp[e];
    }
  });
  for (int b = 0; b <= p; b++)
    if (blk_err[b]) { err = blk_err[b]; return DDLR_ERR_INVALID; }
  for (int b = 0; b < p; b++) P.levels_interior = std::max(P.levels_interior, blk_levels[b]);
  P.levels_c = std::max(1, blk_levels[p]);
  if (opt.c_order == 1) P.ncolors = blk_colors[p];
  std::vector<int> low_rp;
  pvec<int> low_ci;
  prefix(low_cnt, low_rp);
  low_ci.resize(low_rp[n]);
  pool.run_dynamic(p + 1, [&](int b) {
    std::copy(low_blk[b].begin(), low_blk[b].end(), low_ci.begin() + low_rp[P.blk_row0[b]]);
  });
  std::vector<std::vector<int>>().swap(low_blk);
  pool.run(n, [&](long long lo, long long hi) {
    for (int g = int(lo); g < int(hi); g++) P.iperm[P.perm[g]] = g;
  });
  const int m = P.m;
  // the interface list is in ascending original index, so a node's place in
  // it is its rank in that order
  P.iface_rank.resize(s);
  for (int j = 0; j < s; j++) P.iface_rank[j] = loc[P.perm[m + j]];

  // ---- A in device order, sliced ELL for the SpMV
  {
    const int ns = (n + kSlice - 1) / kSlice;
    P.a_nslice = ns;
    P.a_sw.assign(ns, 0);
    pool.run(ns, [&](long long lo, long long hi) {
      for (int g = int(lo); g < int(hi); g++) {
        int w = 0;
        for (int l = 0; l < kSlice; l++) {
          const int r = g * kSlice + l;
          if (r < n) { const int i = P.perm[r]; w = std::max(w, rp[i + 1] - rp[i]); }
        }
        P.a_sw[g] = w;
      }
    }, 256);
    P.a_soff.assign(ns + 1, 0);
    for (int g = 0; g < ns; g++) P.a_soff[g + 1] = P.a_soff[g] + P.a_sw[g] * kSlice;
    P.a_col.resize(P.a_soff[ns]);   // every slot is written below
    P.a_src.resize(P.a_soff[ns]);
    pool.run(ns, [&](long long lo, long long hi) {
      std::vector<std::pair<int, int>> ent;
      for (int g = int(lo); g < int(hi); g++)
        for (int l = 0; l < kSlice; l++) {
          const int r = g * kSlice + l;
          const int rr = r < n ? r : n - 1;
          ent.clear();
          if (r < n) {
            const int i = P.perm[r];
            for (int q = rp[i]; q < rp[i + 1]; q++) ent.push_back({P.iperm[ci[q]], q});
            std::sort(ent.begin(), ent.end());
          }
          for (int kk = 0; kk < P.a_sw[g]; kk++) {
            const int slot = P.a_soff[g] + kk * kSlice + l;
            if (kk < int(ent.size())) { P.a_col[slot] = ent[kk].first; P.a_src[slot] = ent[kk].second; }
            else { P.a_col[slot] = rr; P.a_src[slot] = -1; }
          }
        }
    }, 256);
  }

  // ---- Ehat (interior rows) and Ehat^T (interface rows): count, prefix, fill
  {
    auto build = [&](int rows, int row0, bool want_iface, int shift, std::vector<int> &rpo,
                     pvec<int> &cio, pvec<int> &srco) {
      std::vector<int> cntr(rows, 0);
      pool.run(rows, [&](long long lo, long long hi) {
        for (int g = int(lo); g < int(hi); g++) {
          const int i = P.perm[row0 + g];
          int c = 0;
          for (int q = rp[i]; q < rp[i + 1]; q++) c += (iface[ci[q]] != 0) == want_iface;
          cntr[g] = c;
        }
      });
      prefix(cntr, rpo);
      cio.resize(rpo[rows]);
      srco.resize(rpo[rows]);
      pool.run(rows, [&](long long lo, long long hi) {
        std::vector<std::pair<int, int>> ent;
        for (int g = int(lo); g < int(hi); g++) {
          const int i = P.perm[row0 + g];
          ent.clear();
          for (int q = rp[i]; q < rp[i + 1]; q++)
            if ((iface[ci[q]] != 0) == want_iface) ent.push_back({P.iperm[ci[q]] - shift, q});
          std::sort(ent.begin(), ent.end());
          for (size_t t = 0; t < ent.size(); t++) {
            cio[rpo[g] + t] = ent[t].first;
            srco[rpo[g] + t] = ent[t].second;
          }
        }
      });
    };
    build(m, 0, true, m, P.eh_rp, P.eh_ci, P.eh_src);
    build(s, m, false, 0, P.eht_rp, P.eht_ci, P.eht_src);
  }
  P.nnz_ehat = (long long)P.eh_ci.size();

  // ---- C_a = C + a^2 I as CSR over the interface rows (Chebyshev and
  // approximate-inverse modes)
  if (opt.c_solver >= 1) {
    std::vector<int> cntr(s, 0);
    pool.run(s, [&](long long lo, long long hi) {
      for (int g = int(lo); g < int(hi); g++) {
        const int i = P.perm[m + g];
        int c = 0;
        for (int q = rp[i]; q < rp[i + 1]; q++) c += iface[ci[q]] != 0;
        cntr[g] = c;
      }
    });
    prefix(cntr, P.cc_rp);
    P.cc_ci.resize(P.cc_rp[s]);
    P.cc_src.resize(P.cc_rp[s]);
    P.cc_diag.resize(s);
    pool.run(s, [&](long long lo, long long hi) {
      std::vector<std::pair<int, int>> ent;
      for (int g = int(lo); g < int(hi); g++) {
        const int i = P.perm[m + g];
        ent.clear();
        for (int q = rp[i]; q < rp[i + 1]; q++)
          if (iface[ci[q]]) ent.push_back({P.iperm[ci[q]] - m, q});
        std::sort(ent.begin(), ent.end());
        for (size_t t = 0; t < ent.size(); t++) {
          P.cc_ci[P.cc_rp[g] + t] = ent[t].first;
          P.cc_src[P.cc_rp[g] + t] = ent[t].second;
          if (ent[t].first == g) P.cc_diag[g] = P.cc_rp[g] + int(t);
        }
      }
    });
  }

  // ---- factor pattern in device order with value sources: row g holds its
  // lower columns (ascending) and the diagonal last; the Ehat Ehat^T terms of
  // each entry are counted in a first pass and written in a second
  {
    P.f_rp.assign(n + 1, 0);
    for (int g = 0; g < n; g++) P.f_rp[g + 1] = P.f_rp[g] + low_cnt[g] + 1;
    const long long nf = P.f_rp[n];
    P.f_ci.resize(nf); P.f_row.resize(nf); P.f_src.resize(nf); P.f_cdiag.resize(nf);
    pvec<int> ecnt(nf);             // Ehat Ehat^T terms per factor entry (all written below)
    // (original column, pa, pb) for row i of an interior block
    auto row_pairs = [&](int i, std::vector<std::array<int, 3>> &pairs) {
      pairs.clear();
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        const int j = ci[q];
        if (!iface[j]) continue;
        for (int q2 = rp[j]; q2 < rp[j + 1]; q2++) {
          const int r = ci[q2];
          if (iface[r]) continue;
          pairs.push_back({r, q, find_pos(rp, ci, r, j)});
        }
      }
    };
    pool.run(n, [&](long long lo, long long hi) {
      std::vector<std::array<int, 3>> pairs;
      std::vector<int> cols;
      for (int g = int(lo); g < int(hi); g++) {
        const int i = P.perm[g];
        const int b = blk_of[i];
        cols.assign(low_ci.begin() + low_rp[g], low_ci.begin() + low_rp[g + 1]);
        cols.push_back(g);
        std::sort(cols.begin(), cols.end());
        if (b < p) row_pairs(i, pairs); else pairs.clear();
        long long e = P.f_rp[g];
        for (int c : cols) {
          const int j = P.perm[c];
          P.f_ci[e] = c;
          P.f_row[e] = g;
          P.f_src[e] = find_pos(rp, ci, i, j);
          P.f_cdiag[e] = (b == p && c == g) ? 1 : 0;
          int k = 0;
          for (const auto &pr : pairs) k += pr[0] == j;
          ecnt[e] = k;
          e++;
        }
      }
    });
    prefix(ecnt, P.f_prp);
    P.f_pa.resize(P.f_prp[nf]);
    P.f_pb.resize(P.f_prp[nf]);
    pool.run(n, [&](long long lo, long long hi) {
      std::vector<std::array<int, 3>> pairs;
      for (int g = int(lo); g < int(hi); g++) {
        const int i = P.perm[g];
        if (blk_of[i] >= p || P.f_prp[P.f_rp[g + 1]] == P.f_prp[P.f_rp[g]]) continue;   // no terms in this row
        row_pairs(i, pairs);
        if (pairs.empty()) continue;
        for (long long e = P.f_rp[g]; e < P.f_rp[g + 1]; e++) {
          const int j = P.perm[P.f_ci[e]];
          int w = P.f_prp[e];
          for (const auto &pr : pairs)
            if (pr[0] == j) { P.f_pa[w] = pr[1]; P.f_pb[w] = pr[2]; w++; }
        }
      }
    });
  }
  P.nnz_factor = (long long)P.f_ci.size();
  pvec<int>().swap(low_ci);

  // ---- level records, slices and the triangular-solve layouts
  P.blk_lvl0.assign(p + 2, 0);
  int maxL = 0;
  for (int b = 0; b <= p; b++) {
    P.blk_lvl0[b] = int(P.lvl_row0.size());
    int r0 = P.blk_row0[b], r1 = P.blk_row0[b + 1];
    int r = r0;
    while (r < r1) {
      int l = level_of[P.perm[r]];
      int e = r;
      while (e < r1 && level_of[P.perm[e]] == l) e++;
      P.lvl_row0.push_back(r);
      P.lvl_nrows.push_back(e - r);
      maxL = std::max(maxL, l + 1);
      r = e;
    }
  }
  P.blk_lvl0[p + 1] = int(P.lvl_row0.size());
  const int nlev = int(P.lvl_row0.size());
  P.lvl_slice0.assign(nlev + 1, 0);
  for (int l = 0; l < nlev; l++)
    P.lvl_slice0[l + 1] = P.lvl_slice0[l] + (P.lvl_nrows[l] + kSlice - 1) / kSlice;
  P.nslice = P.lvl_slice0[nlev];
  // level records in (local level, block) order: level L of every block,
  // blocks ascending.  A block's level-L rows are one contiguous record
  // (record blk_lvl0[b] + L, since every level up to a block's last is
  // non-empty), so this is the stable sort of the rows by local level: the
  // factorisation schedule, and the order of the level-order descriptors
  std::vector<int> lrec, lrec_out(1, 0);
  lrec.reserve(nlev);
  lrec_out.reserve(size_t(nlev) + 1);
  P.fl_ptr.assign(maxL + 1, 0);
  for (int L = 0; L < maxL; L++) {
    for (int b = 0; b <= p; b++) {
      const int rec = P.blk_lvl0[b] + L;
      if (rec >= P.blk_lvl0[b + 1]) continue;
      lrec.push_back(rec);
      lrec_out.push_back(lrec_out.back() + P.lvl_nrows[rec]);
    }
    P.fl_ptr[L + 1] = lrec_out.back();
  }
  P.fl_rows.resize(n);
  pool.run(int(lrec.size()), [&](long long lo, long long hi) {
    for (long long t = lo; t < hi; t++)
      for (int i = 0; i < P.lvl_nrows[lrec[t]]; i++) P.fl_rows[lrec_out[t] + i] = P.lvl_row0[lrec[t]] + i;
  }, 16);
  // upper (L^T) rows: for device row c, the factor entries (g, c), g != c,
  // in ascending g (flat CSR up_rp / up_q)
  // The factor is block diagonal, so each block is transposed on its own
  // (rows ascending inside a block give ascending g per column).
  std::vector<int> up_rp(n + 1, 0);
  pvec<int> up_q;
  {
    std::vector<int> boff(p + 2, 0);   // strictly lower entries of the blocks before b
    for (int b = 0; b <= p; b++) {
      const int r0 = P.blk_row0[b], r1 = P.blk_row0[b + 1];
      boff[b + 1] = boff[b] + (P.f_rp[r1] - P.f_rp[r0]) - (r1 - r0);
    }
    up_q.resize(boff[p + 1]);
    pool.run_dynamic(p + 1, [&](int bi) {
      const int b = border[bi];
      const int r0 = P.blk_row0[b], r1 = P.blk_row0[b + 1];
      for (int g = r0; g < r1; g++)   // counts into up_rp[c + 1], c in this block
        for (int q = P.f_rp[g]; q < P.f_rp[g + 1] - 1; q++) up_rp[P.f_ci[q] + 1]++;
      std::vector<int> fill(r1 - r0);
      int run = boff[b];
      for (int c = r0; c < r1; c++) {
        fill[c - r0] = run;
        run += up_rp[c + 1];
        up_rp[c + 1] = run;
      }
      for (int g = r0; g < r1; g++)
        for (int q = P.f_rp[g]; q < P.f_rp[g + 1] - 1; q++) up_q[fill[P.f_ci[q] - r0]++] = q;
    });
  }
  auto upper_size = [&](int r) { return up_rp[r + 1] - up_rp[r]; };
  auto upper_at = [&](int r, int kk) { return up_q[up_rp[r] + kk]; };
  P.l_sw.assign(P.nslice, 0);
  P.u_sw.assign(P.nslice, 0);
  std::vector<int> slice_row0(P.nslice), slice_rows(P.nslice), slice_blk(P.nslice);
  for (int b = 0; b <= p; b++)
    for (int l = P.blk_lvl0[b]; l < P.blk_lvl0[b + 1]; l++)
      for (int g = P.lvl_slice0[l]; g < P.lvl_slice0[l + 1]; g++) {
        int off = (g - P.lvl_slice0[l]) * kSlice;
        slice_row0[g] = P.lvl_row0[l] + off;
        slice_rows[g] = std::min(kSlice, P.lvl_nrows[l] - off);
        slice_blk[g] = b;
      }
  pool.run(P.nslice, [&](long long lo, long long hi) {
    for (int g = int(lo); g < int(hi); g++) {
      int wl = 0, wu = 0;
      for (int t = 0; t < slice_rows[g]; t++) {
        int r = slice_row0[g] + t;
        wl = std::max(wl, P.f_rp[r + 1] - P.f_rp[r] - 1);
        wu = std::max(wu, upper_size(r));
      }
      P.l_sw[g] = wl; P.u_sw[g] = wu;
    }
  }, 256);
  P.l_soff.assign(P.nslice + 1, 0);
  P.u_soff.assign(P.nslice + 1, 0);
  for (int g = 0; g < P.nslice; g++) {
    P.l_soff[g + 1] = P.l_soff[g] + P.l_sw[g] * kSlice;
    P.u_soff[g + 1] = P.u_soff[g] + P.u_sw[g] * kSlice;
  }
  P.l_col.resize(P.l_soff[P.nslice]);   // every slot is written below
  P.u_col.resize(P.u_soff[P.nslice]);
  P.map_l.resize(P.nnz_factor);
  P.map_u.resize(P.nnz_factor);
  pool.run(P.nnz_factor, [&](long long lo, long long hi) {   // -1: diagonal entries
    for (long long e = lo; e < hi; e++) { P.map_l[e] = -1; P.map_u[e] = -1; }
  });
  pool.run(P.nslice, [&](long long lo, long long hi) {
    for (int g = int(lo); g < int(hi); g++) {
      int b = slice_blk[g];
      int first = P.blk_row0[b], last = P.blk_row0[b + 1] - 1;
      for (int t = 0; t < kSlice; t++) {
        int r = slice_row0[g] + t;
        bool live = t < slice_rows[g];
        int nl = live ? P.f_rp[r + 1] - P.f_rp[r] - 1 : 0;
        for (int kk = 0; kk < P.l_sw[g]; kk++) {
          int slot = P.l_soff[g] + kk * kSlice + t;
          if (kk < nl) { int q = P.f_rp[r] + kk; P.l_col[slot] = P.f_ci[q]; P.map_l[q] = slot; }
          else P.l_col[slot] = first;   // level-0 row: final before any use
        }
        int nu = live ? upper_size(r) : 0;
        for (int kk = 0; kk < P.u_sw[g]; kk++) {
          int slot = P.u_soff[g] + kk * kSlice + t;
          if (kk < nu) { int q = upper_at(r, kk); P.u_col[slot] = P.f_row[q]; P.map_u[q] = slot; }
          else P.u_col[slot] = last;    // top-level row: final before any use
        }
      }
    }
  }, 256);
  // level chunks: all blocks by level number, and C_a alone
  {
    const int maxL2 = int(P.fl_ptr.size()) - 1;
    auto add = [&](int rec) {
      for (int i0 = 0; i0 < P.lvl_nrows[rec]; i0 += kChunk) {
        P.chunks.push_back(rec);
        P.chunks.push_back(i0);
        P.chunks.push_back(std::min(kChunk, P.lvl_nrows[rec] - i0));
        P.chunks.push_back(0);
      }
    };
    P.ch_all_ptr.assign(maxL2 + 1, 0);
    for (int L = 0; L < maxL2; L++) {
      for (int b = 0; b <= p; b++)
        if (P.blk_lvl0[b] + L < P.blk_lvl0[b + 1]) add(P.blk_lvl0[b] + L);
      P.ch_all_ptr[L + 1] = int(P.chunks.size() / 4);
    }
    const int Lc = P.blk_lvl0[p + 1] - P.blk_lvl0[p];
    P.ch_c_ptr.assign(Lc + 1, P.ch_all_ptr[maxL2]);
    for (int L = 0; L < Lc; L++) {
      add(P.blk_lvl0[p] + L);
      P.ch_c_ptr[L + 1] = int(P.chunks.size() / 4);
    }
  }
  // inverse diagonal in slice layout, and the capacities of the TMA solve
  P.row_slot.resize(n);   // the levels cover every row
  for (int l = 0; l < nlev; l++)
    for (int i = 0; i < P.lvl_nrows[l]; i++)
      P.row_slot[P.lvl_row0[l] + i] = (P.lvl_slice0[l] + i / kSlice) * kSlice + i % kSlice;
  P.l_span.resize(2 * size_t(n));   // written for every row below
  P.u_span.resize(2 * size_t(n));
  pool.run(n, [&](long long lo, long long hi) {
    for (int g = int(lo); g < int(hi); g++) {
      const int sl = P.row_slot[g] / kSlice, ln = P.row_slot[g] % kSlice;
      P.l_span[2 * g] = P.l_soff[sl] + ln;
      P.l_span[2 * g + 1] = P.f_rp[g + 1] - P.f_rp[g] - 1;
      P.u_span[2 * g] = P.u_soff[sl] + ln;
      P.u_span[2 * g + 1] = upper_size(g);
    }
  });
  {
    std::atomic<bool> fits(true);
    pool.run(n, [&](long long lo, long long hi) {
      for (long long g = lo; g < hi; g++)
        if (!(P.l_span[2 * g + 1] < 65536 && P.u_span[2 * g + 1] < 65536)) { fits = false; return; }
    });
    if (fits) {
      // the rows in (local level, block) order, as in the schedule
      P.lv_ptr = P.fl_ptr;
      P.lv_desc.resize(4 * size_t(n));
      pool.run(n, [&](long long lo, long long hi) {
        for (long long t = lo; t < hi; t++) {
          const int r = P.fl_rows[t];
          int *d = P.lv_desc.data() + 4 * t;
          d[0] = r;
          d[1] = P.l_span[2 * r];
          d[2] = P.u_span[2 * r];
          d[3] = P.l_span[2 * r + 1] | (P.u_span[2 * r + 1] << 16);
        }
      });
    }
  }
  for (int b = 0; b < p; b++) {
    const int l0 = P.blk_lvl0[b], l1 = P.blk_lvl0[b + 1];
    if (l1 == l0) continue;
    P.tma_zs = std::max(P.tma_zs, P.blk_row0[b + 1] - P.blk_row0[b]);
    P.tma_nl = std::max(P.tma_nl, l1 - l0);
    P.tma_ns = std::max(P.tma_ns, P.lvl_slice0[l1] - P.lvl_slice0[l0] + 1);
    long long be = 0, bs = 0;
    for (int l = l0; l < l1; l++) {
      const int s0 = P.lvl_slice0[l], s1 = P.lvl_slice0[l + 1];
      P.tma_e = std::max(P.tma_e, std::max(P.l_soff[s1] - P.l_soff[s0], P.u_soff[s1] - P.u_soff[s0]));
      P.tma_s = std::max(P.tma_s, s1 - s0);
      be += (P.l_soff[s1] - P.l_soff[s0]) + (P.u_soff[s1] - P.u_soff[s0]);
      bs += 2 * (s1 - s0);
    }
    P.tma_blk_e = std::max(P.tma_blk_e, be);
    P.tma_blk_s = std::max(P.tma_blk_s, bs);
  }
  return DDLR_OK;
}

}  // namespace ddlr
