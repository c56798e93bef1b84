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
//    order is ascending original index (b_order 0) or greedy multicolour
//    (b_order 1) for interior blocks, and likewise (c_order) for C_a.
//  * Device order: inside every block the rows are sorted by (dependency
//    level, elimination position).  This is a topological order of the
//    factor's dependency graph, so it leaves the factor unchanged and lets
//    every level be solved in parallel.
#include "ddlr_plan.h"

#include <algorithm>
#include <array>
#include <numeric>

namespace ddlr {

namespace {

// position of column c in row r of the original CSR, -1 if absent
inline int find_pos(const int *rp, const int *ci, int r, int c) {
  const int *b = ci + rp[r], *e = ci + rp[r + 1];
  const int *it = std::lower_bound(b, e, c);
  return (it != e && *it == c) ? int(it - ci) : -1;
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
  for (int i = 0; i < n; i++) {
    if (rp[i + 1] < rp[i]) { err = "rowptr not monotone"; return DDLR_ERR_INVALID; }
    if (part[i] < 0 || part[i] >= p) { err = "part out of range"; return DDLR_ERR_INVALID; }
    bool diag = false;
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      if (ci[q] < 0 || ci[q] >= n) { err = "column index out of range"; return DDLR_ERR_INVALID; }
      if (q > rp[i] && ci[q] <= ci[q - 1]) { err = "columns not strictly ascending"; return DDLR_ERR_INVALID; }
      if (ci[q] == i) diag = true;
    }
    if (!diag) { err = "missing diagonal entry"; return DDLR_ERR_INVALID; }
  }
  const long long nnz = rp[n];
  for (int i = 0; i < n; i++)
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      int t = find_pos(rp, ci, ci[q], i);
      if (t < 0 || val[t] != val[q]) { err = "matrix is not symmetric"; return DDLR_ERR_INVALID; }
    }
  P = Plan();
  P.n = n; P.p = p; P.nnz = nnz;
  P.orig_row.resize(nnz); P.orig_col.resize(nnz); P.diag_pos.resize(n);
  for (int i = 0; i < n; i++)
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      P.orig_row[q] = i; P.orig_col[q] = ci[q];
      if (ci[q] == i) P.diag_pos[i] = q;
    }

  // ---- Sec. 2.1 classification and eq. (Bmat) order
  std::vector<char> iface(n, 0);
  for (int i = 0; i < n; i++)
    for (int q = rp[i]; q < rp[i + 1]; q++)
      if (part[ci[q]] != part[i]) { iface[i] = 1; break; }
  std::vector<std::vector<int>> members(p + 1);
  for (int i = 0; i < n; i++) members[iface[i] ? p : part[i]].push_back(i);
  int s = int(members[p].size());
  if (s == 0) { err = "no interface nodes (p = 1?)"; return DDLR_ERR_INVALID; }
  if (opt.rank_k < 1 || opt.rank_k > s) { err = "rank_k must be in [1, s]"; return DDLR_ERR_INVALID; }
  P.s = s; P.m = n - s;
  std::vector<int> blk_of(n);
  for (int b = 0; b <= p; b++) for (int i : members[b]) blk_of[i] = b;

  const bool exact = opt.factor == 1;
  P.perm.resize(n); P.iperm.resize(n);
  P.blk_row0.assign(p + 2, 0);
  // per node: level in its block's factor; lower factor pattern per device
  // row as device-order columns (flat CSR, filled block by block)
  std::vector<int> level_of(n, 0);
  std::vector<int> low_rp(n + 1, 0), low_ci;
  low_ci.reserve(size_t(nnz));
  int row_w = 0;
  std::vector<int> loc(n, -1);   // index of a node inside its own block
  for (int b = 0; b <= p; b++)
    for (int t = 0; t < int(members[b].size()); t++) loc[members[b][t]] = t;
  std::vector<int> arp, aci, ord, epos, lrp, lci, lev, dev, col, used, cnt;
  for (int b = 0; b <= p; b++) {
    const std::vector<int> &mem = members[b];
    const int nb = int(mem.size());
    P.blk_row0[b] = row_w;
    // block graph (local indices, flat CSR): A restricted to the block, plus,
    // for interior blocks, the pattern of Ehat Ehat^T
    arp.assign(nb + 1, 0);
    aci.clear();
    for (int t = 0; t < nb; t++) {
      const int i = mem[t];
      const size_t a0 = aci.size();
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        const int j = ci[q];
        if (j != i && blk_of[j] == b) aci.push_back(loc[j]);
        if (b < p && iface[j]) {
          for (int q2 = rp[j]; q2 < rp[j + 1]; q2++) {
            const int r = ci[q2];
            if (r != i && !iface[r]) {
              if (blk_of[r] != b) { err = "Ehat Ehat^T couples two subdomains"; return DDLR_ERR_INVALID; }
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
    ord.resize(nb);
    epos.resize(nb);
    std::iota(ord.begin(), ord.end(), 0);
    if ((b == p && opt.c_order == 1) || (b < p && opt.b_order == 1)) {
      col.assign(nb, -1);
      used.assign(nb + 2, -1);
      int nc = 0;
      for (int t = 0; t < nb; t++) {
        for (int q = arp[t]; q < arp[t + 1]; q++) if (aci[q] < t) used[col[aci[q]]] = t;
        int c = 0;
        while (used[c] == t) c++;
        col[t] = c;
        nc = std::max(nc, c + 1);
      }
      if (b == p) P.ncolors = nc;
      // stable counting sort by colour
      cnt.assign(nc + 1, 0);
      for (int t = 0; t < nb; t++) cnt[col[t] + 1]++;
      for (int c = 0; c < nc; c++) cnt[c + 1] += cnt[c];
      for (int t = 0; t < nb; t++) ord[cnt[col[t]]++] = t;
    }
    for (int e = 0; e < nb; e++) epos[ord[e]] = e;
    // lower pattern in elimination positions (flat CSR lrp/lci)
    lrp.assign(nb + 1, 0);
    lci.clear();
    for (int e = 0; e < nb; e++) {
      const int t = ord[e];
      const size_t l0 = lci.size();
      for (int q = arp[t]; q < arp[t + 1]; q++) if (epos[aci[q]] < e) lci.push_back(epos[aci[q]]);
      std::sort(lci.begin() + l0, lci.end());
      lrp[e + 1] = int(lci.size());
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
        if (total > 60000000LL) { err = "exact factor too large"; return DDLR_ERR_INVALID; }
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
    if (b < p) P.levels_interior = std::max(P.levels_interior, nb ? maxlev + 1 : 0);
    else P.levels_c = maxlev + 1;
    // device order: (level, elimination position), stable counting sort
    cnt.assign(maxlev + 2, 0);
    for (int e = 0; e < nb; e++) cnt[lev[e] + 1]++;
    for (int l = 0; l <= maxlev; l++) cnt[l + 1] += cnt[l];
    dev.resize(nb);
    for (int e = 0; e < nb; e++) dev[cnt[lev[e]]++] = e;
    std::vector<int> drow(nb);   // elimination position -> device row
    for (int d = 0; d < nb; d++) drow[dev[d]] = row_w + d;
    for (int d = 0; d < nb; d++) {
      const int e = dev[d];
      const int i = mem[ord[e]];
      P.perm[row_w + d] = i;
      level_of[i] = lev[e];
      for (int q = lrp[e]; q < lrp[e + 1]; q++) low_ci.push_back(drow[lci[q]]);
      low_rp[row_w + d + 1] = int(low_ci.size());
    }
    row_w += nb;
  }
  P.blk_row0[p + 1] = row_w;
  for (int g = 0; g < n; g++) P.iperm[P.perm[g]] = g;
  const int m = P.m;

  // ---- A in device order, sliced ELL for the SpMV
  {
    int ns = (n + kSlice - 1) / kSlice;
    P.a_nslice = ns;
    P.a_soff.assign(ns + 1, 0);
    P.a_sw.assign(ns, 0);
    for (int g = 0; g < ns; g++) {
      int w = 0;
      for (int l = 0; l < kSlice; l++) {
        int r = g * kSlice + l;
        if (r < n) { int i = P.perm[r]; w = std::max(w, rp[i + 1] - rp[i]); }
      }
      P.a_sw[g] = w;
      P.a_soff[g + 1] = P.a_soff[g] + w * kSlice;
    }
    P.a_col.assign(P.a_soff[ns], 0);
    P.a_src.assign(P.a_soff[ns], -1);
    std::vector<std::pair<int, int>> ent;
    for (int g = 0; g < ns; g++)
      for (int l = 0; l < kSlice; l++) {
        int r = g * kSlice + l;
        int rr = r < n ? r : n - 1;
        ent.clear();
        if (r < n) {
          int i = P.perm[r];
          for (int q = rp[i]; q < rp[i + 1]; q++) ent.push_back({P.iperm[ci[q]], q});
          std::sort(ent.begin(), ent.end());
        }
        for (int kk = 0; kk < P.a_sw[g]; kk++) {
          int slot = P.a_soff[g] + kk * kSlice + l;
          if (kk < int(ent.size())) { P.a_col[slot] = ent[kk].first; P.a_src[slot] = ent[kk].second; }
          else { P.a_col[slot] = rr; P.a_src[slot] = -1; }
        }
      }
  }

  // ---- Ehat (interior rows) and Ehat^T (interface rows)
  P.eh_rp.assign(m + 1, 0);
  for (int g = 0; g < m; g++) {
    int i = P.perm[g];
    std::vector<std::pair<int, int>> ent;
    for (int q = rp[i]; q < rp[i + 1]; q++)
      if (iface[ci[q]]) ent.push_back({P.iperm[ci[q]] - m, q});
    std::sort(ent.begin(), ent.end());
    for (auto &e : ent) { P.eh_ci.push_back(e.first); P.eh_src.push_back(e.second); }
    P.eh_rp[g + 1] = int(P.eh_ci.size());
  }
  P.nnz_ehat = (long long)P.eh_ci.size();
  P.eht_rp.assign(s + 1, 0);
  for (int j = 0; j < s; j++) {
    int i = P.perm[m + j];
    std::vector<std::pair<int, int>> ent;
    for (int q = rp[i]; q < rp[i + 1]; q++)
      if (!iface[ci[q]]) ent.push_back({P.iperm[ci[q]], q});
    std::sort(ent.begin(), ent.end());
    for (auto &e : ent) { P.eht_ci.push_back(e.first); P.eht_src.push_back(e.second); }
    P.eht_rp[j + 1] = int(P.eht_ci.size());
  }

  // ---- factor pattern in device order with value sources
  P.f_rp.assign(n + 1, 0);
  {
    const size_t nf_est = low_ci.size() + size_t(n);
    P.f_ci.reserve(nf_est); P.f_row.reserve(nf_est); P.f_src.reserve(nf_est);
    P.f_prp.reserve(nf_est + 1); P.f_cdiag.reserve(nf_est);
  }
  P.f_prp.push_back(0);
  std::vector<std::array<int, 3>> pairs;
  std::vector<int> cols;
  for (int g = 0; g < n; g++) {
    const int i = P.perm[g];
    const int b = blk_of[i];
    cols.assign(low_ci.begin() + low_rp[g], low_ci.begin() + low_rp[g + 1]);
    cols.push_back(g);
    std::sort(cols.begin(), cols.end());
    // Ehat Ehat^T contributions of row i: (original column, pa, pb)
    pairs.clear();
    if (b < p) {
      for (int q = rp[i]; q < rp[i + 1]; q++) {
        const int j = ci[q];
        if (!iface[j]) continue;
        for (int q2 = rp[j]; q2 < rp[j + 1]; q2++) {
          const int r = ci[q2];
          if (iface[r]) continue;
          pairs.push_back({r, q, find_pos(rp, ci, r, j)});
        }
      }
    }
    for (int c : cols) {
      const int j = P.perm[c];
      P.f_ci.push_back(c);
      P.f_row.push_back(g);
      P.f_src.push_back(find_pos(rp, ci, i, j));
      for (const auto &pr : pairs)
        if (pr[0] == j) { P.f_pa.push_back(pr[1]); P.f_pb.push_back(pr[2]); }
      P.f_prp.push_back(int(P.f_pa.size()));
      P.f_cdiag.push_back((b == p && c == g) ? 1 : 0);
    }
    P.f_rp[g + 1] = int(P.f_ci.size());
  }
  P.nnz_factor = (long long)P.f_ci.size();

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
  // factorisation schedule by local level number
  {
    std::vector<std::vector<int>> byL(maxL);
    for (int g = 0; g < n; g++) byL[level_of[P.perm[g]]].push_back(g);
    P.fl_ptr.assign(maxL + 1, 0);
    for (int L = 0; L < maxL; L++) {
      for (int g : byL[L]) P.fl_rows.push_back(g);
      P.fl_ptr[L + 1] = int(P.fl_rows.size());
    }
  }
  // upper (L^T) rows: for device row c, the factor entries (g, c), g != c,
  // in ascending g (flat CSR up_rp / up_q)
  std::vector<int> up_rp(n + 1, 0), up_q;
  for (int g = 0; g < n; g++)
    for (int q = P.f_rp[g]; q < P.f_rp[g + 1] - 1; q++) up_rp[P.f_ci[q] + 1]++;
  for (int c = 0; c < n; c++) up_rp[c + 1] += up_rp[c];
  up_q.assign(up_rp[n], 0);
  {
    std::vector<int> fill(up_rp.begin(), up_rp.end() - 1);
    for (int g = 0; g < n; g++)
      for (int q = P.f_rp[g]; q < P.f_rp[g + 1] - 1; q++) up_q[fill[P.f_ci[q]]++] = q;
  }
  auto upper_size = [&](int r) { return up_rp[r + 1] - up_rp[r]; };
  auto upper_at = [&](int r, int kk) { return up_q[up_rp[r] + kk]; };
  P.l_soff.assign(P.nslice + 1, 0); P.l_sw.assign(P.nslice, 0);
  P.u_soff.assign(P.nslice + 1, 0); P.u_sw.assign(P.nslice, 0);
  std::vector<int> slice_row0(P.nslice), slice_rows(P.nslice), slice_blk(P.nslice);
  for (int b = 0; b <= p; b++)
    for (int l = P.blk_lvl0[b]; l < P.blk_lvl0[b + 1]; l++)
      for (int g = P.lvl_slice0[l]; g < P.lvl_slice0[l + 1]; g++) {
        int off = (g - P.lvl_slice0[l]) * kSlice;
        slice_row0[g] = P.lvl_row0[l] + off;
        slice_rows[g] = std::min(kSlice, P.lvl_nrows[l] - off);
        slice_blk[g] = b;
      }
  for (int g = 0; g < P.nslice; g++) {
    int wl = 0, wu = 0;
    for (int t = 0; t < slice_rows[g]; t++) {
      int r = slice_row0[g] + t;
      wl = std::max(wl, P.f_rp[r + 1] - P.f_rp[r] - 1);
      wu = std::max(wu, upper_size(r));
    }
    P.l_sw[g] = wl; P.u_sw[g] = wu;
    P.l_soff[g + 1] = P.l_soff[g] + wl * kSlice;
    P.u_soff[g + 1] = P.u_soff[g] + wu * kSlice;
  }
  P.l_col.assign(P.l_soff[P.nslice], 0);
  P.u_col.assign(P.u_soff[P.nslice], 0);
  P.map_l.assign(P.nnz_factor, -1);
  P.map_u.assign(P.nnz_factor, -1);
  for (int g = 0; g < P.nslice; g++) {
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
  // level chunks: all blocks by level number, and C_a alone
  {
    const int maxL = int(P.fl_ptr.size()) - 1;
    auto add = [&](int rec) {
      for (int i0 = 0; i0 < P.lvl_nrows[rec]; i0 += kChunk) {
        P.chunks.push_back(rec);
        P.chunks.push_back(i0);
        P.chunks.push_back(std::min(kChunk, P.lvl_nrows[rec] - i0));
        P.chunks.push_back(0);
      }
    };
    P.ch_all_ptr.assign(maxL + 1, 0);
    for (int L = 0; L < maxL; L++) {
      for (int b = 0; b <= p; b++)
        if (P.blk_lvl0[b] + L < P.blk_lvl0[b + 1]) add(P.blk_lvl0[b] + L);
      P.ch_all_ptr[L + 1] = int(P.chunks.size() / 4);
    }
    const int Lc = P.blk_lvl0[p + 1] - P.blk_lvl0[p];
    P.ch_c_ptr.assign(Lc + 1, P.ch_all_ptr[maxL]);
    for (int L = 0; L < Lc; L++) {
      add(P.blk_lvl0[p] + L);
      P.ch_c_ptr[L + 1] = int(P.chunks.size() / 4);
    }
  }
  // inverse diagonal in slice layout, and the capacities of the TMA solve
  P.row_slot.assign(n, 0);
  for (int l = 0; l < nlev; l++)
    for (int i = 0; i < P.lvl_nrows[l]; i++)
      P.row_slot[P.lvl_row0[l] + i] = (P.lvl_slice0[l] + i / kSlice) * kSlice + i % kSlice;
  P.l_span.assign(2 * size_t(n), 0);
  P.u_span.assign(2 * size_t(n), 0);
  for (int g = 0; g < n; g++) {
    const int sl = P.row_slot[g] / kSlice, ln = P.row_slot[g] % kSlice;
    P.l_span[2 * g] = P.l_soff[sl] + ln;
    P.l_span[2 * g + 1] = P.f_rp[g + 1] - P.f_rp[g] - 1;
    P.u_span[2 * g] = P.u_soff[sl] + ln;
    P.u_span[2 * g + 1] = upper_size(g);
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
