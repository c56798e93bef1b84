// plan_probe.cpp -- test helper: runs the library's host analysis
// (build_plan, csrc/ddlr_plan.cpp) on a pattern read from a file and writes
// the plan's arrays to another, so that tests/test_plan_host.py can check
// them against the definitions on the CPU (no GPU, no CUDA runtime).
//
// Input (native-endian int32 unless noted):
//   n, nnz, p, variant, rank_k, factor, c_order, b_order, c_solver, fill_level,
//   rowptr[n+1], colind[nnz], val[nnz] (float64), part[n]
// Output: status, then records {name length, name bytes, count, int32[count]}
// and a final record of length 0.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ddlr_plan.h"

using ddlr::Plan;

static bool rd(FILE *f, void *p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

template <typename V>
static void put(FILE *f, const char *name, const V &v) {
  const int len = int(std::strlen(name)), cnt = int(v.size());
  fwrite(&len, 4, 1, f);
  fwrite(name, 1, len, f);
  fwrite(&cnt, 4, 1, f);
  for (int i = 0; i < cnt; i++) {
    const int x = int(v[i]);
    fwrite(&x, 4, 1, f);
  }
}

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *in = std::fopen(argv[1], "rb");
  if (!in) return 2;
  int hdr[10];
  if (!rd(in, hdr, sizeof hdr)) return 2;
  const int n = hdr[0], nnz = hdr[1], p = hdr[2];
  std::vector<int> rp(n + 1), ci(nnz), part(n);
  std::vector<double> va(nnz);
  if (!rd(in, rp.data(), 4 * rp.size()) || !rd(in, ci.data(), 4 * ci.size()) ||
      !rd(in, va.data(), 8 * va.size()) || !rd(in, part.data(), 4 * part.size()))
    return 2;
  std::fclose(in);
  ddlr_options o;
  std::memset(&o, 0, sizeof o);
  o.variant = hdr[3];
  o.rank_k = hdr[4];
  o.alpha = 1.0;
  o.theta_mode = 1;
  o.factor = hdr[5];
  o.c_order = hdr[6];
  o.b_order = hdr[7];
  o.c_solver = hdr[8];
  o.fill_level = hdr[9];
  o.lanczos_check = 10;
  o.lanczos_eps = 1e-4;
  o.max_nrhs = 1;
  Plan P;
  std::string err;
  const int st = int(ddlr::build_plan(n, rp.data(), ci.data(), va.data(), part.data(), p, o, P, err));
  FILE *out = std::fopen(argv[2], "wb");
  if (!out) return 2;
  fwrite(&st, 4, 1, out);
  if (st == 0) {
    const std::vector<int> sc = {P.n, P.p, P.s, P.m, P.levels_interior, P.levels_c, P.ncolors, P.nslice};
    put(out, "scalars", sc);
    put(out, "perm", P.perm);
    put(out, "iperm", P.iperm);
    put(out, "blk_row0", P.blk_row0);
    put(out, "f_rp", P.f_rp);
    put(out, "f_ci", P.f_ci);
    put(out, "f_src", P.f_src);
    put(out, "f_prp", P.f_prp);
    put(out, "f_pa", P.f_pa);
    put(out, "f_pb", P.f_pb);
    put(out, "f_cdiag", P.f_cdiag);
    put(out, "lvl_row0", P.lvl_row0);
    put(out, "lvl_nrows", P.lvl_nrows);
    put(out, "lvl_slice0", P.lvl_slice0);
    put(out, "blk_lvl0", P.blk_lvl0);
    put(out, "fl_ptr", P.fl_ptr);
    put(out, "fl_rows", P.fl_rows);
    put(out, "l_soff", P.l_soff);
    put(out, "l_sw", P.l_sw);
    put(out, "l_col", P.l_col);
    put(out, "u_soff", P.u_soff);
    put(out, "u_sw", P.u_sw);
    put(out, "u_col", P.u_col);
    put(out, "map_l", P.map_l);
    put(out, "map_u", P.map_u);
    put(out, "row_slot", P.row_slot);
    put(out, "chunks", P.chunks);
    put(out, "ch_all_ptr", P.ch_all_ptr);
    put(out, "ch_c_ptr", P.ch_c_ptr);
    put(out, "lv_ptr", P.lv_ptr);
    put(out, "lv_desc", P.lv_desc);
    put(out, "eh_rp", P.eh_rp);
    put(out, "eh_ci", P.eh_ci);
    put(out, "eh_src", P.eh_src);
    put(out, "eht_rp", P.eht_rp);
    put(out, "eht_ci", P.eht_ci);
    put(out, "a_soff", P.a_soff);
    put(out, "a_sw", P.a_sw);
    put(out, "a_col", P.a_col);
    put(out, "a_src", P.a_src);
    put(out, "iface_rank", P.iface_rank);
  } else {
    const int len = int(err.size());
    fwrite(&len, 4, 1, out);
    fwrite(err.data(), 1, len, out);
  }
  const int zero = 0;
  fwrite(&zero, 4, 1, out);
  std::fclose(out);
  return 0;
}
