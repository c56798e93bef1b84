// ddlr_plan.h -- host-side symbolic analysis of the DDLR library.
//
// The plan holds everything that depends only on the sparsity pattern and the
// partition: the interior/interface classification (Sec. 2.1), the global
// reordering (eq. Bmat), the elimination order and factor pattern of every
// block of A0 (eq. split), the dependency levels of each factor, and the
// device layouts (CSR / sliced-ELL index arrays and gather maps into the
// caller's value array).  Numeric work (scaling, block forming, factorisation,
// Lanczos) runs on the GPU from these index arrays.
#pragma once
#include <string>
#include <vector>

#include "ddlr.h"

namespace ddlr {

constexpr int kSlice = 32;  // rows per sliced-ELL slice (one warp)
constexpr int kChunk = 256;  // rows per CTA of the level-chunk solve (one per thread)

struct Plan {
  int n = 0, p = 0, s = 0, m = 0;
  long long nnz = 0;
  // ordering: device order ("new") -> original index, and inverse
  std::vector<int> perm, iperm;
  std::vector<int> blk_row0;   // p+2: block b = rows [blk_row0[b], blk_row0[b+1]); block p = C_a
  std::vector<int> iface_rank; // s: rank of interface row m+j in ascending original index
  // original CSR helpers (for scaling on the device)
  std::vector<int> orig_row;   // nnz: row of each original entry
  std::vector<int> orig_col;   // nnz: column of each original entry
  std::vector<int> diag_pos;   // n: position of a_ii in the original arrays
  // A in device order as sliced ELL (SpMV of PCG); pad: col = row, src = -1
  int a_nslice = 0;
  std::vector<int> a_soff, a_sw;        // slice offsets (nslice+1) and widths
  std::vector<int> a_col, a_src;        // padded arrays
  // Ehat rows (interior rows, m) -> interface column j in [0, s)
  std::vector<int> eh_rp, eh_ci, eh_src;
  // Ehat^T rows (interface rows, s) -> interior row (device index < m)
  std::vector<int> eht_rp, eht_ci, eht_src;
  // C_a over the interface rows (Chebyshev mode only): columns = device
  // index - m, ascending; value source in the original arrays; the position
  // of each row's diagonal (a^2 is added there)
  std::vector<int> cc_rp, cc_ci, cc_src, cc_diag;
  // factor pattern: CSR in device order, columns ascending, diagonal last
  std::vector<int> f_rp, f_ci, f_row;
  std::vector<int> f_src;               // value source in the original arrays, -1 = fill
  std::vector<int> f_prp, f_pa, f_pb;   // a^-2 * val[pa]*val[pb] terms (Ehat Ehat^T)
  std::vector<unsigned char> f_cdiag;   // diagonal entry of C_a: add a^2
  // dependency levels: level records in device order
  std::vector<int> lvl_row0, lvl_nrows, lvl_slice0;  // nlev (+1 for slice0)
  std::vector<int> blk_lvl0;            // p+2
  // factorisation schedule: rows of all blocks with local level L
  std::vector<int> fl_ptr, fl_rows;
  // triangular-solve layouts (sliced ELL over the rows of each level)
  int nslice = 0;
  std::vector<int> l_soff, l_sw, l_col;   // strictly lower part of L
  std::vector<int> u_soff, u_sw, u_col;   // strictly upper part of L^T
  std::vector<int> map_l, map_u;          // factor entry -> slot (-1 for diagonal)
  std::vector<int> row_slot;              // row -> slice*32 + lane (inverse diagonal in slice layout)
  std::vector<int> l_span, u_span;        // per row: {first slot, entries} of its L and L^T rows
  // shared-memory capacities of the TMA-pipelined interior solve
  int tma_zs = 0, tma_nl = 0, tma_ns = 0, tma_e = 0, tma_s = 0;
  long long tma_blk_e = 0, tma_blk_s = 0;   // largest per-block totals over all stages
  // level chunks (record, first row, rows) of at most kChunk rows: level L of
  // every block = chunks [ch_all_ptr[L], ch_all_ptr[L+1]); level L of C_a alone
  // = [ch_c_ptr[L], ch_c_ptr[L+1])
  std::vector<int> chunks;                // 4 ints per chunk
  std::vector<int> ch_all_ptr, ch_c_ptr;
  // level-order row descriptors: level L of every block (blocks in order) =
  // entries [lv_ptr[L], lv_ptr[L+1]), each {row, first slot of its L row,
  // first slot of its L^T row, L entries | L^T entries << 16}; empty when a
  // row has 65,536 entries or more (the chunk tables then serve alone)
  std::vector<int> lv_ptr, lv_desc;
  // statistics
  int levels_interior = 0, levels_c = 0, ncolors = 0;
  long long nnz_ehat = 0, nnz_factor = 0;
};

// Builds the plan; returns DDLR_OK or an error status with a message in err.
ddlr_status build_plan(int n, const int *rowptr, const int *colind,
                       const double *val, const int *part, int p,
                       const ddlr_options &opt, Plan &P, std::string &err);

}  // namespace ddlr
