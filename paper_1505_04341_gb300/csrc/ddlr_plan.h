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
#include <memory>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "ddlr.h"

namespace ddlr {

constexpr int kSlice = 32;  // rows per sliced-ELL slice (one warp)

// Allocator that leaves new elements uninitialised: the large plan arrays are
// filled in parallel right after they are sized, so the serial zero-fill of
// std::vector's resize would only cost time (first-touch of tens of MB).
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U> struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <typename U> NoInitAlloc(const NoInitAlloc<U> &) {}
  template <typename U> void construct(U *p) noexcept { ::new (static_cast<void *>(p)) U; }
  template <typename U, typename... A> void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T> using pvec = std::vector<T, NoInitAlloc<T>>;
constexpr int kChunk = 256;  // rows per CTA of the level-chunk solve (one per thread)

struct Plan {
  int n = 0, p = 0, s = 0, m = 0;
  long long nnz = 0;
  // ordering: device order ("new") -> original index, and inverse
  pvec<int> perm, iperm;
  std::vector<int> blk_row0;   // p+2: block b = rows [blk_row0[b], blk_row0[b+1]); block p = C_a
  pvec<int> iface_rank;        // s: rank of interface row m+j in ascending original index
  // original CSR helpers (for scaling on the device)
  pvec<int> orig_row;          // nnz: row of each original entry
  pvec<int> orig_col;          // nnz: column of each original entry
  pvec<int> diag_pos;          // n: position of a_ii in the original arrays
  // A in device order as sliced ELL (SpMV of PCG); pad: col = row, src = -1
  int a_nslice = 0;
  std::vector<int> a_soff, a_sw;        // slice offsets (nslice+1) and widths
  pvec<int> a_col, a_src;               // padded arrays
  // Ehat rows (interior rows, m) -> interface column j in [0, s)
  std::vector<int> eh_rp;
  pvec<int> eh_ci, eh_src;
  // Ehat^T rows (interface rows, s) -> interior row (device index < m)
  std::vector<int> eht_rp;
  pvec<int> eht_ci, eht_src;
  // C_a over the interface rows (c_solver 1 and 2 only): columns = device
  // index - m, ascending; value source in the original arrays; the position
  // of each row's diagonal (a^2 is added there)
  std::vector<int> cc_rp;
  pvec<int> cc_ci, cc_src, cc_diag;
  // factor pattern: CSR in device order, columns ascending, diagonal last
  std::vector<int> f_rp;
  pvec<int> f_ci, f_row;
  pvec<int> f_src;                      // value source in the original arrays, -1 = fill
  std::vector<int> f_prp;
  pvec<int> f_pa, f_pb;                 // a^-2 * val[pa]*val[pb] terms (Ehat Ehat^T)
  pvec<unsigned char> f_cdiag;          // diagonal entry of C_a: add a^2
  // dependency levels: level records in device order
  std::vector<int> lvl_row0, lvl_nrows, lvl_slice0;  // nlev (+1 for slice0)
  std::vector<int> blk_lvl0;            // p+2
  // factorisation schedule: rows of all blocks with local level L
  std::vector<int> fl_ptr;
  pvec<int> fl_rows;
  // triangular-solve layouts (sliced ELL over the rows of each level)
  int nslice = 0;
  std::vector<int> l_soff, l_sw, u_soff, u_sw;
  pvec<int> l_col, u_col;                 // strictly lower part of L, strictly upper part of L^T
  pvec<int> map_l, map_u;                 // factor entry -> slot (-1 for diagonal)
  pvec<int> row_slot;                     // row -> slice*32 + lane (inverse diagonal in slice layout)
  pvec<int> l_span, u_span;               // per row: {first slot, entries} of its L and L^T rows
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
  std::vector<int> lv_ptr;
  pvec<int> lv_desc;
  // statistics
  int levels_interior = 0, levels_c = 0, ncolors = 0;
  long long nnz_ehat = 0, nnz_factor = 0;
};

// Builds the plan; returns DDLR_OK or an error status with a message in err.
ddlr_status build_plan(int n, const int *rowptr, const int *colind,
                       const double *val, const int *part, int p,
                       const ddlr_options &opt, Plan &P, std::string &err);

}  // namespace ddlr
