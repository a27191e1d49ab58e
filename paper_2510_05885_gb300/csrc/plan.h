// Internal symbolic plan shared by the host analysis (analyze.cpp) and the
// device runtime (runtime.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ncl {

// Kinds of diagonal contribution of a lower KKT entry.
enum : int8_t { DIAG_NONE = 0, DIAG_PRIMAL = 1 /* Sigma_i + delta */, DIAG_DUAL = 2 /* -1/rho */ };

struct Instance {
  int32_t n = 0, m = 0;
  int64_t dim = 0;        // n+m (K2r) or n (K)
  int64_t row_off = 0;    // first KKT row of the instance in the batch
  int64_t H_off = 0;      // first H value
  int64_t J_off = 0;      // first J value
  int64_t S_off = 0;      // first Sigma entry
  int64_t nnzH = 0, nnzJ = 0;
};

struct Plan {
  int32_t form = 0;
  int64_t dim = 0;
  std::vector<Instance> inst;
  int64_t nnzH_total = 0, nnzJ_total = 0, nS_total = 0;

  // ---- lower KKT pattern in natural numbering, CSC (rows >= col, sorted),
  // and the recipe of each entry's FP64 value
  int64_t nnzA = 0;
  std::vector<int64_t> A_colptr;       // dim+1
  std::vector<int32_t> A_row;          // nnzA
  std::vector<int32_t> e_h;            // H value index or -1
  std::vector<int32_t> e_j;            // J value index or -1 (K2r off-diagonal block)
  std::vector<int8_t> e_kind;          // DIAG_*
  std::vector<int32_t> e_var;          // Sigma index for DIAG_PRIMAL
  std::vector<int64_t> pair_ptr;       // nnzA+1 (condensed: J^T J products)
  std::vector<int32_t> pair_p, pair_q; // J value indices of each product
  std::vector<int32_t> row_inst;       // dim: instance of each KKT row
  std::vector<int8_t> row_sign;        // dim: +1 primal, -1 dual (natural numbering)

  // ---- full symmetric CSR (natural numbering) for residuals / norms
  std::vector<int64_t> F_rowptr;       // dim+1
  std::vector<int32_t> F_col;          // nnzF
  std::vector<int32_t> F_src;          // lower entry id of each full entry

  // ---- adjoint helpers
  std::vector<int32_t> H_row;          // row of each H value (batch numbering of vars)
  std::vector<int32_t> H_col;
  std::vector<int32_t> J_row;          // KKT/J row of each J value (batch constraint numbering)
  std::vector<int32_t> J_col;          // var of each J value (batch var numbering)
  std::vector<int32_t> J_inst;         // instance of each J value
  std::vector<int32_t> var_row;        // KKT row of each primal var (batch)
  std::vector<int32_t> con_row;        // KKT row of each constraint (K2r; -1 for K)
  std::vector<int64_t> J_rowptr_all;   // CSR of the concatenated J (rows = all constraints)
  int64_t mcon_total = 0;

  // ---- ordering: perm[k] = natural index of pivot k; iperm inverse
  std::vector<int32_t> perm, iperm;

  // ---- supernodes (in postorder, children before parents)
  int32_t ns = 0;
  std::vector<int32_t> sn_col0, sn_ncol, sn_ncolp, sn_nrow, sn_parent, sn_level;
  std::vector<int64_t> sn_rows_off;    // ns+1 (into sn_rows)
  std::vector<int32_t> sn_rows;        // permuted global row indices
  std::vector<int64_t> sn_Loff;        // factor block offsets (elements), ns+1
  std::vector<int64_t> sn_Uoff;        // update block offsets (elements), ns+1
  std::vector<int64_t> sn_Woff;        // forward-solve update vector offsets, ns+1
  std::vector<int32_t> child_ptr, child_list;
  // relmap: for each supernode, for each below row, position in parent's rows
  std::vector<int64_t> relmap_off;     // ns+1
  std::vector<int32_t> relmap;
  // assembly map by front row: entries of the permuted lower matrix that land
  // in row r of supernode s (front-row id = sn_rows_off[s] + r)
  std::vector<int64_t> amap_ptr;       // total rows + 1
  std::vector<int32_t> amap_col;       // local column in the front
  std::vector<int32_t> amap_src;       // lower entry id
  // levels
  int32_t nlevels = 0;
  std::vector<int32_t> level_ptr, level_list;
  std::vector<int32_t> col_inst;       // instance of each permuted column
  std::vector<int8_t> col_sign;        // block sign of each permuted column

  // ---- statistics
  int64_t nnzL = 0;                    // algorithmic strictly-lower nonzeros
  int64_t L_stored = 0, U_stored = 0;
  double flops = 0;
  std::vector<double> inst_flops;
  std::vector<int64_t> inst_nnzL;
  int64_t max_front = 0, max_pivots = 0;
  double analyze_ms = 0;
};

struct AnalyzeInput {
  int32_t form;
  int32_t count;
  const int32_t* n;
  const int32_t* m;
  const int32_t* const* H_rowptr;
  const int32_t* const* H_colind;
  const int32_t* const* J_rowptr;
  const int32_t* const* J_colind;
  int32_t leaf_size;
  int32_t colpad;   // factor block row stride is padded to a multiple of this
};

// Returns "" on success, else an error message (pattern errors start with "pattern:").
std::string analyze(const AnalyzeInput& in, Plan& plan);

}  // namespace ncl
