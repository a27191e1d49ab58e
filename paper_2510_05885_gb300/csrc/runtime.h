// Device-side plan, numeric state and kernel launchers (internal).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

namespace ncl {

// Tile/chunk constants shared by the launch planner and the kernels.
constexpr int ASM_ROWS = 32;      // front rows per assembly CTA
constexpr int PANEL_NB = 32;      // pivot columns of a diagonal sub-block
constexpr int MACRO_NB = 128;     // pivot columns per panel of a large front
constexpr int MACRO_ROWS = 64;    // rows below the macro panel per CTA
constexpr int GEMM_TILE = 64;     // SIMT update tile (rows x cols)
constexpr int SOLVE_ROWS = 64;     // below rows per solve CTA
constexpr int MAX_RHS_SWEEP = 8;   // right-hand sides per triangular sweep
constexpr int CHAIN_ROWS = 128;    // pivot rows per CTA of the chained sweeps
constexpr int SMALL_SMEM = 64 * 1024;      // front bytes (nrow x ncolp) of a small front, at most
constexpr int SMALL_SMEM_MAX = 96 * 1024;  // dynamic smem limit of the small-front kernel

// Pointers into device copies of the symbolic plan.
struct DevPlan {
  int64_t dim;
  int32_t ns, ninst, form;
  int64_t nnzA;
  // value recipe of the lower KKT entries (natural numbering)
  const int32_t* e_h;
  const int32_t* e_j;
  const int32_t* e_var;
  const int32_t* e_inst;
  const int8_t* e_kind;
  const int64_t* pair_ptr;
  const int32_t* pair_p;
  const int32_t* pair_q;
  // full symmetric CSR (natural numbering)
  const int64_t* F_rowptr;
  const int32_t* F_col;
  const int32_t* F_src;
  const int32_t* row_inst;
  // supernodes
  const int32_t* sn_col0;
  const int32_t* sn_ncol;
  const int32_t* sn_ncolp;
  const int32_t* sn_nrow;
  const int64_t* sn_rows_off;
  const int32_t* sn_rows;
  const int64_t* sn_Loff;
  const int64_t* sn_Uoff;
  const int64_t* sn_Woff;
  const int64_t* sn_Poff;
  const int32_t* child_ptr;
  const int32_t* child_list;
  const int64_t* relmap_off;
  const int32_t* relmap;
  const int64_t* amap_ptr;
  const int32_t* amap_col;
  const int32_t* amap_src;
  const int32_t* amap_row;   // front row of each assembly-map entry (within its front)
  const int32_t* perm;       // pivot k -> natural index
  const int32_t* col_inst;   // instance of pivot k
  const int8_t* col_sign;    // block sign of pivot k
  int64_t Wtot, Ptot;        // forward / backward solve workspace per RHS
  // adjoint
  const int32_t* H_row;
  const int32_t* H_col;
  const int32_t* J_con;      // constraint of each J value
  const int32_t* J_col;      // KKT row of the variable of each J value
  const int32_t* J_inst;
  const int32_t* con_row;    // KKT row of each constraint (K2r), -1 (K)
  const int64_t* J_rowptr;   // concatenated J by constraint
  const int32_t* var_row;    // KKT row of each primal variable
  const int32_t* con_inst;   // instance of each constraint
  int64_t nnzH, nnzJ, nvar, ncon;
  const int64_t* inst_row_off;  // ninst+1
  const int64_t* sn_Soff;       // split-operand offset of a tensor-core front, -1 otherwise
  const int8_t* sn_flags;       // bit 0: front factored by panels (large front)
  const int64_t* sn_Ioff;       // offset of the inverted 32 x 32 diagonal blocks of L11
  // the J values of each variable (by its KKT row), in constraint order
  const int64_t* JT_ptr;        // dim+1
  const int32_t* JT_idx;        // J value indices
  const int32_t* row_var;       // primal variable of each KKT row, -1 for a dual row
  const int32_t* row_con;       // constraint of each KKT row (K2r dual rows), -1 otherwise
};

// Device pointers of a Newton point (Section 3.1, Eq. K3): n-vectors over the
// concatenated primal variables, m-vectors over the concatenated constraints.
struct NewtonDev {
  const double *g, *x, *lo, *up, *zl, *zu;   // n
  const double *c, *y, *yk, *r;              // m
};

// Numeric state for one precision T (float or double).
template <typename T>
struct DevNum {
  T* L;            // supernodal factor blocks (row-major, ld = ncolp)
  T* U;            // multifrontal update blocks (row-major lower, ld = nbelow)
  T* D;            // pivots, permuted order
  int8_t* piv;     // pivot status: 0 ok, 1 perturbed, 2 zero (stop policy), 3 non-finite
  const double* Klow;  // FP64 lower KKT values (natural numbering)
  float* S;        // split TF32 operands (L_hi, L_lo, W_hi, W_lo planes) of tensor-core fronts
  T* Linv;         // inverses of the unit lower 32 x 32 diagonal blocks of every L11 (row-major)
};

// A dense update C -= A diag(d) B^T restricted to the lower part, over a
// set of fronts: problems are concatenated; each owns a run of tiles, and a
// per-tile array gives each CTA its problem.
struct GemmProb {
  int64_t c_off;     // C element offset (in L or U storage)
  int64_t a_off;     // A = rows of a factor block
  int64_t b_off;     // B = rows of the same block
  int64_t d_off;     // pivots d (index into D)
  int32_t ldc, lda;
  int32_t M, N, K;   // C is M x N (lower part: row + diag_shift >= col), inner dim K
  int32_t c_in_u;    // 1: C lives in U storage, 0: in L storage
  int32_t Nt;        // column tiles
  int64_t tile0;     // first tile of this problem in its launch
};

// One dense update handled by the tensor-core kernel (tc_update.cu):
//   C[i][j] -= sum_{k < 32 nk} L[row_a+i][k0+k] d[k0+k] L[row_b+j][k0+k], j <= i,
// with the four split planes of the front addressed by tensor maps 4*map..4*map+3.
struct TcProb {
  int64_t c_off;
  int64_t tile0;
  int32_t ldc, c_in_u, map, row_a, row_b, k0, nk, M, N, Nt;
};

// One task of the persistent factorisation of a level's large fronts
// (front_dag.cu): kind DAG_DIAG (diagonal block of panel p), DAG_ROWS (the
// 64 rows qe + 64 x.. below panel p) or DAG_UPD (tile (x, y) of panel p's
// trailing update).  cbase / rbase: the front's tile counters (Rt x Ct) and
// row-task counters (P x Rt) in the level's counter array; slot: the sync
// slot of (s, p) (sub-block flags at slot + 1 ..); map: the front's first
// tensor map (4 per front) or -1 for the FMA path.
enum : int32_t { DAG_DIAG = 0, DAG_ROWS = 1, DAG_UPD = 2 };
struct DagTask {
  int32_t kind, s, p, x, y, slot, cbase, rbase, Ct, Rt, map, pad;
};
int front_dag_smem(int esz);
template <typename T>
void launch_front_dag(const DevPlan& P, const DevNum<T>& N, const DagTask* tasks, int ntasks, int grid, int* head,
                      int* cnt, int* sync, const CUtensorMap* maps, int* err, double eps, int policy, long long wait,
                      cudaStream_t st);

void launch_update_tc(const DevPlan& P, const DevNum<float>& N, const TcProb* probs, const int32_t* tile_prob,
                      int64_t ntiles, int stages, const CUtensorMap* maps, int* err, long long wait, cudaStream_t st);
bool tc_encode_maps(const float* split, int64_t rows, int64_t ld, CUtensorMap* out4, std::string* why);
int64_t tc_tiles(int M, int N, int* Nt_out);
int tc_smem_bytes();
void launch_split_rows(const float* L, const float* d, int rows, int ld, int K, float* S, cudaStream_t st);

// launchers (factor.cu)
void launch_kkt_values(const DevPlan& P, const double* const* vals, const double* delta, const double* rho,
                       const double* w, double* Klow, cudaStream_t st);
void launch_row_weights(const DevPlan& P, const double* const* vals, const double* rho, double* w, double* dw,
                        double* ss, cudaStream_t st);
void launch_k1s_rhs(const DevPlan& P, const double* Jv, const double* rho, const double* ss, int nrhs,
                    const double* RT, int64_t ldt, const double* RS, int64_t ldr, double* OUT, int64_t ldo,
                    cudaStream_t st);
void launch_newton_rhs(const DevPlan& P, const double* Jv, const double* rho, const double* mu, NewtonDev pt,
                       double* B, cudaStream_t st);
void launch_newton_recover(const DevPlan& P, const double* Jv, const double* rho, const double* mu, NewtonDev pt,
                           const double* X, double* dx, double* dy, double* dr, double* dzl, double* dzu,
                           cudaStream_t st);
void launch_slack_step(const DevPlan& P, const double* Jv, const double* rho, const double* ss, int nrhs,
                       const double* DT, int64_t ldt, const double* RS, int64_t ldr, double* DS, int64_t lds,
                       cudaStream_t st);
// Kf: the values of the full pattern (nnzF entries) in its row order
void launch_full_values(const DevPlan& P, const double* Klow, double* Kf, int64_t nnzF, cudaStream_t st);
void launch_knorm(const DevPlan& P, const double* Kf, unsigned long long* knorm, cudaStream_t st);
template <typename T>
void launch_assemble(const DevPlan& P, const DevNum<T>& N, const int2* items, const int32_t* cptr, const int4* cran,
                     int count, cudaStream_t st);
template <typename T>
void launch_factor_small(const DevPlan& P, const DevNum<T>& N, const int32_t* list, int count, int smem_bytes,
                         double eps, int policy, cudaStream_t st);
template <typename T>
void launch_gemm_simt(const DevPlan& P, const DevNum<T>& N, const GemmProb* probs, const int32_t* tile_prob,
                      int64_t ntiles, cudaStream_t st);

// launchers (panel.cu)
int small_front_smem(int nrow, int ncp, int esz);
template <typename T>
void launch_invert_blocks(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, cudaStream_t st);
template <typename T>
void launch_subtree_factor(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes,
                           int* counter, int smem, int nsm, double eps, int policy, cudaStream_t st);
template <typename T>
void launch_macro_panel(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int* sync, int* err,
                        double eps, int policy, long long wait, cudaStream_t st);
template <typename T>
void launch_inertia(const DevPlan& P, const DevNum<T>& N, long long* counts, cudaStream_t st);


// launchers (solve.cu)
template <typename T>
void launch_perm_in(const DevPlan& P, T* xp, const double* B, int64_t ldb, int nrhs, cudaStream_t st);
template <typename T>
void launch_perm_out(const DevPlan& P, const T* xp, double* X, int64_t ldx, int nrhs, int accumulate,
                     cudaStream_t st);
int chain_smem(int rows, int esz);
template <typename T>
void launch_fwd_chain(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int smem, bool multi,
                      const int32_t* pptr, const int4* pran, T* xp, const T* W, int nrhs, int* tickets, int* flags,
                      int* err, long long wait, cudaStream_t st);
template <typename T>
void launch_fwd_below(const DevPlan& P, const DevNum<T>& N, const int2* items, const int32_t* cptr, const int4* cran,
                      int count, T* xp, T* W, int nrhs, cudaStream_t st);
template <typename T>
void launch_bwd_below(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int narrow, const T* xp,
                      T* Pw, int nrhs, cudaStream_t st);
template <typename T>
void launch_bwd_chain(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int smem, bool multi, T* xp,
                      const T* Pw, int nrhs, int* tickets, int* flags, int* err, long long wait, cudaStream_t st);
int region_smem(int esz);
template <typename T>
void launch_region_fwd(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes, T* xp,
                       T* W, int nrhs, int* counter, int nsm, cudaStream_t st);
template <typename T>
void launch_region_bwd(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes, T* xp,
                       int nrhs, int* counter, int nsm, cudaStream_t st);
void launch_residual(const DevPlan& P, const double* Kf, const double* B, int64_t ldb, const double* X,
                     int64_t ldx, double* R, int64_t ldr, int nrhs, unsigned long long* rnorm,
                     unsigned long long* xnorm, cudaStream_t st);
void launch_vec_norm(const DevPlan& P, const double* B, int64_t ldb, int nrhs, unsigned long long* out,
                     cudaStream_t st);
void launch_spmv(const DevPlan& P, const double* Klow, const double* X, double* Y, cudaStream_t st);
void launch_multidot(int64_t n, const double* V, int64_t ldv, int nv, const double* w, double* partial,
                     cudaStream_t st);
void launch_multi_axpy(int64_t n, const double* V, int64_t ldv, int nv, const double* c, double a, double* w,
                       cudaStream_t st);
int vec_grid();
void launch_axpy_inplace(double* X, int64_t ldx, const double* Y, int64_t ldy, double a, int64_t dim,
                         int nrhs, cudaStream_t st);
void launch_adjoint_values(const DevPlan& P, const double* Jv, const double* w, const double* X,
                           int64_t ldx, const double* GB, int64_t ldgb, int nrhs, double* G_H,
                           double* G_J, double* G_S, double* G_scal, double* jx, double* jg,
                           cudaStream_t st);

}  // namespace ncl
