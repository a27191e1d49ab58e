// C ABI entry points (include/ncl_kkt.h): handle, device plan, launch
// schedule, factor / solve with FP64 iterative refinement, adjoint.
#include "../../include/ncl_kkt.h"
#include "plan.h"
#include "runtime.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

namespace ncl {
void launch_adjoint_scalars(const DevPlan& P, const int64_t* inst_n, const int64_t* inst_con_off, const double* rho,
                            const double* dw,
                            const double* X, int64_t ldx, const double* GB, int64_t ldgb, int nrhs,
                            const double* jx, const double* jg, double* G_scal, cudaStream_t st);
}

using namespace ncl;

namespace {

thread_local std::string g_last_error;

ncl_status fail(ncl_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

struct CudaError {
  cudaError_t err;
  std::string where;
};

#define CK(x)                                                  \
  do {                                                         \
    cudaError_t e_ = (x);                                      \
    if (e_ != cudaSuccess) throw CudaError{e_, #x};            \
  } while (0)

// In the FP32 path the large fronts with at least options.tc_min_pivots
// pivots (default 256) get split TF32 operands: their update block
// F22 -= L21 D1 L21^T runs on the tensor cores, and with use_tensor_cores =
// 2 (the default) also the K = 128 trailing updates of their panels; shorter
// inner dimensions stay on the FMA kernels.

// default bound of the inter-CTA waits inside the kernels (about 2 s at 2 GHz)
constexpr long long DEFAULT_WAIT_CYCLES = 4000000000LL;

// per-launch arithmetic (flops on the stored blocks) and minimum traffic
// (bytes), used only for profiling reports
struct Cost {
  double flops = 0, bytes = 0;
};

struct Step {                 // one macro panel of every large front of a level
  int64_t panel_off = 0;      // (s, q0, sync slot, 0): the diagonal CTA and the row CTAs of each front
  int panel_cnt = 0;
  int64_t prob_off = 0;       // SIMT trailing updates
  int prob_cnt = 0;
  int64_t tiles = 0;
  int64_t tp_off = 0;
  int64_t tc_off = 0;         // tensor-core trailing updates
  int tc_cnt = 0;
  int64_t tc_tiles = 0;
  int64_t ttp_off = 0;
  Cost panel_cost, gemm_cost, tc_cost;
};

struct Level {
  int64_t asm_off = 0;
  int asm_cnt = 0;
  int64_t small_off = 0;
  int small_cnt = 0;
  int64_t small_smem = 0;     // dynamic shared memory of the small-front launch
  std::vector<Step> steps;
  int64_t syrk_off = 0;
  int syrk_cnt = 0;
  int64_t syrk_tiles = 0;
  int64_t syrk_tp_off = 0;
  int64_t tsyrk_off = 0;  // tensor-core update-block problems
  int tsyrk_cnt = 0;
  int64_t tsyrk_tiles = 0;
  int64_t tsyrk_tp_off = 0;
  int tsyrk_stages = 1;
  int64_t chain_off = 0;  // block-row items of the level (sweeps)
  int chain_cnt = 0;
  int64_t chain_smem = 0; // dynamic shared memory of the chained sweep kernels
  bool chain_multi = false;  // some supernode of the level has more than one block-row
  int64_t below_off = 0;  // (s, a0) solve items
  int below_cnt = 0;
  int64_t bbelow_off = 0; // (s, a0, k0) backward solve items
  int bbelow_cnt = 0;
  int bbelow_narrow = 0;  //   the first ones: supernodes of at most 32 columns (one warp each)
  int64_t dag_off = 0;    // tasks of the persistent large-front launch
  int dag_cnt = 0;
  Cost asm_cost, small_cost, syrk_cost, fdiag_cost, fbelow_cost, bdiag_cost, bbelow_cost, dag_cost;
};

struct KStat {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

struct Pending {
  const char* name;
  cudaEvent_t a, b;
  Cost c;
};

std::atomic<int64_t> g_kernel_launches{0};

struct HostSched {
  std::vector<int2> asmv, belowv;
  std::vector<int32_t> smallv;
  std::vector<int4> chainv;               // (supernode, first block-row, first 32-row block, 0) per block-row (sweeps)
  std::vector<int32_t> chain_pptr;        // per global 32-row pivot block: its run of child ranges
  std::vector<int4> chain_pran;           // (child, alo, ahi, 0): child W entries landing on the block
  int64_t nblocks = 0;                    // 32-row pivot blocks in all
  int64_t nbrows = 0;                     // block-rows of the chained sweeps in all
  std::vector<int4> bbelowv;              // (s, a0, k0, 0): backward below-rows items, 256 columns each
  std::vector<int32_t> below_cptr;        // per below-rows solve item: its run of child ranges
  std::vector<int4> below_cran;           // (child, lo, hi, 0)
  std::vector<int32_t> asm_cptr;          // per assembly item: its run of child row ranges
  std::vector<int4> asm_cran;             // (child, alo, ahi, 0)
  std::vector<int4> panelv;
  int64_t panel_sync = 0;                 // ints of the panel tickets and sub-block flags
  std::vector<GemmProb> probv;
  std::vector<int32_t> tilep, tilep_tc;   // problem of every tile, per launch
  // tensor-core path (FP32): problems, split-operand offsets, fronts in map order
  bool tc = false;
  std::vector<TcProb> tcv;
  std::vector<int64_t> sn_Soff;
  std::vector<int32_t> tc_fronts;
  int64_t split_max = 0;
  std::vector<int8_t> sn_flags;
  std::vector<int64_t> sn_Ioff;
  // persistent large-front factorisation: tasks of every level, and the
  // counters they wait on (one queue head per level, then the fronts'
  // tile and row-task counters)
  bool dag = false;
  std::vector<DagTask> dagv;
  int64_t dag_counters = 0;
  // triangular sweeps of the region of small subtrees: supernodes with at
  // most 32 pivots all of whose descendants have at most 32 (one warp per
  // maximal subtree); the level launches skip them
  std::vector<int8_t> inreg;
  std::vector<int32_t> regnodes;          // each subtree's supernodes in postorder
  std::vector<int2> regitems;             // (first node, count) per subtree
  Cost reg_fwd_cost, reg_bwd_cost, reg_fac_cost;
  std::vector<int2> invv;                 // (large front, 32-column sub-block): inverses after the factorisation
  int64_t reg_smem = 0;                   // dynamic shared memory of the subtree factorisation
};

}  // namespace

struct ncl_kkt_s {
  Plan plan;
  DevPlan dp{};
  ncl_kkt_options opt{};
  int device = 0;
  int ninst = 1;
  std::vector<void*> allocs;
  int64_t device_bytes = 0;
  // numeric state
  DevNum<float> nf{};
  DevNum<double> nd{};
  double* Klow = nullptr;
  double* Kf = nullptr;        // FP64 values of the full pattern (F) in its row order, for the residual
  double* d_delta = nullptr;
  double* d_rho = nullptr;
  unsigned long long* d_knorm = nullptr;
  unsigned long long* d_norms = nullptr;   // rnorm | xnorm | bnorm, ninst*MAX_RHS_SWEEP each
  long long* d_counts = nullptr;
  int64_t* d_inst_n = nullptr;
  int64_t* d_inst_con_off = nullptr;
  double* h_pinned = nullptr;              // host staging (pinned)
  // schedule
  std::vector<Level> levels;
  HostSched hs;
  int2* d_asm = nullptr;
  int32_t* d_asm_cptr = nullptr;
  int4* d_asm_cran = nullptr;
  int32_t* d_small = nullptr;
  int4* d_panel = nullptr;
  int* d_panel_sync = nullptr;
  GemmProb* d_probs = nullptr;
  int32_t* d_tilep = nullptr;
  int32_t* d_tilep_tc = nullptr;
  int4* d_chain = nullptr;
  int32_t* d_chain_pptr = nullptr;
  int4* d_chain_pran = nullptr;
  int* d_chain_sync = nullptr;              // tickets (fwd, bwd) then flags (fwd, bwd) of the pivot blocks
  int2* d_below = nullptr;
  int4* d_bbelow = nullptr;
  int32_t* d_below_cptr = nullptr;
  int4* d_below_cran = nullptr;
  // solve workspace
  void* xp = nullptr;
  void* own_xp = nullptr;                  // the handle's own sweep workspace
  void* W = nullptr;
  void* Pw = nullptr;
  double* R = nullptr;
  double* jx = nullptr;
  double* jg = nullptr;
  double* GBtmp = nullptr;
  double* Jcopy = nullptr;                 // J values of the last factor (adjoint, K1s, Newton step)
  double* d_mu = nullptr;                  // barrier parameter per instance (Newton step)
  double* d_w = nullptr;                   // condensed form: row weights of J^T W J (Eq. K1 / K1s)
  double* d_dw = nullptr;                  //   their derivative in rho (adjoint)
  double* d_ss = nullptr;                  //   the slack terms Sigma_s (+inf: no slack)
  // FGMRES refinement workspace (allocated on first use)
  double* gm_V = nullptr;                  // (GM_M + 1) x dim Krylov basis
  double* gm_Z = nullptr;                  // GM_M x dim preconditioned directions
  double* gm_w = nullptr;
  double* gm_part = nullptr;               // (GM_M + 1) x vec_grid() partial sums
  double* gm_coef = nullptr;
  double* gm_host = nullptr;               // pinned mirror of gm_part
  const double** d_valptr = nullptr;       // {H, J, Sigma, Sigma_s} pointers of the current factor call
  CUtensorMap* d_maps = nullptr;           // 4 tensor maps per tensor-core front
  TcProb* d_tc = nullptr;
  int* d_err = nullptr;                    // device error flags (bounded waits)
  int2* d_invv = nullptr;                  // sub-blocks whose inverses follow the factorisation
  int2* d_regitems = nullptr;              // small-subtree sweep items and their nodes
  int32_t* d_regnodes = nullptr;
  DagTask* d_dag = nullptr;                // persistent large-front tasks
  int* d_dag_cnt = nullptr;                //   their queue heads and counters
  int n_sm = 148;                          // multiprocessors of the device
  // CUDA graphs: the factor and the triangular sweeps are captured once (on
  // a private stream, after one direct call) and replayed
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t fgraph = nullptr;
  cudaGraphExec_t sgraph[9] = {};
  int factor_calls = 0;
  int sweep_calls[9] = {};
  bool capturing = false;
  // FP64 twin used when the FP32 factor cannot be trusted (built on first use)
  ncl_kkt_s* twin = nullptr;
  bool use_twin = false;
  bool skip_values = false;     // a twin factors the FP64 values copied from its parent
  // per instance, the smallest penalty rho at which an FP32 factorisation had
  // to be replaced by the FP64 one although the FP64 factors were regular
  // (+inf: none yet); precision_fallback = 1 starts later factorisations
  // with rho_i >= fp32_fail_rho[i] for some instance i directly in FP64
  std::vector<double> fp32_fail_rho;
  // one graph for factor + solve + refinement (batch_factor_solve)
  cudaGraphExec_t fsgraph = nullptr;
  int64_t fsgraph_nodes = 0;
  int fs_calls = 0;
  int fs_nir = 0;
  const void* fs_key[2] = {nullptr, nullptr};
  int64_t fs_keyi[3] = {0, 0, 0};
  int64_t fgraph_nodes = 0;
  int64_t sgraph_nodes[9] = {};
  bool factored = false;
  // profiling
  int prof_on = 0;
  std::map<std::string, KStat> prof;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  std::vector<double> h_delta, h_rho;
  std::vector<double> knorm_host;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  template <typename T>
  T* alloc(int64_t count) {
    if (count <= 0) count = 1;
    size_t bytes = (size_t)count * sizeof(T);
    if (opt.max_device_bytes > 0 && device_bytes + (int64_t)bytes > opt.max_device_bytes)
      throw std::bad_alloc();
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    allocs.push_back(p);
    device_bytes += (int64_t)bytes;
    return (T*)p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>((int64_t)v.size());
    if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  ~ncl_kkt_s() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    for (void* p : allocs) cudaFree(p);
    if (h_pinned) cudaFreeHost(h_pinned);
    if (gm_host) cudaFreeHost(gm_host);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    if (fgraph) cudaGraphExecDestroy(fgraph);
    if (fsgraph) cudaGraphExecDestroy(fsgraph);
    delete twin;
    for (auto& g : sgraph)
      if (g) cudaGraphExecDestroy(g);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cudaSetDevice(cur);
  }
};

namespace {

bool is_fp32(const ncl_kkt_s* h) { return h->opt.prec == NCL_PREC_FP32_IR; }
HostSched& hs_ref(ncl_kkt_s* h) { return h->hs; }

// ---------------------------------------------------------------------------
// device plan + schedule
// ---------------------------------------------------------------------------
// launch schedule (host vectors) + bounds validation; no device work
void build_schedule(ncl_kkt_s* h) {
  Plan& P = h->plan;
  const size_t esz = is_fp32(h) ? 4 : 8;
  HostSched& hs = h->hs;
  std::vector<int2>& asmv = hs.asmv;
  std::vector<int2>& belowv = hs.belowv;
  std::vector<int32_t>& smallv = hs.smallv;
  std::vector<int4>& panelv = hs.panelv;
  std::vector<GemmProb>& probv = hs.probv;
  hs.tc = is_fp32(h) && h->opt.use_tensor_cores;
  hs.dag = h->opt.persistent_fronts != 0;
  const int PNB = MACRO_NB;   // pivot columns per panel step
  hs.dagv.clear();
  hs.dag_counters = (int64_t)P.nlevels;   // one queue head per level first
  hs.invv.clear();
  hs.inreg.assign(P.ns, 0);
  hs.regnodes.clear();
  hs.regitems.clear();
  hs.reg_fwd_cost = hs.reg_bwd_cost = hs.reg_fac_cost = Cost{};
  hs.reg_smem = 0;
  if (h->opt.subtree_sweeps) {
    // at most 32 pivots (one inverse block for the sweeps) and small enough
    // for the shared-memory front (the subtree factorisation)
    for (int32_t s = 0; s < P.ns; s++)
      hs.inreg[s] = P.sn_ncol[s] <= 32 && P.sn_nrow[s] <= 512 &&
                    (int64_t)P.sn_nrow[s] * P.sn_ncolp[s] * (int64_t)esz <= SMALL_SMEM;
    // children come before their parent: a supernode outside the region
    // takes its parent out
    for (int32_t s = 0; s < P.ns; s++)
      if (!hs.inreg[s] && P.sn_parent[s] >= 0) hs.inreg[P.sn_parent[s]] = 0;
    std::vector<int32_t> stack;
    for (int32_t r = 0; r < P.ns; r++) {
      if (!hs.inreg[r] || (P.sn_parent[r] >= 0 && hs.inreg[P.sn_parent[r]])) continue;
      // the subtree of r in postorder (iterative: children first)
      const int32_t first = (int32_t)hs.regnodes.size();
      stack.assign(1, r);
      std::vector<int32_t> pre;
      while (!stack.empty()) {
        const int32_t v = stack.back();
        stack.pop_back();
        pre.push_back(v);
        for (int32_t k = P.child_ptr[v]; k < P.child_ptr[v + 1]; k++) stack.push_back(P.child_list[k]);
      }
      // reversed preorder (node after its children, children pushed in
      // order) is a postorder
      for (auto it = pre.rbegin(); it != pre.rend(); ++it) hs.regnodes.push_back(*it);
      hs.regitems.push_back(make_int2(first, (int32_t)pre.size()));
    }
    // largest subtrees first: the kernels hand subtrees out in item order
    // (a work counter), so the longest ones start early and the tail is short
    {
      std::vector<double> wgt(hs.regitems.size(), 0.0);
      for (size_t i = 0; i < hs.regitems.size(); i++)
        for (int q = 0; q < hs.regitems[i].y; q++) {
          const int32_t v = hs.regnodes[hs.regitems[i].x + q];
          wgt[i] += (double)P.sn_nrow[v] * (P.sn_ncol[v] + 1);
        }
      std::vector<size_t> ord(hs.regitems.size());
      for (size_t i = 0; i < ord.size(); i++) ord[i] = i;
      std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return wgt[a] > wgt[b]; });
      std::vector<int2> sorted(ord.size());
      for (size_t i = 0; i < ord.size(); i++) sorted[i] = hs.regitems[ord[i]];
      hs.regitems.swap(sorted);
    }
    for (int32_t s : hs.regnodes) {
      hs.reg_smem = std::max<int64_t>(hs.reg_smem, (small_front_smem(P.sn_nrow[s], P.sn_ncolp[s], (int)esz) + 15) / 16 * 16);
      {
        // subtree factorisation: zero + assemble (L block, update block,
        // children's update blocks), write back, the update block's update
        const double nr = P.sn_nrow[s], ncp = P.sn_ncolp[s], nbb = nr - P.sn_ncol[s], ncc = P.sn_ncol[s];
        double cu = 0;
        for (int32_t k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
          const double cb = P.sn_nrow[P.child_list[k]] - P.sn_ncol[P.child_list[k]];
          cu += 0.5 * cb * (cb + 1);
        }
        hs.reg_fac_cost.bytes += esz * (nr * ncp + 1.5 * nbb * (nbb + 1) + cu) +
                                 12.0 * (double)(P.amap_ptr[P.sn_rows_off[s + 1]] - P.amap_ptr[P.sn_rows_off[s]]);
        hs.reg_fac_cost.flops += 2.0 * (ncc * ncc * ncc / 3.0 + nbb * ncc * ncc) + nbb * (nbb + 1) * ncc;
      }
      const double nb = P.sn_nrow[s] - P.sn_ncol[s], nc = P.sn_ncol[s];
      double child = 0;
      for (int32_t k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++)
        child += P.sn_nrow[P.child_list[k]] - P.sn_ncol[P.child_list[k]];
      hs.reg_fwd_cost.bytes += esz * (1024.0 + nb * nc + 2.0 * nb + child + 2.0 * nc) + 4.0 * child;
      hs.reg_fwd_cost.flops += 2.0 * (nc * nc + nb * nc);
      hs.reg_bwd_cost.bytes += esz * (1024.0 + nb * nc + nb + 3.0 * nc) + 4.0 * nb;
      hs.reg_bwd_cost.flops += 2.0 * (nc * nc + nb * nc);
    }
  }
  hs.sn_Soff.assign(P.ns, -1);
  hs.sn_flags.assign(P.ns, 0);
  hs.sn_Ioff.assign(P.ns + 1, 0);
  hs.asm_cptr.assign(1, 0);
  hs.chain_pptr.assign(1, 0);
  hs.below_cptr.assign(1, 0);
  for (int32_t s = 0; s < P.ns; s++)
    hs.sn_Ioff[s + 1] = hs.sn_Ioff[s] + (int64_t)((P.sn_ncol[s] + 31) / 32) * 1024;
  // problems of one launch are pushed consecutively; each launch's tiles map
  // to its problems through a contiguous run of the per-tile index arrays
  auto push_gemm = [&](GemmProb g, int64_t prob_base, int64_t& tiles, Cost& c) {
    const int Mt = (g.M + GEMM_TILE - 1) / GEMM_TILE, Nt = (g.N + GEMM_TILE - 1) / GEMM_TILE;
    g.Nt = Nt;
    g.tile0 = tiles;
    const int64_t nt = (int64_t)Nt * (Nt + 1) / 2 + (int64_t)(Mt - Nt) * Nt;
    const int32_t idx = (int32_t)((int64_t)probv.size() - prob_base);
    probv.push_back(g);
    hs.tilep.insert(hs.tilep.end(), (size_t)nt, idx);
    tiles += nt;
    const double centries = (double)g.M * g.N - 0.5 * (double)g.N * (g.N - 1);
    c.flops += 2.0 * g.K * centries;
    c.bytes += esz * (2.0 * centries + (double)(g.M + g.N) * g.K);
  };
  auto push_tc = [&](TcProb q, int64_t prob_base, int64_t& tiles, Cost& c) {
    q.tile0 = tiles;
    const int64_t nt = tc_tiles(q.M, q.N, &q.Nt);
    const int32_t idx = (int32_t)((int64_t)hs.tcv.size() - prob_base);
    hs.tcv.push_back(q);
    hs.tilep_tc.insert(hs.tilep_tc.end(), (size_t)nt, idx);
    tiles += nt;
    const double centries = (double)q.M * q.N - 0.5 * (double)q.N * (q.N - 1);
    const double K = 32.0 * q.nk;
    c.flops += 2.0 * K * centries;
    c.bytes += 4.0 * (2.0 * centries) + 16.0 * (double)(q.M + q.N) * K;
  };
  std::vector<int32_t> fid(P.ns, -1);
  h->levels.assign(P.nlevels, Level{});
  for (int32_t l = 0; l < P.nlevels; l++) {
    Level& L = h->levels[l];
    L.asm_off = (int64_t)asmv.size();
    L.small_off = (int64_t)smallv.size();
    L.chain_off = (int64_t)hs.chainv.size();
    L.below_off = (int64_t)belowv.size();
    L.bbelow_off = (int64_t)hs.bbelowv.size();
    std::vector<int32_t> large, small;
    for (int32_t k = P.level_ptr[l]; k < P.level_ptr[l + 1]; k++) {
      const int32_t s = P.level_list[k];
      const int nrow = P.sn_nrow[s], ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s];
      const bool reg = hs.inreg[s] != 0;   // factored and swept by the subtree kernels
      for (int r0 = 0; r0 < nrow && !reg; r0 += ASM_ROWS) {
        asmv.push_back(make_int2(s, r0));
        // rows [alo, ahi) of each child's update block that land on the
        // item's rows [r0, r1) (the relative map is increasing)
        const int r1 = std::min(r0 + ASM_ROWS, nrow);
        for (int32_t k2 = P.child_ptr[s]; k2 < P.child_ptr[s + 1]; k2++) {
          const int32_t c = P.child_list[k2];
          const int32_t* rel = P.relmap.data() + P.relmap_off[c];
          const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
          const int alo = (int)(std::lower_bound(rel, rel + nbc, r0) - rel);
          const int ahi = (int)(std::lower_bound(rel, rel + nbc, r1) - rel);
          if (ahi > alo) hs.asm_cran.push_back(make_int4(c, alo, ahi, 0));
        }
        hs.asm_cptr.push_back((int32_t)hs.asm_cran.size());
      }
      {
        // block-rows of the chained sweeps (every item of the supernode
        // carries its first block-row and first 32-row block) and, per
        // 32-row block, the children's W entries that land on its rows
        const int nblk = (ncol + 31) / 32, nbr = (ncol + CHAIN_ROWS - 1) / CHAIN_ROWS;
        if (!hs.inreg[s]) {
          for (int B = 0; B < nbr; B++) hs.chainv.push_back(make_int4(s, (int32_t)hs.nbrows, (int32_t)hs.nblocks, 0));
          L.chain_smem = std::max<int64_t>(L.chain_smem, chain_smem(std::min(CHAIN_ROWS, ncol), (int)esz));
          if (nbr > 1) L.chain_multi = true;
        }
        for (int b = 0; b < nblk; b++) {
          const int lo = 32 * b, hi = std::min(32 * b + 32, ncol);
          for (int32_t k2 = P.child_ptr[s]; k2 < P.child_ptr[s + 1]; k2++) {
            const int32_t c = P.child_list[k2];
            const int32_t* rel = P.relmap.data() + P.relmap_off[c];
            const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
            const int alo = (int)(std::lower_bound(rel, rel + nbc, lo) - rel);
            const int ahi = (int)(std::lower_bound(rel, rel + nbc, hi) - rel);
            if (ahi > alo) hs.chain_pran.push_back(make_int4(c, alo, ahi, 0));
          }
          hs.chain_pptr.push_back((int32_t)hs.chain_pran.size());
        }
        hs.nblocks += nblk;
        hs.nbrows += nbr;
      }
      for (int a0 = 0; a0 < nrow - ncol && !hs.inreg[s]; a0 += SOLVE_ROWS) {
        belowv.push_back(make_int2(s, a0));
        for (int k0 = 0; k0 < ncol; k0 += 256) hs.bbelowv.push_back(make_int4(s, a0, k0, 0));
        // the children's W entries that land on the rows [a0, a1) below
        const int a1 = std::min(a0 + SOLVE_ROWS, nrow - ncol);
        for (int32_t k2 = P.child_ptr[s]; k2 < P.child_ptr[s + 1]; k2++) {
          const int32_t c = P.child_list[k2];
          const int32_t* rel = P.relmap.data() + P.relmap_off[c];
          const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
          const int lo = (int)(std::lower_bound(rel, rel + nbc, ncol + a0) - rel);
          const int hi = (int)(std::lower_bound(rel, rel + nbc, ncol + a1) - rel);
          if (hi > lo) hs.below_cran.push_back(make_int4(c, lo, hi, 0));
        }
        hs.below_cptr.push_back((int32_t)hs.below_cran.size());
      }
      const bool is_small = ncol <= 64 && nrow <= 512 && (int64_t)nrow * ncp * (int64_t)esz <= SMALL_SMEM;
      if (reg) {
        // the subtree kernels take care of it
      } else if (is_small) {
        smallv.push_back(s);
        small.push_back(s);
        L.small_smem = std::max<int64_t>(L.small_smem, (small_front_smem(nrow, ncp, (int)esz) + 15) / 16 * 16);
      } else {
        large.push_back(s);
      }
      const double nb = nrow - ncol;
      // assembly writes the L and U blocks, reads the children's U blocks
      double child_u = 0;
      for (int32_t k2 = P.child_ptr[s]; k2 < P.child_ptr[s + 1]; k2++) {
        const double cb = P.sn_nrow[P.child_list[k2]] - P.sn_ncol[P.child_list[k2]];
        child_u += 0.5 * cb * (cb + 1);
      }
      if (!reg)
        L.asm_cost.bytes += esz * ((double)nrow * ncp + 0.5 * nb * (nb + 1) + child_u) +
                            12.0 * (double)(P.amap_ptr[P.sn_rows_off[s + 1]] - P.amap_ptr[P.sn_rows_off[s]]);
      if (is_small && !reg) {
        L.small_cost.flops += 2.0 * (ncol * (double)ncol * ncol / 3.0 + nb * ncol * ncol);
        L.small_cost.bytes += esz * 2.0 * nrow * ncp;
      }
      if (!hs.inreg[s]) {
        L.fdiag_cost.bytes += esz * 0.5 * ncol * (ncol + 1.0);
        L.fdiag_cost.flops += (double)ncol * ncol;
        L.fbelow_cost.bytes += esz * nb * ncol;
        L.fbelow_cost.flops += 2.0 * nb * ncol;
        L.bdiag_cost = L.fdiag_cost;
        L.bbelow_cost.bytes += esz * nb * ncol;
        L.bbelow_cost.flops += 2.0 * nb * ncol;
      }
    }
    L.asm_cnt = (int)(asmv.size() - L.asm_off);
    L.small_cnt = (int)(smallv.size() - L.small_off);
    L.chain_cnt = (int)(hs.chainv.size() - L.chain_off);
    L.below_cnt = (int)(belowv.size() - L.below_off);
    L.bbelow_cnt = (int)(hs.bbelowv.size() - L.bbelow_off);
    {
      // the items of supernodes with at most 32 columns first (a warp each),
      // then the others (a CTA each), each group in supernode order
      auto b0 = hs.bbelowv.begin() + L.bbelow_off;
      auto mid = std::stable_partition(b0, hs.bbelowv.end(), [&](const int4& it) { return P.sn_ncol[it.x] <= 32; });
      L.bbelow_narrow = (int)(mid - b0);
    }
    if (hs.tc) {
      int64_t off = 0;
      for (int32_t s : large) {
        if (P.sn_ncol[s] < h->opt.tc_min_pivots) continue;
        fid[s] = (int32_t)hs.tc_fronts.size();
        hs.tc_fronts.push_back(s);
        hs.sn_Soff[s] = off;
        off += (4 * (int64_t)P.sn_nrow[s] * P.sn_ncolp[s] + 31) / 32 * 32;
      }
      hs.split_max = std::max(hs.split_max, off);
    }
    for (int32_t s : large) {
      hs.sn_flags[s] = 1;
      for (int b = 0; b < (P.sn_ncol[s] + 31) / 32; b++) hs.invv.push_back(make_int2(s, b));
    }
    int maxm = 0;
    for (int32_t s : large) maxm = std::max(maxm, (P.sn_ncol[s] + PNB - 1) / PNB);
    L.steps.resize(maxm);
    for (int m = 0; m < maxm; m++) {
      Step& S = L.steps[m];
      S.panel_off = (int64_t)panelv.size();
      S.prob_off = (int64_t)probv.size();
      S.tp_off = (int64_t)hs.tilep.size();
      S.tc_off = (int64_t)hs.tcv.size();
      S.ttp_off = (int64_t)hs.tilep_tc.size();
      for (int32_t s : large) {
        const int nrow = P.sn_nrow[s], ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s];
        const int q0 = m * PNB;
        if (q0 >= ncol) continue;
        const int qe = std::min(q0 + PNB, ncol), w = qe - q0;
        // one diagonal CTA and one CTA per MACRO_ROWS rows below, sharing a
        // sync slot (ticket counter, four sub-block flags)
        const int nrc = (nrow - qe + MACRO_ROWS - 1) / MACRO_ROWS;
        for (int k = 0; k <= nrc; k++) panelv.push_back(make_int4(s, q0, (int32_t)hs.panel_sync, 0));
        hs.panel_sync += 8;
        S.panel_cost.flops += 2.0 * w * (double)w * w / 3.0 + 32.0 * 32 * w + (double)(nrow - qe) * w * (w + 1.0);
        S.panel_cost.bytes += esz * ((double)w * (w + 1) + 1024.0 * ((w + 31) / 32) + 2.0 * w) +
                              esz * 2.0 * (nrow - qe) * w + (fid[s] >= 0 ? 16.0 * (nrow - qe) * w : 0.0);
        if (qe >= ncol) continue;
        if (fid[s] >= 0 && h->opt.use_tensor_cores > 1 && w % 32 == 0) {
          TcProb q{};
          q.c_off = P.sn_Loff[s] + (int64_t)qe * ncp + qe;
          q.ldc = ncp;
          q.c_in_u = 0;
          q.map = fid[s];
          q.row_a = qe;
          q.row_b = qe;
          q.k0 = q0;
          q.nk = w / 32;
          q.M = nrow - qe;
          q.N = ncol - qe;
          push_tc(q, S.tc_off, S.tc_tiles, S.tc_cost);
        } else {
          GemmProb g{};
          g.c_off = P.sn_Loff[s] + (int64_t)qe * ncp + qe;
          g.a_off = P.sn_Loff[s] + (int64_t)qe * ncp + q0;
          g.b_off = g.a_off;
          g.d_off = P.sn_col0[s] + q0;
          g.ldc = ncp;
          g.lda = ncp;
          g.M = nrow - qe;
          g.N = ncol - qe;
          g.K = w;
          g.c_in_u = 0;
          push_gemm(g, S.prob_off, S.tiles, S.gemm_cost);
        }
      }
      S.panel_cnt = (int)(panelv.size() - S.panel_off);
      S.prob_cnt = (int)(probv.size() - S.prob_off);
      S.tc_cnt = (int)(hs.tcv.size() - S.tc_off);
    }
    if (hs.dag && !large.empty()) {
      // the persistent launch's tasks: per front f, panels p of 128 columns;
      // counters cnt[i][j] (trailing updates applied to tile (i, j)) and
      // rows[p][t] (row tasks of panel p done in row tile t).  Order: panel
      // 0's DIAG and ROWS, then per p the tiles of panel p + 1's columns,
      // panel p + 1's DIAG and ROWS, the rest of panel p's trailing update
      // (every dependency of a task comes before it).
      L.dag_off = (int64_t)hs.dagv.size();
      struct FrontDag {
        int32_t s, P, Rt, Ct, map;
        int64_t cbase, rbase;
        std::vector<int32_t> slot;
      };
      std::vector<FrontDag> fr;
      for (int32_t s : large) {
        FrontDag F;
        F.s = s;
        F.P = (P.sn_ncol[s] + MACRO_NB - 1) / MACRO_NB;
        F.Ct = F.P;
        F.Rt = (P.sn_nrow[s] + MACRO_NB - 1) / MACRO_NB;
        F.map = fid[s];
        F.cbase = hs.dag_counters;
        hs.dag_counters += (int64_t)F.Rt * F.Ct;
        F.rbase = hs.dag_counters;
        hs.dag_counters += (int64_t)F.P * F.Rt;
        for (int p = 0; p < F.P; p++) {
          F.slot.push_back((int32_t)hs.panel_sync);
          hs.panel_sync += 8;
        }
        fr.push_back(std::move(F));
      }
      auto task = [&](const FrontDag& F, int kind, int p, int x, int y) {
        DagTask t{};
        t.kind = kind;
        t.s = F.s;
        t.p = p;
        t.x = x;
        t.y = y;
        t.slot = F.slot[p];
        t.cbase = (int32_t)F.cbase;
        t.rbase = (int32_t)F.rbase;
        t.Ct = F.Ct;
        t.Rt = F.Rt;
        t.map = F.map;
        hs.dagv.push_back(t);
      };
      auto diag_rows = [&](const FrontDag& F, int p) {
        task(F, DAG_DIAG, p, 0, 0);
        const int qe = std::min((p + 1) * MACRO_NB, (int)P.sn_ncol[F.s]);
        const int nrc = (P.sn_nrow[F.s] - qe + MACRO_ROWS - 1) / MACRO_ROWS;
        for (int r = 0; r < nrc; r++) task(F, DAG_ROWS, p, r, 0);
      };
      int maxP = 0;
      for (const FrontDag& F : fr) maxP = std::max(maxP, F.P);
      for (const FrontDag& F : fr) diag_rows(F, 0);
      for (int p = 0; p + 1 < maxP; p++) {
        for (const FrontDag& F : fr)
          if (p + 1 < F.P)
            for (int ti = p + 1; ti < F.Rt; ti++) task(F, DAG_UPD, p, ti, p + 1);
        for (const FrontDag& F : fr)
          if (p + 1 < F.P) diag_rows(F, p + 1);
        for (const FrontDag& F : fr)
          if (p + 1 < F.P)
            for (int tj = p + 2; tj < F.Ct; tj++)
              for (int ti = tj; ti < F.Rt; ti++) task(F, DAG_UPD, p, ti, tj);
      }
      L.dag_cnt = (int)(hs.dagv.size() - L.dag_off);
      for (const Step& S : L.steps) {
        L.dag_cost.flops += S.panel_cost.flops + S.gemm_cost.flops + S.tc_cost.flops;
        L.dag_cost.bytes += S.panel_cost.bytes + S.gemm_cost.bytes + S.tc_cost.bytes;
      }
    }
    // update blocks F22 -= L21 D1 L21^T: tensor cores for the fronts with
    // enough pivots, the SIMT kernel for the rest (small fronts included)
    L.syrk_off = (int64_t)probv.size();
    L.syrk_tp_off = (int64_t)hs.tilep.size();
    L.tsyrk_off = (int64_t)hs.tcv.size();
    L.tsyrk_tp_off = (int64_t)hs.tilep_tc.size();
    for (int32_t s : large) {
      const int nrow = P.sn_nrow[s], ncol = P.sn_ncol[s];
      const int nb = nrow - ncol;
      if (nb == 0 || !(hs.tc && fid[s] >= 0)) continue;
      TcProb q{};
      q.c_off = P.sn_Uoff[s];
      q.ldc = nb;
      q.c_in_u = 1;
      q.map = fid[s];
      q.row_a = ncol;
      q.row_b = ncol;
      q.k0 = 0;
      q.nk = (ncol + 31) / 32;
      q.M = nb;
      q.N = nb;
      L.tsyrk_stages = std::max(L.tsyrk_stages, std::min(q.nk, 3));
      push_tc(q, L.tsyrk_off, L.tsyrk_tiles, L.syrk_cost);
    }
    auto push_syrk = [&](int32_t s) {
      const int nrow = P.sn_nrow[s], ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s];
      const int nb = nrow - ncol;
      if (nb == 0 || (hs.tc && fid[s] >= 0)) return;
      GemmProb g{};
      g.c_off = P.sn_Uoff[s];
      g.a_off = P.sn_Loff[s] + (int64_t)ncol * ncp;
      g.b_off = g.a_off;
      g.d_off = P.sn_col0[s];
      g.ldc = nb;
      g.lda = ncp;
      g.M = nb;
      g.N = nb;
      g.K = ncol;
      g.c_in_u = 1;
      push_gemm(g, L.syrk_off, L.syrk_tiles, L.syrk_cost);
    };
    for (int32_t s : large) push_syrk(s);
    for (int32_t s : small) push_syrk(s);   // (region fronts are in neither list)
    L.syrk_cnt = (int)(probv.size() - L.syrk_off);
    L.tsyrk_cnt = (int)(hs.tcv.size() - L.tsyrk_off);
  }
  // bounds of every launch item against its buffers, checked on the host
  // before anything runs on the device
  {
    auto bad = [](const char* what) { throw std::runtime_error(std::string("internal plan check: ") + what); };
    const int64_t Lsz = P.L_stored, Usz = P.U_stored;
    for (int32_t s = 0; s < P.ns; s++) {
      const int64_t nrow = P.sn_nrow[s], ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s], nb = nrow - ncol;
      if (ncol <= 0 || nrow < ncol || ncp < ncol) bad("supernode sizes");
      if (P.sn_Loff[s] + nrow * ncp > P.sn_Loff[s + 1] || P.sn_Loff[s + 1] > Lsz) bad("L block");
      if (P.sn_Uoff[s] + nb * nb > P.sn_Uoff[s + 1] || P.sn_Uoff[s + 1] > Usz) bad("U block");
      if (P.sn_col0[s] < 0 || P.sn_col0[s] + ncol > P.dim) bad("columns");
      if (P.sn_parent[s] >= 0 && P.sn_parent[s] <= s) bad("parent order");
      const int32_t par = P.sn_parent[s];
      for (int64_t a = 0; a < nb; a++) {
        const int32_t r = P.relmap[P.relmap_off[s] + a];
        if (par < 0 || r < 0 || r >= P.sn_nrow[par] || (a > 0 && r <= P.relmap[P.relmap_off[s] + a - 1]))
          bad("relmap");
      }
      for (int64_t r = 0; r < nrow; r++) {
        const int32_t g = P.sn_rows[P.sn_rows_off[s] + r];
        if (g < 0 || g >= P.dim) bad("rows");
        for (int64_t q = P.amap_ptr[P.sn_rows_off[s] + r]; q < P.amap_ptr[P.sn_rows_off[s] + r + 1]; q++)
          if (P.amap_col[q] < 0 || P.amap_col[q] >= ncol || P.amap_col[q] > r || P.amap_src[q] < 0 ||
              P.amap_src[q] >= P.nnzA)
            bad("assembly map");
      }
    }
    if (hs.chain_pptr.size() != (size_t)hs.nblocks + 1 || hs.chainv.size() > (size_t)hs.nbrows) bad("pivot blocks");
    // the small-subtree region: every node once, in a subtree of its own
    // region, children before parents within it, at most 32 pivots
    {
      std::vector<int> seen(P.ns, 0);
      for (const int2& it : hs.regitems) {
        if (it.x < 0 || it.y <= 0 || (size_t)(it.x + it.y) > hs.regnodes.size()) bad("subtree item");
        for (int q = 0; q < it.y; q++) {
          const int32_t v = hs.regnodes[it.x + q];
          if (v < 0 || v >= P.ns || !hs.inreg[v] || P.sn_ncol[v] > 32 || seen[v]++) bad("subtree node");
          for (int32_t k = P.child_ptr[v]; k < P.child_ptr[v + 1]; k++)
            if (!seen[P.child_list[k]]) bad("subtree order");
        }
      }
      for (int32_t v = 0; v < P.ns; v++)
        if (hs.inreg[v] && !seen[v]) bad("subtree coverage");
      if (hs.reg_smem > SMALL_SMEM_MAX) bad("subtree shared memory");
      for (int32_t v = 0; v < P.ns; v++)
        if (hs.inreg[v] && (P.sn_ncol[v] > 32 || P.sn_nrow[v] > 512 ||
                            small_front_smem(P.sn_nrow[v], P.sn_ncolp[v], (int)esz) > hs.reg_smem))
          bad("subtree front");
    }
    for (size_t i = 0; i < hs.chainv.size(); i++) {
      const int4 it = hs.chainv[i];
      if (it.x < 0 || it.x >= P.ns || it.y < 0 || it.y + (P.sn_ncol[it.x] + CHAIN_ROWS - 1) / CHAIN_ROWS > hs.nbrows ||
          it.z < 0 || it.z + (P.sn_ncol[it.x] + 31) / 32 > hs.nblocks)
        bad("pivot blocks");
    }
    for (const Level& L : h->levels)
      if (L.chain_smem > chain_smem(CHAIN_ROWS, (int)esz)) bad("chain shared memory");
    for (int64_t g = 0; g < hs.nblocks; g++) {
      if (hs.chain_pptr[g] > hs.chain_pptr[g + 1] || hs.chain_pptr[g + 1] > (int32_t)hs.chain_pran.size())
        bad("pivot block ranges");
    }
    for (size_t i = 0; i < hs.chainv.size(); i++) {
      const int4 it = hs.chainv[i];
      const int nblk = (P.sn_ncol[it.x] + 31) / 32;
      for (int b = 0; b < nblk; b++)
        for (int32_t e = hs.chain_pptr[it.z + b]; e < hs.chain_pptr[it.z + b + 1]; e++) {
          const int4 cr = hs.chain_pran[e];
          if (cr.x < 0 || cr.x >= P.ns || P.sn_parent[cr.x] != it.x || cr.y < 0 || cr.y >= cr.z ||
              cr.z > P.sn_nrow[cr.x] - P.sn_ncol[cr.x])
            bad("pivot block ranges");
          const int32_t* rel = P.relmap.data() + P.relmap_off[cr.x];
          if (rel[cr.y] < 32 * b || rel[cr.z - 1] >= std::min(32 * b + 32, (int)P.sn_ncol[it.x])) bad("pivot block ranges");
        }
    }
    if (hs.asm_cptr.size() != asmv.size() + 1) bad("assembly child ranges");
    for (size_t i = 0; i < asmv.size(); i++) {
      const int2 it = asmv[i];
      if (it.x < 0 || it.x >= P.ns || it.y < 0 || it.y >= P.sn_nrow[it.x]) bad("assembly item");
      if (hs.asm_cptr[i] > hs.asm_cptr[i + 1] || hs.asm_cptr[i + 1] > (int32_t)hs.asm_cran.size())
        bad("assembly child ranges");
      for (int32_t e = hs.asm_cptr[i]; e < hs.asm_cptr[i + 1]; e++) {
        const int4 cr = hs.asm_cran[e];
        if (cr.x < 0 || cr.x >= P.ns || P.sn_parent[cr.x] != it.x || cr.y < 0 || cr.y >= cr.z ||
            cr.z > P.sn_nrow[cr.x] - P.sn_ncol[cr.x])
          bad("assembly child ranges");
      }
    }
    for (const int4& it : hs.bbelowv)
      if (it.x < 0 || it.x >= P.ns || it.y < 0 || it.y >= P.sn_nrow[it.x] - P.sn_ncol[it.x] || it.y % SOLVE_ROWS ||
          it.z < 0 || it.z >= P.sn_ncol[it.x] || it.z % 256)
        bad("solve item");
    for (const Level& L : h->levels)
      for (int i = 0; i < L.bbelow_cnt; i++)
        if ((i < L.bbelow_narrow) != (P.sn_ncol[hs.bbelowv[L.bbelow_off + i].x] <= 32)) bad("narrow solve items");
    if (hs.below_cptr.size() != belowv.size() + 1) bad("solve child ranges");
    for (size_t i = 0; i < belowv.size(); i++) {
      const int2 it = belowv[i];
      if (it.x < 0 || it.x >= P.ns || it.y < 0 || it.y >= P.sn_nrow[it.x] - P.sn_ncol[it.x]) bad("solve item");
      if (hs.below_cptr[i] > hs.below_cptr[i + 1] || hs.below_cptr[i + 1] > (int32_t)hs.below_cran.size())
        bad("solve child ranges");
      const int a1 = std::min(it.y + SOLVE_ROWS, P.sn_nrow[it.x] - P.sn_ncol[it.x]);
      for (int32_t e = hs.below_cptr[i]; e < hs.below_cptr[i + 1]; e++) {
        const int4 cr = hs.below_cran[e];
        if (cr.x < 0 || cr.x >= P.ns || P.sn_parent[cr.x] != it.x || cr.y < 0 || cr.y >= cr.z ||
            cr.z > P.sn_nrow[cr.x] - P.sn_ncol[cr.x])
          bad("solve child ranges");
        const int32_t* rel = P.relmap.data() + P.relmap_off[cr.x];
        if (rel[cr.y] < P.sn_ncol[it.x] + it.y || rel[cr.z - 1] >= P.sn_ncol[it.x] + a1) bad("solve child ranges");
      }
    }
    for (int32_t s : smallv)
      if (small_front_smem(P.sn_nrow[s], P.sn_ncolp[s], (int)esz) > SMALL_SMEM_MAX || P.sn_ncol[s] > 64 ||
          P.sn_nrow[s] > 512)
        bad("small front smem");
    for (const Level& L : h->levels)
      if (L.small_smem > SMALL_SMEM_MAX) bad("small front smem");
    // every sync slot is shared by exactly 1 + (rows below / MACRO_ROWS) items
    // of one front and panel (the roles come from the slot's ticket counter)
    for (size_t i = 0; i < panelv.size();) {
      const int4 it = panelv[i];
      const int s = it.x;
      if (s < 0 || s >= P.ns || it.y < 0 || it.y >= P.sn_ncol[s] || it.y % PNB || it.z < 0 ||
          it.z + 8 > hs.panel_sync || it.z % 8)
        bad("macro panel item");
      const int qe = std::min(it.y + PNB, P.sn_ncol[s]);
      const size_t n = 1 + (size_t)((P.sn_nrow[s] - qe + MACRO_ROWS - 1) / MACRO_ROWS);
      if (i + n > panelv.size()) bad("macro panel item");
      for (size_t k = 0; k < n; k++)
        if (panelv[i + k].x != s || panelv[i + k].y != it.y || panelv[i + k].z != it.z) bad("macro panel item");
      if (i + n < panelv.size() && panelv[i + n].z == it.z) bad("macro panel item");
      i += n;
    }
    // persistent large-front tasks: every index against its front, its
    // counters, its sync slot and the tensor maps
    for (const DagTask& t : hs.dagv) {
      if (t.s < 0 || t.s >= P.ns) bad("front task");
      const int ncol = P.sn_ncol[t.s], nrow = P.sn_nrow[t.s];
      const int Pf = (ncol + MACRO_NB - 1) / MACRO_NB, Rt = (nrow + MACRO_NB - 1) / MACRO_NB;
      if (t.p < 0 || t.p >= Pf || t.Ct != Pf || t.Rt != Rt) bad("front task");
      if (t.cbase < P.nlevels || (int64_t)t.cbase + (int64_t)Rt * Pf > hs.dag_counters ||
          t.rbase < P.nlevels || (int64_t)t.rbase + (int64_t)Pf * Rt > hs.dag_counters)
        bad("front task counters");
      if (t.slot < 0 || t.slot % 8 || t.slot + 8 > hs.panel_sync) bad("front task slot");
      if (t.map >= (int)hs.tc_fronts.size() || (t.map >= 0 && hs.tc_fronts[t.map] != t.s)) bad("front task map");
      const int qe = std::min((t.p + 1) * MACRO_NB, ncol);
      if (t.kind == DAG_ROWS) {
        if (t.x < 0 || qe + MACRO_ROWS * t.x >= nrow) bad("front task rows");
      } else if (t.kind == DAG_UPD) {
        if (t.p + 1 >= Pf || t.y < t.p + 1 || t.y >= Pf || t.x < t.y || t.x >= Rt) bad("front task tile");
        if (t.map >= 0 && (qe - t.p * MACRO_NB) % 32) bad("front task tile");
      } else if (t.kind != DAG_DIAG) {
        bad("front task kind");
      }
    }
    {
      // replay the task lists in order with the kernel's wait conditions:
      // every task's dependencies must be met by tasks listed before it (the
      // CTAs take tasks in list order, so this makes the waits deadlock-free)
      std::vector<int> c((size_t)hs.dag_counters, 0);
      for (const DagTask& t : hs.dagv) {
        const int ncol = P.sn_ncol[t.s], nrow = P.sn_nrow[t.s];
        const int q0 = t.p * MACRO_NB, qe = std::min(q0 + MACRO_NB, ncol);
        int* tc = c.data() + t.cbase;
        int* rd = c.data() + t.rbase;
        if (t.kind == DAG_DIAG) {
          if (tc[t.p * t.Ct + t.p] < t.p) bad("front task order");
        } else if (t.kind == DAG_ROWS) {
          const int r0 = qe + MACRO_ROWS * t.x, r1 = std::min(r0 + MACRO_ROWS, nrow);
          for (int rt = r0 / MACRO_NB; rt <= (r1 - 1) / MACRO_NB; rt++)
            if (tc[rt * t.Ct + t.p] < t.p) bad("front task order");
          if (qe < ncol) rd[t.p * t.Rt + r0 / MACRO_NB]++;
        } else {
          const int ei = (MACRO_NB * t.x + MACRO_ROWS < nrow) ? 2 : 1;
          const int ej = (MACRO_NB * t.y + MACRO_ROWS < nrow) ? 2 : 1;
          if (rd[t.p * t.Rt + t.x] < ei || rd[t.p * t.Rt + t.y] < ej || tc[t.x * t.Ct + t.y] != t.p)
            bad("front task order");
          tc[t.x * t.Ct + t.y] = t.p + 1;
        }
      }
      // and every trailing update of every front was applied
      for (const DagTask& t : hs.dagv)
        if (t.kind == DAG_DIAG) {
          const int* tc = c.data() + t.cbase;
          for (int tj = 0; tj < t.Ct; tj++)
            for (int ti = tj; ti < t.Rt; ti++)
              if (tc[ti * t.Ct + tj] != std::min(tj, ti)) bad("front task coverage");
        }
    }
    for (const int2& it : hs.invv)
      if (it.x < 0 || it.x >= P.ns || it.y < 0 || 32 * it.y >= P.sn_ncol[it.x] || !hs.sn_flags[it.x] ||
          hs.sn_Ioff[it.x] + (int64_t)(it.y + 1) * 1024 > hs.sn_Ioff[it.x + 1])
        bad("inverse item");
    for (const TcProb& q : hs.tcv) {
      const int64_t csz = q.c_in_u ? Usz : Lsz;
      if (q.map < 0 || q.map >= (int)hs.tc_fronts.size()) bad("tc map");
      const int32_t s = hs.tc_fronts[q.map];
      if (q.M <= 0 || q.N <= 0 || q.N > q.M || q.nk <= 0) bad("tc shape");
      if (q.c_off < 0 || q.c_off + (int64_t)(q.M - 1) * q.ldc + q.N > csz) bad("tc C");
      if (q.row_a + q.M > P.sn_nrow[s] || q.row_b + q.N > P.sn_nrow[s] || q.k0 % 4 != 0) bad("tc operands");
    }
    for (const GemmProb& g : probv) {
      const int64_t csz = g.c_in_u ? Usz : Lsz;
      if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.N > g.M) bad("gemm shape");
      if (g.c_off < 0 || g.c_off + (int64_t)(g.M - 1) * g.ldc + g.N > csz) bad("gemm C");
      if (g.a_off < 0 || g.a_off + (int64_t)(g.M - 1) * g.lda + g.K > Lsz) bad("gemm A");
      if (g.b_off < 0 || g.b_off + (int64_t)(g.N - 1) * g.lda + g.K > Lsz) bad("gemm B");
      if (g.d_off < 0 || g.d_off + g.K > P.dim) bad("gemm d");
    }
    // every tile index of a launch names a problem of that launch
    for (const Level& L : h->levels) {
      auto check = [&](int64_t tp_off, int64_t tiles, int64_t prob_off, int cnt, size_t tp_size, size_t nprob,
                       const std::vector<int32_t>& tp) {
        if (tiles == 0) return;
        if (tp_off < 0 || tp_off + tiles > (int64_t)tp_size || prob_off + cnt > (int64_t)nprob) bad("tile index");
        for (int64_t t = 0; t < tiles; t++)
          if (tp[tp_off + t] < 0 || tp[tp_off + t] >= cnt) bad("tile index");
      };
      for (const Step& S : L.steps) {
        check(S.tp_off, S.tiles, S.prob_off, S.prob_cnt, hs.tilep.size(), probv.size(), hs.tilep);
        check(S.ttp_off, S.tc_tiles, S.tc_off, S.tc_cnt, hs.tilep_tc.size(), hs.tcv.size(), hs.tilep_tc);
      }
      check(L.syrk_tp_off, L.syrk_tiles, L.syrk_off, L.syrk_cnt, hs.tilep.size(), probv.size(), hs.tilep);
      check(L.tsyrk_tp_off, L.tsyrk_tiles, L.tsyrk_off, L.tsyrk_cnt, hs.tilep_tc.size(), hs.tcv.size(), hs.tilep_tc);
    }
  }
}

void build_device(ncl_kkt_s* h) {
  Plan& P = h->plan;
  DevPlan& d = h->dp;
  d.dim = P.dim;
  d.ns = P.ns;
  d.ninst = (int32_t)P.inst.size();
  d.form = P.form;
  d.nnzA = P.nnzA;
  std::vector<int32_t> e_inst(P.nnzA);
  for (int64_t c = 0; c < P.dim; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) e_inst[p] = P.row_inst[P.A_row[p]];
  d.e_h = h->upload(P.e_h);
  d.e_j = h->upload(P.e_j);
  d.e_var = h->upload(P.e_var);
  d.e_inst = h->upload(e_inst);
  d.e_kind = h->upload(P.e_kind);
  d.pair_ptr = h->upload(P.pair_ptr);
  d.pair_p = h->upload(P.pair_p);
  d.pair_q = h->upload(P.pair_q);
  d.F_rowptr = h->upload(P.F_rowptr);
  d.F_col = h->upload(P.F_col);
  d.F_src = h->upload(P.F_src);
  d.row_inst = h->upload(P.row_inst);
  d.sn_col0 = h->upload(P.sn_col0);
  d.sn_ncol = h->upload(P.sn_ncol);
  d.sn_ncolp = h->upload(P.sn_ncolp);
  d.sn_nrow = h->upload(P.sn_nrow);
  d.sn_rows_off = h->upload(P.sn_rows_off);
  d.sn_rows = h->upload(P.sn_rows);
  d.sn_Loff = h->upload(P.sn_Loff);
  d.sn_Uoff = h->upload(P.sn_Uoff);
  d.sn_Woff = h->upload(P.sn_Woff);
  std::vector<int64_t> Poff(P.ns + 1, 0);
  for (int32_t s = 0; s < P.ns; s++) {
    int64_t nb = P.sn_nrow[s] - P.sn_ncol[s];
    Poff[s + 1] = Poff[s] + ((nb + SOLVE_ROWS - 1) / SOLVE_ROWS) * P.sn_ncol[s];
  }
  d.sn_Poff = h->upload(Poff);
  d.child_ptr = h->upload(P.child_ptr);
  d.child_list = h->upload(P.child_list);
  d.relmap_off = h->upload(P.relmap_off);
  d.relmap = h->upload(P.relmap);
  d.amap_ptr = h->upload(P.amap_ptr);
  d.amap_col = h->upload(P.amap_col);
  d.amap_src = h->upload(P.amap_src);
  {
    std::vector<int32_t> arow(P.amap_src.size() ? P.amap_src.size() : 1, 0);
    for (int32_t s = 0; s < P.ns; s++)
      for (int64_t i = P.sn_rows_off[s]; i < P.sn_rows_off[s + 1]; i++)
        for (int64_t q = P.amap_ptr[i]; q < P.amap_ptr[i + 1]; q++) arow[q] = (int32_t)(i - P.sn_rows_off[s]);
    d.amap_row = h->upload(arow);
  }
  d.perm = h->upload(P.perm);
  d.col_inst = h->upload(P.col_inst);
  d.col_sign = h->upload(P.col_sign);
  d.Wtot = P.sn_Woff[P.ns];
  d.Ptot = Poff[P.ns];
  d.H_row = h->upload(P.H_row);
  d.H_col = h->upload(P.H_col);
  d.J_con = h->upload(P.J_row);
  d.J_col = h->upload(P.J_col);
  d.J_inst = h->upload(P.J_inst);
  d.con_row = h->upload(P.con_row);
  d.J_rowptr = h->upload(P.J_rowptr_all);
  d.var_row = h->upload(P.var_row);
  d.nnzH = P.nnzH_total;
  d.nnzJ = P.nnzJ_total;
  d.nvar = P.nS_total;
  d.ncon = P.mcon_total;
  std::vector<int64_t> ro(P.inst.size() + 1), in(P.inst.size()), co(P.inst.size() + 1, 0);
  for (size_t i = 0; i < P.inst.size(); i++) {
    ro[i] = P.inst[i].row_off;
    in[i] = P.inst[i].n;
    co[i + 1] = co[i] + P.inst[i].m;
  }
  ro[P.inst.size()] = P.dim;
  d.inst_row_off = h->upload(ro);
  {
    std::vector<int32_t> ci((size_t)std::max<int64_t>(P.mcon_total, 1), 0);
    for (size_t i = 0; i < P.inst.size(); i++)
      for (int64_t c = co[i]; c < co[i + 1]; c++) ci[c] = (int32_t)i;
    d.con_inst = h->upload(ci);
  }
  {
    // J values by variable (KKT row), in constraint order: counting sort
    std::vector<int64_t> tp((size_t)P.dim + 1, 0);
    for (int32_t c : P.J_col) tp[(size_t)c + 1]++;
    for (int64_t v = 0; v < P.dim; v++) tp[v + 1] += tp[v];
    std::vector<int32_t> ti((size_t)std::max<int64_t>((int64_t)P.J_col.size(), 1), 0);
    std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
    for (size_t e = 0; e < P.J_col.size(); e++) ti[fill[P.J_col[e]]++] = (int32_t)e;
    d.JT_ptr = h->upload(tp);
    d.JT_idx = h->upload(ti);
    // KKT row -> primal variable / constraint
    std::vector<int32_t> rv((size_t)std::max<int64_t>(P.dim, 1), -1), rc((size_t)std::max<int64_t>(P.dim, 1), -1);
    for (size_t v = 0; v < P.var_row.size(); v++) rv[P.var_row[v]] = (int32_t)v;
    for (size_t c = 0; c < P.con_row.size(); c++)
      if (P.con_row[c] >= 0) rc[P.con_row[c]] = (int32_t)c;
    d.row_var = h->upload(rv);
    d.row_con = h->upload(rc);
  }
  h->d_inst_n = h->upload(in);
  h->d_inst_con_off = h->upload(co);

  // numeric storage
  const int ni = d.ninst;
  h->Klow = h->alloc<double>(P.nnzA);
  h->Kf = h->alloc<double>((int64_t)P.F_col.size());
  h->d_delta = h->alloc<double>(ni);
  h->d_rho = h->alloc<double>(ni);
  h->d_knorm = h->alloc<unsigned long long>(ni);
  h->d_norms = h->alloc<unsigned long long>(3 * (int64_t)ni * MAX_RHS_SWEEP);
  h->d_counts = h->alloc<long long>(4 * (int64_t)ni + 1);
  const size_t esz = is_fp32(h) ? 4 : 8;
  auto alloc_num = [&](auto& N, auto tag) {
    using T = decltype(tag);
    N.L = h->alloc<T>(P.L_stored);
    N.U = h->alloc<T>(P.U_stored);
    N.D = h->alloc<T>(P.dim);
    N.piv = h->alloc<int8_t>(P.dim);
    N.Linv = h->alloc<T>(h->hs.sn_Ioff[P.ns]);
    N.Klow = h->Klow;
  };
  if (is_fp32(h)) alloc_num(h->nf, float{});
  else alloc_num(h->nd, double{});
  h->xp = h->alloc<char>((int64_t)P.dim * MAX_RHS_SWEEP * esz);
  h->own_xp = h->xp;
  h->W = h->alloc<char>(std::max<int64_t>(d.Wtot, 1) * MAX_RHS_SWEEP * esz);
  h->Pw = h->alloc<char>(std::max<int64_t>(d.Ptot, 1) * MAX_RHS_SWEEP * esz);
  h->R = h->alloc<double>((int64_t)P.dim * MAX_RHS_SWEEP);
  h->GBtmp = h->alloc<double>((int64_t)P.dim * MAX_RHS_SWEEP);
  h->jx = h->alloc<double>(std::max<int64_t>(d.ncon, 1) * MAX_RHS_SWEEP);
  h->jg = h->alloc<double>(std::max<int64_t>(d.ncon, 1) * MAX_RHS_SWEEP);
  h->Jcopy = h->alloc<double>(std::max<int64_t>(d.nnzJ, 1));
  h->d_mu = h->alloc<double>(std::max<int64_t>(d.ninst, 1));
  if (P.form == 1) {
    h->d_w = h->alloc<double>(std::max<int64_t>(d.ncon, 1));
    h->d_dw = h->alloc<double>(std::max<int64_t>(d.ncon, 1));
    h->d_ss = h->alloc<double>(std::max<int64_t>(d.ncon, 1));
  }
  h->d_valptr = h->alloc<const double*>(4);
  if (hs_ref(h).tc) {
    HostSched& hs = h->hs;
    h->nf.S = h->alloc<float>(std::max<int64_t>(hs.split_max, 32));
    d.sn_Soff = h->upload(hs.sn_Soff);
    std::vector<CUtensorMap> maps(4 * std::max<size_t>(hs.tc_fronts.size(), 1));
    for (size_t f = 0; f < hs.tc_fronts.size(); f++) {
      const int32_t s = hs.tc_fronts[f];
      std::string why;
      if (!tc_encode_maps(h->nf.S + hs.sn_Soff[s], P.sn_nrow[s], P.sn_ncolp[s], &maps[4 * f], &why))
        throw std::runtime_error("tensor map: " + why);
    }
    h->d_maps = reinterpret_cast<CUtensorMap*>(h->alloc<char>((int64_t)(maps.size() * sizeof(CUtensorMap))));
    CK(cudaMemcpy(h->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    h->d_tc = h->upload(hs.tcv);
    h->d_tilep_tc = h->upload(hs.tilep_tc);
  }
  h->d_err = h->alloc<int>(4);
  if (!h->hs.dagv.empty()) h->d_dag = h->upload(h->hs.dagv);
  if (!h->hs.invv.empty()) h->d_invv = h->upload(h->hs.invv);
  if (!h->hs.regitems.empty()) {
    h->d_regitems = h->upload(h->hs.regitems);
    h->d_regnodes = h->upload(h->hs.regnodes);
  }
  h->d_dag_cnt = h->alloc<int>(h->hs.dag_counters + 1);   // + the subtree factorisation's counter
  {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    h->n_sm = std::max(1, nsm);
  }
  d.sn_flags = h->upload(h->hs.sn_flags);
  d.sn_Ioff = h->upload(h->hs.sn_Ioff);
  CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));

  HostSched& hs = h->hs;
  h->d_asm = h->upload(hs.asmv);
  h->d_asm_cptr = h->upload(hs.asm_cptr);
  h->d_asm_cran = h->upload(hs.asm_cran);
  h->d_small = h->upload(hs.smallv);
  h->d_panel = h->upload(hs.panelv);
  h->d_panel_sync = h->alloc<int>(std::max<int64_t>(hs.panel_sync, 8));
  h->d_probs = h->upload(hs.probv);
  h->d_tilep = h->upload(hs.tilep);
  h->d_chain = h->upload(hs.chainv);
  h->d_chain_pptr = h->upload(hs.chain_pptr);
  h->d_chain_pran = h->upload(hs.chain_pran);
  h->d_chain_sync = h->alloc<int>(2 * (int64_t)P.ns + 2 * hs.nbrows + 2);   // + the two subtree-sweep counters
  h->d_below = h->upload(hs.belowv);
  h->d_bbelow = h->upload(hs.bbelowv);
  h->d_below_cptr = h->upload(hs.below_cptr);
  h->d_below_cran = h->upload(hs.below_cran);
  CK(cudaMallocHost(&h->h_pinned, sizeof(double) * (size_t)(7 * ni + 64 + 3 * ni * MAX_RHS_SWEEP)));
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
}

// ---------------------------------------------------------------------------
// numeric phases
// ---------------------------------------------------------------------------

// one kernel launch (skipped when it has no work), counted, and bracketed
// by events when profiling is on
template <typename F>
void klaunch(ncl_kkt_s* h, cudaStream_t st, const char* name, int64_t work, Cost c, F&& f) {
  if (work <= 0) return;
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  if (!h->prof_on) {
    f();
    return;
  }
  while (h->evpool.size() < h->evnext + 2) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->evpool.push_back(e);
  }
  cudaEvent_t a = h->evpool[h->evnext++], b = h->evpool[h->evnext++];
  CK(cudaEventRecord(a, st));
  f();
  CK(cudaEventRecord(b, st));
  h->pending.push_back(Pending{name, a, b, c});
}

// fold the recorded launches into the per-kernel totals (after a sync)
void prof_collect(ncl_kkt_s* h) {
  for (const Pending& p : h->pending) {
    float ms = 0;
    cudaEventElapsedTime(&ms, p.a, p.b);
    KStat& k = h->prof[p.name];
    k.launches++;
    k.ms += ms;
    k.flops += p.c.flops;
    k.bytes += p.c.bytes;
  }
  h->pending.clear();
  h->evnext = 0;
}

Cost scaled(Cost c, double f) {
  c.flops *= f;
  c.bytes *= f;
  return c;
}

// Run `body(stream)` directly, or as a captured graph replayed on `st`.
// The first call of a kind runs directly (it also loads the kernels), the
// second captures on the handle's private stream, later calls replay.
template <typename F>
void run_graphed(ncl_kkt_s* h, cudaGraphExec_t* exec, int64_t* nodes, int* calls, bool allow, cudaStream_t st,
                 F&& body) {
  if (!allow || h->prof_on || h->capturing) {
    body(st);
    return;
  }
  if (!*exec && *calls >= 1) {
    // capturing records the work without running it; the graph then runs on st
    cudaGraph_t g = nullptr;
    const int64_t l0 = g_kernel_launches.load();
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    body(h->cap_stream);
    h->capturing = false;
    CK(cudaStreamEndCapture(h->cap_stream, &g));
    *nodes = g_kernel_launches.load() - l0;
    g_kernel_launches.fetch_sub(*nodes);
    cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
  }
  (*calls)++;
  if (*exec) {
    CK(cudaGraphLaunch(*exec, st));
    g_kernel_launches.fetch_add(*nodes);
  } else {
    body(st);
  }
}

template <typename T>
void run_factor(ncl_kkt_s* h, DevNum<T>& N, cudaStream_t st) {
  const DevPlan& P = h->dp;
  const bool f32 = sizeof(T) == 4;
  const double eps = h->opt.pivot_eps;
  const int pol = h->opt.pivot_policy;
  // the region of small subtrees first (one CTA per subtree, all of it in
  // one launch): every front below a level launch's fronts is then done
  klaunch(h, st, f32 ? "subtree_factor_f32" : "subtree_factor_f64", (int64_t)h->hs.regitems.size(),
          h->hs.reg_fac_cost, [&] {
            launch_subtree_factor<T>(P, N, h->d_regitems, (int)h->hs.regitems.size(), h->d_regnodes,
                                     h->d_dag_cnt + h->hs.dag_counters, (int)h->hs.reg_smem, h->n_sm, eps, pol, st);
          });
  for (const Level& L : h->levels) {
    klaunch(h, st, f32 ? "assemble_f32" : "assemble_f64", L.asm_cnt, L.asm_cost,
            [&] {
              launch_assemble<T>(P, N, h->d_asm + L.asm_off, h->d_asm_cptr + L.asm_off, h->d_asm_cran, L.asm_cnt, st);
            });
    klaunch(h, st, f32 ? "factor_small_f32" : "factor_small_f64", L.small_cnt, L.small_cost, [&] {
      launch_factor_small<T>(P, N, h->d_small + L.small_off, L.small_cnt, (int)L.small_smem, eps, pol, st);
    });
    if (L.dag_cnt > 0) {
      // the level's large fronts in one persistent launch (panels, rows and
      // trailing-update tiles as dependent tasks)
      const int li = (int)(&L - h->levels.data());
      const int grid = std::min(L.dag_cnt, h->n_sm);
      klaunch(h, st, f32 ? "front_dag_f32" : "front_dag_f64", L.dag_cnt, L.dag_cost, [&] {
        launch_front_dag<T>(P, N, h->d_dag + L.dag_off, L.dag_cnt, grid, h->d_dag_cnt + li, h->d_dag_cnt,
                            h->d_panel_sync, h->d_maps, h->d_err, eps, pol, h->opt.wait_cycles, st);
      });
    }
    for (const Step& S : L.steps) {
      if (L.dag_cnt > 0) break;
      klaunch(h, st, f32 ? "macro_panel_f32" : "macro_panel_f64", S.panel_cnt, S.panel_cost, [&] {
        launch_macro_panel<T>(P, N, h->d_panel + S.panel_off, S.panel_cnt, h->d_panel_sync, h->d_err,
                              eps, pol, h->opt.wait_cycles, st);
      });
      klaunch(h, st, f32 ? "update_simt_f32" : "update_simt_f64", S.tiles, S.gemm_cost, [&] {
        launch_gemm_simt<T>(P, N, h->d_probs + S.prob_off, h->d_tilep + S.tp_off, S.tiles, st);
      });
      if constexpr (sizeof(T) == 4)
        klaunch(h, st, "update_tc_f32", S.tc_tiles, S.tc_cost, [&] {
          launch_update_tc(P, N, h->d_tc + S.tc_off, h->d_tilep_tc + S.ttp_off, S.tc_tiles, 3, h->d_maps,
                           h->d_err, h->opt.wait_cycles, st);
        });
    }
    klaunch(h, st, f32 ? "update_simt_f32" : "update_simt_f64", L.syrk_tiles, L.syrk_cost, [&] {
      launch_gemm_simt<T>(P, N, h->d_probs + L.syrk_off, h->d_tilep + L.syrk_tp_off, L.syrk_tiles, st);
    });
    if constexpr (sizeof(T) == 4)
      klaunch(h, st, "update_tc_f32", L.tsyrk_tiles, L.syrk_cost, [&] {
        launch_update_tc(P, N, h->d_tc + L.tsyrk_off, h->d_tilep_tc + L.tsyrk_tp_off, L.tsyrk_tiles,
                         L.tsyrk_stages, h->d_maps, h->d_err, h->opt.wait_cycles, st);
      });
  }
  const int ninv = (int)h->hs.invv.size();
  klaunch(h, st, f32 ? "invert_blocks_f32" : "invert_blocks_f64", ninv,
          Cost{ninv * 32.0 * 32 * 32 / 3.0, ninv * 2.0 * 1024 * sizeof(T)},
          [&] { launch_invert_blocks<T>(P, N, h->d_invv, ninv, st); });
  CK(cudaGetLastError());
}

template <typename T>
void run_sweeps(ncl_kkt_s* h, DevNum<T>& N, int nrhs, cudaStream_t st) {
  const DevPlan& P = h->dp;
  T* xp = (T*)h->xp;
  T* W = (T*)h->W;
  T* Pw = (T*)h->Pw;
  const bool f32 = sizeof(T) == 4;
  const int64_t ns = P.ns, nb = h->hs.nbrows;
  int* tk_f = h->d_chain_sync;
  int* tk_b = tk_f + ns;
  int* fl_f = tk_b + ns;
  int* fl_b = fl_f + nb;
  int* serr = h->d_err + 1;
  int* reg_ctr = h->d_chain_sync + 2 * ns + 2 * nb;
  const HostSched& hs = h->hs;
  CK(cudaMemsetAsync(h->d_chain_sync, 0, (2 * ns + 2 * nb + 2) * sizeof(int), st));
  klaunch(h, st, f32 ? "subtree_fwd_f32" : "subtree_fwd_f64", (int64_t)hs.regitems.size(),
          scaled(hs.reg_fwd_cost, nrhs), [&] {
            launch_region_fwd<T>(P, N, h->d_regitems, (int)hs.regitems.size(), h->d_regnodes, xp, W, nrhs, reg_ctr,
                                 h->n_sm, st);
          });
  for (const Level& L : h->levels) {
    // levels with a supernode of more than one block-row run the chained
    // instantiation (named apart in the profile)
    const char* fname = L.chain_multi ? (f32 ? "fwd_chain_multi_f32" : "fwd_chain_multi_f64")
                                      : (f32 ? "fwd_chain_f32" : "fwd_chain_f64");
    klaunch(h, st, fname, L.chain_cnt, scaled(L.fdiag_cost, nrhs), [&] {
      launch_fwd_chain<T>(P, N, h->d_chain + L.chain_off, L.chain_cnt, (int)L.chain_smem, L.chain_multi,
                          h->d_chain_pptr, h->d_chain_pran, xp, W, nrhs, tk_f, fl_f, serr, h->opt.wait_cycles, st);
    });
    klaunch(h, st, f32 ? "fwd_below_f32" : "fwd_below_f64", L.below_cnt, scaled(L.fbelow_cost, nrhs),
            [&] {
              launch_fwd_below<T>(P, N, h->d_below + L.below_off, h->d_below_cptr + L.below_off, h->d_below_cran,
                                  L.below_cnt, xp, W, nrhs, st);
            });
  }
  for (int l = (int)h->levels.size() - 1; l >= 0; l--) {
    const Level& L = h->levels[l];
    klaunch(h, st, f32 ? "bwd_below_f32" : "bwd_below_f64", L.bbelow_cnt, scaled(L.bbelow_cost, nrhs),
            [&] {
              launch_bwd_below<T>(P, N, h->d_bbelow + L.bbelow_off, L.bbelow_cnt, L.bbelow_narrow, xp, Pw, nrhs, st);
            });
    const char* bname = L.chain_multi ? (f32 ? "bwd_chain_multi_f32" : "bwd_chain_multi_f64")
                                      : (f32 ? "bwd_chain_f32" : "bwd_chain_f64");
    klaunch(h, st, bname, L.chain_cnt, scaled(L.bdiag_cost, nrhs), [&] {
      launch_bwd_chain<T>(P, N, h->d_chain + L.chain_off, L.chain_cnt, (int)L.chain_smem, L.chain_multi, xp, Pw,
                          nrhs, tk_b, fl_b, serr, h->opt.wait_cycles, st);
    });
  }
  klaunch(h, st, f32 ? "subtree_bwd_f32" : "subtree_bwd_f64", (int64_t)hs.regitems.size(),
          scaled(hs.reg_bwd_cost, nrhs), [&] {
            launch_region_bwd<T>(P, N, h->d_regitems, (int)hs.regitems.size(), h->d_regnodes, xp, nrhs, reg_ctr + 1,
                                 h->n_sm, st);
          });
  CK(cudaGetLastError());
}

// X (+)= K^{-1} B with the low-precision factors (one sweep)
void apply_inverse(ncl_kkt_s* h, const double* B, int64_t ldb, double* X, int64_t ldx, int nrhs, int accumulate,
                   cudaStream_t st) {
  // graphs capture the handle's own workspace pointers
  const bool own = h->xp == h->own_xp;
  auto sweeps = [&](cudaStream_t s2) {
    if (is_fp32(h)) run_sweeps<float>(h, h->nf, nrhs, s2);
    else run_sweeps<double>(h, h->nd, nrhs, s2);
  };
  if (is_fp32(h)) {
    klaunch(h, st, "perm_in", h->dp.dim, Cost{0, 12.0 * h->dp.dim * nrhs},
            [&] { launch_perm_in<float>(h->dp, (float*)h->xp, B, ldb, nrhs, st); });
    run_graphed(h, &h->sgraph[nrhs], &h->sgraph_nodes[nrhs], &h->sweep_calls[nrhs], own, st, sweeps);
    klaunch(h, st, "perm_out", h->dp.dim, Cost{0, 20.0 * h->dp.dim * nrhs},
            [&] { launch_perm_out<float>(h->dp, (const float*)h->xp, X, ldx, nrhs, accumulate, st); });
  } else {
    klaunch(h, st, "perm_in", h->dp.dim, Cost{0, 16.0 * h->dp.dim * nrhs},
            [&] { launch_perm_in<double>(h->dp, (double*)h->xp, B, ldb, nrhs, st); });
    run_graphed(h, &h->sgraph[nrhs], &h->sgraph_nodes[nrhs], &h->sweep_calls[nrhs], own, st, sweeps);
    klaunch(h, st, "perm_out", h->dp.dim, Cost{0, 24.0 * h->dp.dim * nrhs},
            [&] { launch_perm_out<double>(h->dp, (const double*)h->xp, X, ldx, nrhs, accumulate, st); });
  }
}

// backward error per (instance, rhs) from the norm slots; returns the max
double backward_errors(ncl_kkt_s* h, int nrhs, cudaStream_t st, std::vector<double>* per = nullptr,
                       const unsigned long long* copied = nullptr) {
  const int ni = h->dp.ninst;
  const size_t cnt = 3 * (size_t)ni * MAX_RHS_SWEEP;
  if (!copied) {
    CK(cudaMemcpyAsync(h->h_pinned, h->d_norms, cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  const unsigned long long* u = copied ? copied : reinterpret_cast<const unsigned long long*>(h->h_pinned);
  auto as_d = [](unsigned long long v) {
    double d;
    std::memcpy(&d, &v, 8);
    return d;
  };
  double worst = 0.0;
  if (per) per->assign((size_t)ni * nrhs, 0.0);
  for (int i = 0; i < ni; i++)
    for (int r = 0; r < nrhs; r++) {
      const double rn = as_d(u[i * nrhs + r]);
      const double xn = as_d(u[ni * MAX_RHS_SWEEP + i * nrhs + r]);
      const double bn = as_d(u[2 * ni * MAX_RHS_SWEEP + i * nrhs + r]);
      const double den = h->knorm_host[i] * xn + bn;
      double eta = den > 0 ? rn / den : (rn > 0 ? INFINITY : 0.0);
      if (!std::isfinite(rn) || !std::isfinite(xn)) eta = INFINITY;
      if (per) (*per)[(size_t)i * nrhs + r] = eta;
      worst = std::max(worst, eta);
    }
  return worst;
}

// residual R = B - K X and the norms; returns max backward error
double residual_eta(ncl_kkt_s* h, const double* B, int64_t ldb, const double* X, int64_t ldx, int nrhs,
                    cudaStream_t st) {
  const int ni = h->dp.ninst;
  CK(cudaMemsetAsync(h->d_norms, 0, 2 * (size_t)ni * MAX_RHS_SWEEP * sizeof(unsigned long long), st));
  const double nnzF = (double)h->plan.F_col.size();
  klaunch(h, st, "residual_f64", h->dp.dim, Cost{2.0 * nnzF * nrhs, nnzF * 16.0 + 8.0 * h->dp.dim * (1 + 3.0 * nrhs)}, [&] {
    launch_residual(h->dp, h->Kf, B, ldb, X, ldx, h->R, h->dp.dim, nrhs, h->d_norms,
                    h->d_norms + ni * MAX_RHS_SWEEP, st);
  });
  CK(cudaGetLastError());
  return backward_errors(h, nrhs, st);
}

// ---------------------------------------------------------------------------
// FGMRES(m)-IR (right preconditioned, flexible GMRES in FP64 with the
// low-precision LDL^T as the preconditioner), for one right-hand side of a
// single-instance handle; used when Richardson refinement stagnates.
// ---------------------------------------------------------------------------
constexpr int GM_M = 20;
constexpr int GM_RESTARTS = 6;

// sums of the per-block partial dot products, in block order
void gm_dots(ncl_kkt_s* h, const double* V, int64_t ldv, int nv, const double* w, double* out, cudaStream_t st) {
  const int G = vec_grid();
  launch_multidot(h->dp.dim, V, ldv, nv, w, h->gm_part, st);
  CK(cudaMemcpyAsync(h->gm_host, h->gm_part, sizeof(double) * G * nv, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < nv; i++) {
    double acc = 0.0;
    for (int b = 0; b < G; b++) acc += h->gm_host[i * G + b];
    out[i] = acc;
  }
}

void gm_axpy(ncl_kkt_s* h, const double* V, int64_t ldv, int nv, const double* c_host, double a, double* w,
             cudaStream_t st) {
  double* hc = h->gm_host + (GM_M + 1) * vec_grid();
  for (int i = 0; i < nv; i++) hc[i] = c_host[i];
  CK(cudaMemcpyAsync(h->gm_coef, hc, sizeof(double) * nv, cudaMemcpyHostToDevice, st));
  launch_multi_axpy(h->dp.dim, V, ldv, nv, h->gm_coef, a, w, st);
  CK(cudaStreamSynchronize(st));   // the pinned coefficients are reused
}

double residual_eta(ncl_kkt_s* h, const double* B, int64_t ldb, const double* X, int64_t ldx, int nrhs,
                    cudaStream_t st);

// refine column x (device) of b; returns the final backward error
double fgmres_column(ncl_kkt_s* h, const double* b, double* x, cudaStream_t st, int* iters) {
  const int64_t dim = h->dp.dim;
  if (!h->gm_V) {
    h->gm_V = h->alloc<double>((GM_M + 1) * dim);
    h->gm_Z = h->alloc<double>(GM_M * dim);
    h->gm_w = h->alloc<double>(dim);
    h->gm_part = h->alloc<double>((GM_M + 1) * (int64_t)vec_grid());
    h->gm_coef = h->alloc<double>(GM_M + 1);
    CK(cudaMallocHost(&h->gm_host, sizeof(double) * ((GM_M + 1) * vec_grid() + GM_M + 8)));
  }
  const int ni = h->dp.ninst;
  CK(cudaMemsetAsync(h->d_norms + 2 * ni * MAX_RHS_SWEEP, 0, (size_t)ni * MAX_RHS_SWEEP * 8, st));
  launch_vec_norm(h->dp, b, dim, 1, h->d_norms + 2 * ni * MAX_RHS_SWEEP, st);
  double eta = residual_eta(h, b, dim, x, dim, 1, st);   // h->R = b - K x
  for (int rs = 0; rs < GM_RESTARTS && eta > h->opt.ir_tol && std::isfinite(eta); rs++) {
    const unsigned long long* u = reinterpret_cast<const unsigned long long*>(h->h_pinned);
    double xn, bn;
    std::memcpy(&xn, &u[MAX_RHS_SWEEP * h->dp.ninst], 8);
    std::memcpy(&bn, &u[2 * MAX_RHS_SWEEP * h->dp.ninst], 8);
    const double target = 0.5 * h->opt.ir_tol * (h->knorm_host[0] * xn + bn);
    double beta;
    gm_dots(h, h->R, dim, 1, h->R, &beta, st);
    beta = std::sqrt(beta);
    if (!(beta > 0)) break;
    const double inv = 1.0 / beta;
    gm_axpy(h, h->R, dim, 1, &inv, 0.0, h->gm_V, st);
    std::vector<double> H((GM_M + 1) * GM_M, 0.0), g(GM_M + 1, 0.0), cs(GM_M), sn(GM_M);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < GM_M; j++) {
      double* Vj = h->gm_V + j * dim;
      double* Zj = h->gm_Z + j * dim;
      apply_inverse(h, Vj, dim, Zj, dim, 1, 0, st);
      launch_spmv(h->dp, h->Klow, Zj, h->gm_w, st);
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; pass++) {
        double hc[GM_M + 1], nc[GM_M + 1];
        gm_dots(h, h->gm_V, dim, j + 1, h->gm_w, hc, st);
        for (int i = 0; i <= j; i++) {
          H[i * GM_M + j] += hc[i];
          nc[i] = -hc[i];
        }
        gm_axpy(h, h->gm_V, dim, j + 1, nc, 1.0, h->gm_w, st);
      }
      double hn;
      gm_dots(h, h->gm_w, dim, 1, h->gm_w, &hn, st);
      hn = std::sqrt(hn);
      H[(j + 1) * GM_M + j] = hn;
      if (hn > 0) {
        const double ih = 1.0 / hn;
        gm_axpy(h, h->gm_w, dim, 1, &ih, 0.0, h->gm_V + (j + 1) * dim, st);
      }
      // Givens rotations on column j of the Hessenberg matrix
      for (int i = 0; i < j; i++) {
        const double a = H[i * GM_M + j], c = H[(i + 1) * GM_M + j];
        H[i * GM_M + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * GM_M + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[j * GM_M + j], c = H[(j + 1) * GM_M + j];
      const double r = std::hypot(a, c);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? c / r : 0.0;
      H[j * GM_M + j] = r;
      H[(j + 1) * GM_M + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      (*iters)++;
      if (std::fabs(g[j + 1]) <= target || !(hn > 0)) break;
    }
    // y = H^-1 g (upper triangular), x += Z y
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; i--) {
      double acc = g[i];
      for (int t = i + 1; t < k; t++) acc -= H[i * GM_M + t] * y[t];
      y[i] = H[i * GM_M + i] != 0 ? acc / H[i * GM_M + i] : 0.0;
    }
    gm_axpy(h, h->gm_Z, dim, k, y.data(), 1.0, x, st);
    eta = residual_eta(h, b, dim, x, dim, 1, st);
  }
  return eta;
}

ncl_status refine_block(ncl_kkt_s* h, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                        cudaStream_t st, ncl_kkt_solve_info* info, double eta, int it);

// solve nrhs <= MAX_RHS_SWEEP columns with Richardson refinement
ncl_status solve_block(ncl_kkt_s* h, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                       cudaStream_t st, ncl_kkt_solve_info* info) {
  const int ni = h->dp.ninst;
  CK(cudaMemsetAsync(h->d_norms + 2 * ni * MAX_RHS_SWEEP, 0, (size_t)ni * MAX_RHS_SWEEP * 8, st));
  klaunch(h, st, "vec_norm", h->dp.dim, Cost{0, 8.0 * h->dp.dim * nrhs},
          [&] { launch_vec_norm(h->dp, B, ldb, nrhs, h->d_norms + 2 * ni * MAX_RHS_SWEEP, st); });
  apply_inverse(h, B, ldb, X, ldx, nrhs, 0, st);
  const double eta0 = residual_eta(h, B, ldb, X, ldx, nrhs, st);
  return refine_block(h, nrhs, B, ldb, X, ldx, st, info, eta0, 0);
}

// Richardson refinement from the current X (h->R holds B - K X and eta its
// backward error), FGMRES when it stagnates
ncl_status refine_block(ncl_kkt_s* h, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                        cudaStream_t st, ncl_kkt_solve_info* info, double eta, int it) {
  const int maxit = h->opt.ir_max_iter;
  bool stagnated = false;
  while (eta > h->opt.ir_tol && it < maxit && std::isfinite(eta)) {
    apply_inverse(h, h->R, h->dp.dim, X, ldx, nrhs, 1, st);
    it++;
    const double prev = eta;
    eta = residual_eta(h, B, ldb, X, ldx, nrhs, st);
    if (eta > h->opt.ir_switch * prev && h->opt.use_fgmres && h->dp.ninst == 1) {
      stagnated = true;   // Richardson stagnates (kappa * u_factor is not small): switch to FGMRES
      break;
    }
  }
  bool used_gm = false;
  if (eta > h->opt.ir_tol && std::isfinite(eta) && h->opt.use_fgmres && h->dp.ninst == 1 &&
      (stagnated || it >= maxit)) {
    used_gm = true;
    eta = 0.0;
    for (int r = 0; r < nrhs; r++)
      eta = std::max(eta, fgmres_column(h, B + r * ldb, X + r * ldx, st, &it));
  }
  if (info) {
    info->ir_iters = std::max(info->ir_iters, it);
    info->backward_err = std::max(info->backward_err, eta);
    if (used_gm) info->used_fgmres = 1;
  }
  if (!std::isfinite(eta)) return fail(NCL_ERR_NUMERIC, "non-finite residual or solution");
  if (eta > h->opt.ir_tol) return NCL_ERR_IR_NOT_CONVERGED;
  return NCL_OK;
}

ncl_status do_solve(ncl_kkt_s* h, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                    cudaStream_t st, ncl_kkt_solve_info* info, bool allow_escalate = true);

// validate and stage the scalars and value pointers of a factor call
ncl_status prepare_factor(ncl_kkt_s* h, const double* Hv, const double* Jv, const double* S, const double* delta,
                          const double* rho, cudaStream_t st, const double* Ss = nullptr) {
  const int ni = h->dp.ninst;
  for (int i = 0; i < ni; i++) {
    if (!(rho[i] > 0) || !std::isfinite(rho[i])) return fail(NCL_ERR_INVALID_ARG, "rho must be positive and finite");
    if (!std::isfinite(delta[i])) return fail(NCL_ERR_INVALID_ARG, "delta must be finite");
  }
  if ((h->dp.nnzH && !Hv) || (h->dp.nnzJ && !Jv) || (h->dp.nvar && !S))
    return fail(NCL_ERR_INVALID_ARG, "NULL value array");
  h->factored = false;
  double* hp = h->h_pinned;
  for (int i = 0; i < ni; i++) {
    hp[i] = delta[i];
    hp[ni + i] = rho[i];
  }
  const double** vp = reinterpret_cast<const double**>(hp + 2 * ni + 4 * ni + 1 + ni);
  vp[0] = Hv;
  vp[1] = Jv;
  vp[2] = S;
  vp[3] = Ss;
  CK(cudaEventRecord(h->ev0, st));
  CK(cudaMemcpyAsync(h->d_delta, hp, ni * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_rho, hp + ni, ni * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_valptr, vp, 4 * sizeof(double*), cudaMemcpyHostToDevice, st));
  if (h->Jcopy && h->dp.nnzJ)
    CK(cudaMemcpyAsync(h->Jcopy, Jv, h->dp.nnzJ * sizeof(double), cudaMemcpyDeviceToDevice, st));
  h->h_delta.assign(delta, delta + ni);
  h->h_rho.assign(rho, rho + ni);
  return NCL_OK;
}

// the FP64 values of the matrix (K2r blocks or H + Sigma + delta I +
// rho J^T W J) from the user's arrays, on stream s2
void enqueue_values(ncl_kkt_s* h, cudaStream_t s2) {
  if (!h->skip_values) {
    const double np = (double)h->plan.pair_p.size();
    if (h->dp.form == 1 && h->dp.ncon > 0)
      klaunch(h, s2, "row_weights_f64", h->dp.ncon, Cost{4.0 * h->dp.ncon, 48.0 * h->dp.ncon},
              [&] { launch_row_weights(h->dp, h->d_valptr, h->d_rho, h->d_w, h->d_dw, h->d_ss, s2); });
    klaunch(h, s2, "kkt_values_f64", h->dp.nnzA,
            Cost{2.0 * np, 33.0 * h->dp.nnzA + 24.0 * np + 8.0 * (h->dp.nnzH + h->dp.nnzJ + h->dp.nvar)},
            [&] { launch_kkt_values(h->dp, h->d_valptr, h->d_delta, h->d_rho, h->d_w, h->Klow, s2); });
  }
}

// all device work of a factorisation, on stream s2 (capturable)
void enqueue_factor(ncl_kkt_s* h, cudaStream_t s2) {
  const int ni = h->dp.ninst;
  enqueue_values(h, s2);
  CK(cudaMemsetAsync(h->d_knorm, 0, ni * sizeof(unsigned long long), s2));
  const int64_t nnzF = (int64_t)h->plan.F_col.size();
  klaunch(h, s2, "full_values_f64", nnzF, Cost{0, 20.0 * (double)nnzF},
          [&] { launch_full_values(h->dp, h->Klow, h->Kf, nnzF, s2); });
  klaunch(h, s2, "knorm_f64", h->dp.dim, Cost{0, 8.0 * (double)nnzF + 8.0 * h->dp.dim},
          [&] { launch_knorm(h->dp, h->Kf, h->d_knorm, s2); });
  CK(cudaMemsetAsync(h->d_counts, 0, (4 * ni + 1) * sizeof(long long), s2));
  CK(cudaMemsetAsync(h->d_err, 0, 4 * sizeof(int), s2));
  CK(cudaMemsetAsync(h->d_panel_sync, 0, std::max<int64_t>(h->hs.panel_sync, 8) * sizeof(int), s2));
  CK(cudaMemsetAsync(h->d_dag_cnt, 0, (h->hs.dag_counters + 1) * sizeof(int), s2));
  if (is_fp32(h)) {
    run_factor<float>(h, h->nf, s2);
    klaunch(h, s2, "inertia", h->dp.dim, Cost{0, 5.0 * h->dp.dim},
            [&] { launch_inertia<float>(h->dp, h->nf, h->d_counts, s2); });
  } else {
    run_factor<double>(h, h->nd, s2);
    klaunch(h, s2, "inertia", h->dp.dim, Cost{0, 9.0 * h->dp.dim},
            [&] { launch_inertia<double>(h->dp, h->nd, h->d_counts, s2); });
  }
}

// read back inertia, norms and the error flag; fill the infos
ncl_status finish_factor(ncl_kkt_s* h, cudaStream_t st, ncl_kkt_factor_info* infos) {
  const int ni = h->dp.ninst;
  double* hp = h->h_pinned;
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev1, st));
  long long* hc = reinterpret_cast<long long*>(hp + 2 * ni);
  CK(cudaMemcpyAsync(hc, h->d_counts, (4 * ni + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st));
  unsigned long long* hk = reinterpret_cast<unsigned long long*>(hp + 2 * ni + 4 * ni + 1);
  CK(cudaMemcpyAsync(hk, h->d_knorm, ni * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  int* herr = reinterpret_cast<int*>(hp + 7 * ni + 8);
  CK(cudaMemcpyAsync(herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*herr) {
    h->factored = false;
    return fail(NCL_ERR_TIMEOUT, "a bounded device wait of the factorisation (macro panel or tensor-core update) ran out");
  }
  prof_collect(h);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->knorm_host.resize(ni);
  for (int i = 0; i < ni; i++) std::memcpy(&h->knorm_host[i], &hk[i], 8);
  ncl_status stt = NCL_OK;
  if (hc[4 * ni] > 0) stt = fail(NCL_ERR_NUMERIC, "non-finite pivot");
  for (int i = 0; i < ni; i++) {
    if (infos) {
      ncl_kkt_factor_info& f = infos[i];
      f.n_pos = hc[4 * i];
      f.n_neg = hc[4 * i + 1];
      f.n_zero = hc[4 * i + 2];
      f.n_perturbed = hc[4 * i + 3];
      f.nnz_L = h->plan.inst_nnzL[i];
      f.flops = h->plan.inst_flops[i];
      f.ms = ms;
    }
    if (stt == NCL_OK && h->opt.pivot_policy == NCL_PIVOT_STOP && hc[4 * i + 2] > 0)
      stt = fail(NCL_ERR_ZERO_PIVOT, "zero pivot under the stop policy");
  }
  h->factored = (stt == NCL_OK || stt == NCL_ERR_ZERO_PIVOT);
  return stt;
}

void build_schedule(ncl_kkt_s* h);
void build_device(ncl_kkt_s* h);

// does the factor's inertia match the form's regular one for every instance?
bool inertia_regular(ncl_kkt_s* h) {
  const int ni = h->dp.ninst;
  const long long* hc = reinterpret_cast<const long long*>(h->h_pinned + 2 * ni);
  for (int i = 0; i < ni; i++) {
    const Instance& I = h->plan.inst[i];
    const long long np = hc[4 * i], nn = hc[4 * i + 1], nz = hc[4 * i + 2];
    const long long want_neg = h->plan.form == 0 ? I.m : 0;
    if (np != I.n || nn != want_neg || nz != 0) return false;
  }
  return true;
}

// which instances' inertia is not the regular one (after finish_factor)
std::vector<char> irregular_instances(ncl_kkt_s* h) {
  const int ni = h->dp.ninst;
  const long long* hc = reinterpret_cast<const long long*>(h->h_pinned + 2 * ni);
  std::vector<char> out(ni, 0);
  for (int i = 0; i < ni; i++) {
    const Instance& I = h->plan.inst[i];
    const long long want_neg = h->plan.form == 0 ? I.m : 0;
    out[i] = !(hc[4 * i] == I.n && hc[4 * i + 1] == want_neg && hc[4 * i + 2] == 0);
  }
  return out;
}

// refactor the parent's FP64 values in FP64 on the twin handle
ncl_status escalate(ncl_kkt_s* h, cudaStream_t st, ncl_kkt_factor_info* infos) {
  if (!h->twin) {
    std::unique_ptr<ncl_kkt_s> t(new ncl_kkt_s());
    t->plan = h->plan;
    t->opt = h->opt;
    t->opt.prec = NCL_PREC_FP64;
    t->opt.ir_tol = h->opt.ir_tol;
    t->opt.precision_fallback = 0;
    t->device = h->device;
    t->ninst = h->ninst;
    t->dp.ninst = h->dp.ninst;
    t->skip_values = true;
    build_schedule(t.get());
    build_device(t.get());
    h->twin = t.release();
  }
  ncl_kkt_s* t = h->twin;
  const int ni = h->dp.ninst;
  CK(cudaEventRecord(t->ev0, st));
  CK(cudaMemcpyAsync(t->Klow, h->Klow, h->dp.nnzA * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(t->d_delta, h->d_delta, ni * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(t->d_rho, h->d_rho, ni * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (t->Jcopy && h->Jcopy && h->dp.nnzJ)
    CK(cudaMemcpyAsync(t->Jcopy, h->Jcopy, h->dp.nnzJ * sizeof(double), cudaMemcpyDeviceToDevice, st));
  t->h_delta = h->h_delta;
  t->h_rho = h->h_rho;
  run_graphed(t, &t->fgraph, &t->fgraph_nodes, &t->factor_calls, true, st,
              [&](cudaStream_t s2) { enqueue_factor(t, s2); });
  ncl_status s = finish_factor(t, st, infos);
  if (infos)
    for (int i = 0; i < ni; i++) infos[i].fp64_fallback = 1;
  h->use_twin = t->factored;
  return s;
}

// the FP32 factors of the values just factored were not trusted (irregular
// inertia, or refinement short of ir_tol) while the FP64 ones are regular:
// remember the penalty of every instance (of the irregular ones only, when
// the inertia told which)
void note_fp32_failure(ncl_kkt_s* h, const std::vector<char>* which) {
  if (h->opt.precision_fallback != 1 || !h->twin || !h->use_twin || !inertia_regular(h->twin)) return;
  const int ni = h->dp.ninst;
  if ((int)h->fp32_fail_rho.size() != ni) h->fp32_fail_rho.assign(ni, HUGE_VAL);
  for (int i = 0; i < ni; i++)
    if (!which || (*which)[i]) h->fp32_fail_rho[i] = std::min(h->fp32_fail_rho[i], h->h_rho[i]);
}

// start this factorisation directly in FP64? (an instance's penalty is at
// least one at which its FP32 factors were already replaced)
bool skip_fp32(const ncl_kkt_s* h, const double* rho) {
  if (!is_fp32(h) || h->opt.precision_fallback != 1 || (int)h->fp32_fail_rho.size() != h->dp.ninst) return false;
  for (int i = 0; i < h->dp.ninst; i++)
    if (rho[i] >= h->fp32_fail_rho[i]) return true;
  return false;
}

// the FP64 factorisation straight away: values on this handle, factors on
// the twin; the infos say fp64_fallback = 2
ncl_status factor_fp64_direct(ncl_kkt_s* h, cudaStream_t st, ncl_kkt_factor_info* infos) {
  enqueue_values(h, st);
  const ncl_status s = escalate(h, st, infos);
  if (infos)
    for (int i = 0; i < h->dp.ninst; i++) infos[i].fp64_fallback = 2;
  return s;
}

ncl_status do_factor(ncl_kkt_s* h, const double* Hv, const double* Jv, const double* S, const double* delta,
                     const double* rho, cudaStream_t st, ncl_kkt_factor_info* infos, const double* Ss = nullptr) {
  h->use_twin = false;
  ncl_status s0 = prepare_factor(h, Hv, Jv, S, delta, rho, st, Ss);
  if (s0 != NCL_OK) return s0;
  if (skip_fp32(h, rho)) return factor_fp64_direct(h, st, infos);
  run_graphed(h, &h->fgraph, &h->fgraph_nodes, &h->factor_calls, true, st,
              [&](cudaStream_t s2) { enqueue_factor(h, s2); });
  ncl_status s1 = finish_factor(h, st, infos);
  if (infos)
    for (int i = 0; i < h->dp.ninst; i++) infos[i].fp64_fallback = 0;
  if (is_fp32(h) && h->opt.precision_fallback && (s1 == NCL_OK || s1 == NCL_ERR_NUMERIC) && !inertia_regular(h)) {
    const std::vector<char> irr = irregular_instances(h);
    const ncl_status se = escalate(h, st, infos);
    note_fp32_failure(h, &irr);
    return se;
  }
  return s1;
}

// factor + solve of nrhs <= 8 columns + a fixed number of refinement steps
// as one captured graph (after a direct first call that learns how many
// refinement steps the systems need); the host checks the backward error
// afterwards and refines further only if needed
// did a bounded wait of the pivot-block sweeps run out since the factor?
bool sweep_failed(ncl_kkt_s* h, cudaStream_t st) {
  int* he = reinterpret_cast<int*>(h->h_pinned + 7 * h->dp.ninst + 9);
  CK(cudaMemcpyAsync(he, h->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return *he != 0;
}

ncl_status do_factor_solve(ncl_kkt_s* h, const double* Hv, const double* Jv, const double* S, const double* delta,
                           const double* rho, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                           cudaStream_t st, ncl_kkt_factor_info* infos, ncl_kkt_solve_info* sinfo) {
  const int ni = h->dp.ninst;
  const bool same_key = h->fs_key[0] == B && h->fs_key[1] == X && h->fs_keyi[0] == ldb && h->fs_keyi[1] == ldx &&
                        h->fs_keyi[2] == nrhs;
  if (!same_key && h->fsgraph) {
    cudaGraphExecDestroy(h->fsgraph);
    h->fsgraph = nullptr;
    h->fs_calls = 0;
  }
  h->fs_key[0] = B;
  h->fs_key[1] = X;
  h->fs_keyi[0] = ldb;
  h->fs_keyi[1] = ldx;
  h->fs_keyi[2] = nrhs;
  const bool direct64 = skip_fp32(h, rho);
  if (h->fs_calls == 0 || h->prof_on || direct64) {
    // direct: the regular calls, which also tell how many steps are needed
    // (not those of an FP64 factorisation started directly)
    ncl_status s1 = do_factor(h, Hv, Jv, S, delta, rho, st, infos);
    if (s1 != NCL_OK && s1 != NCL_ERR_ZERO_PIVOT) return s1;
    ncl_status s2 = do_solve(h, nrhs, B, ldb, X, ldx, st, sinfo);
    if (!h->prof_on && !direct64 && !(sinfo && sinfo->fp64_fallback)) {
      h->fs_calls = 1;
      h->fs_nir = sinfo ? sinfo->ir_iters : h->opt.ir_max_iter;
      if (sinfo && sinfo->used_fgmres) h->fs_nir = 0;
    }
    return s2 != NCL_OK ? s2 : s1;
  }
  ncl_status s0 = prepare_factor(h, Hv, Jv, S, delta, rho, st);
  if (s0 != NCL_OK) return s0;
  if (sinfo) *sinfo = ncl_kkt_solve_info{};
  unsigned long long* hn = reinterpret_cast<unsigned long long*>(h->h_pinned + 7 * ni + 64);
  const int nir = h->fs_nir;
  auto body = [&](cudaStream_t s2) {
    enqueue_factor(h, s2);
    CK(cudaMemsetAsync(h->d_norms, 0, 3 * (size_t)ni * MAX_RHS_SWEEP * sizeof(unsigned long long), s2));
    klaunch(h, s2, "vec_norm", h->dp.dim, Cost{0, 8.0 * h->dp.dim * nrhs},
            [&] { launch_vec_norm(h->dp, B, ldb, nrhs, h->d_norms + 2 * ni * MAX_RHS_SWEEP, s2); });
    apply_inverse(h, B, ldb, X, ldx, nrhs, 0, s2);
    for (int k = 0; k <= nir; k++) {
      CK(cudaMemsetAsync(h->d_norms, 0, 2 * (size_t)ni * MAX_RHS_SWEEP * sizeof(unsigned long long), s2));
      const double nnzF = (double)h->plan.F_col.size();
      klaunch(h, s2, "residual_f64", h->dp.dim, Cost{2.0 * nnzF * nrhs, nnzF * 16.0}, [&] {
        launch_residual(h->dp, h->Kf, B, ldb, X, ldx, h->R, h->dp.dim, nrhs, h->d_norms,
                        h->d_norms + ni * MAX_RHS_SWEEP, s2);
      });
      if (k < nir) apply_inverse(h, h->R, h->dp.dim, X, ldx, nrhs, 1, s2);
    }
    CK(cudaMemcpyAsync(hn, h->d_norms, 3 * (size_t)ni * MAX_RHS_SWEEP * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s2));
  };
  h->use_twin = false;
  run_graphed(h, &h->fsgraph, &h->fsgraph_nodes, &h->fs_calls, true, st, body);
  ncl_status sf = finish_factor(h, st, infos);
  if (infos)
    for (int i = 0; i < ni; i++) infos[i].fp64_fallback = 0;
  if (is_fp32(h) && h->opt.precision_fallback && (sf == NCL_OK || sf == NCL_ERR_NUMERIC) && !inertia_regular(h)) {
    const std::vector<char> irr = irregular_instances(h);
    ncl_status se = escalate(h, st, infos);
    note_fp32_failure(h, &irr);
    if (se != NCL_OK && se != NCL_ERR_ZERO_PIVOT) return se;
    ncl_status s2 = do_solve(h, nrhs, B, ldb, X, ldx, st, sinfo);
    return s2 != NCL_OK ? s2 : se;
  }
  if (sf != NCL_OK && sf != NCL_ERR_ZERO_PIVOT) return sf;
  const double eta = backward_errors(h, nrhs, st, nullptr, hn);
  ncl_status sr = NCL_OK;
  if (!(eta <= h->opt.ir_tol)) sr = refine_block(h, nrhs, B, ldb, X, ldx, st, sinfo, eta, nir);
  else if (sinfo) {
    sinfo->ir_iters = nir;
    sinfo->backward_err = eta;
  }
  if (sr == NCL_ERR_IR_NOT_CONVERGED && is_fp32(h) && h->opt.precision_fallback) {
    ncl_status se = escalate(h, st, nullptr);
    note_fp32_failure(h, nullptr);
    if (se != NCL_OK && se != NCL_ERR_ZERO_PIVOT) return se;
    return do_solve(h, nrhs, B, ldb, X, ldx, st, sinfo);
  }
  CK(cudaEventRecord(h->ev1, st));
  CK(cudaEventSynchronize(h->ev1));
  if (sinfo) cudaEventElapsedTime(&sinfo->ms, h->ev0, h->ev1);
  if (sweep_failed(h, st)) return fail(NCL_ERR_TIMEOUT, "a bounded device wait of the triangular sweeps ran out");
  if (sr == NCL_ERR_IR_NOT_CONVERGED) g_last_error = "iterative refinement did not reach ir_tol";
  return sr != NCL_OK ? sr : sf;
}

ncl_status do_solve(ncl_kkt_s* h, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                    cudaStream_t st, ncl_kkt_solve_info* info, bool allow_escalate) {
  if (h->use_twin) {
    ncl_status s = do_solve(h->twin, nrhs, B, ldb, X, ldx, st, info, false);
    if (info) info->fp64_fallback = 1;
    return s;
  }
  if (!h->factored) return fail(NCL_ERR_STATE, "solve before a successful factor");
  if (nrhs < 0 || (nrhs > 0 && (!B || !X)) || ldb < h->dp.dim || ldx < h->dp.dim)
    return fail(NCL_ERR_INVALID_ARG, "bad right-hand side block");
  if (info) *info = ncl_kkt_solve_info{};
  // the sweeps' error flag reports on this solve only
  CK(cudaMemsetAsync(h->d_err + 1, 0, sizeof(int), st));
  CK(cudaEventRecord(h->ev0, st));
  ncl_status worst = NCL_OK;
  for (int r0 = 0; r0 < nrhs; r0 += MAX_RHS_SWEEP) {
    const int nr = std::min(MAX_RHS_SWEEP, nrhs - r0);
    ncl_status s = solve_block(h, nr, B + r0 * ldb, ldb, X + r0 * ldx, ldx, st, info);
    if (s != NCL_OK && worst == NCL_OK) worst = s;
  }
  CK(cudaEventRecord(h->ev1, st));
  CK(cudaEventSynchronize(h->ev1));
  prof_collect(h);
  if (info) cudaEventElapsedTime(&info->ms, h->ev0, h->ev1);
  if (sweep_failed(h, st)) return fail(NCL_ERR_TIMEOUT, "a bounded device wait of the triangular sweeps ran out");
  if (worst == NCL_ERR_IR_NOT_CONVERGED && allow_escalate && is_fp32(h) && h->opt.precision_fallback) {
    // the FP32 factors cannot reach the tolerance: refactor in FP64, solve again
    ncl_status se = escalate(h, st, nullptr);
    note_fp32_failure(h, nullptr);
    if (se != NCL_OK && se != NCL_ERR_ZERO_PIVOT) return se;
    return do_solve(h, nrhs, B, ldb, X, ldx, st, info, false);
  }
  if (worst == NCL_ERR_IR_NOT_CONVERGED) g_last_error = "iterative refinement did not reach ir_tol";
  return worst;
}

template <typename F>
ncl_status guarded(ncl_kkt_s* h, F&& f) {
  try {
    int cur = 0;
    cudaGetDevice(&cur);
    if (h && cur != h->device) cudaSetDevice(h->device);
    ncl_status s = f();
    if (h && cur != h->device) cudaSetDevice(cur);
    return s;
  } catch (const CudaError& e) {
    return fail(NCL_ERR_CUDA, e.where + ": " + cudaGetErrorString(e.err));
  } catch (const std::bad_alloc&) {
    return fail(NCL_ERR_OOM, "device or host allocation failed");
  } catch (const std::exception& e) {
    return fail(NCL_ERR_INVALID_ARG, e.what());
  }
}

// options of a new handle, validated, with the precision-dependent defaults
static ncl_status init_options(ncl_kkt_s* h, const ncl_kkt_options* opt) {
  ncl_kkt_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (h->opt.prec != NCL_PREC_FP64 && h->opt.prec != NCL_PREC_FP32_IR) return fail(NCL_ERR_INVALID_ARG, "bad prec");
  if (h->opt.pivot_policy != NCL_PIVOT_PERTURB && h->opt.pivot_policy != NCL_PIVOT_STOP)
    return fail(NCL_ERR_INVALID_ARG, "bad pivot policy");
  if (!(h->opt.pivot_eps >= 0)) return fail(NCL_ERR_INVALID_ARG, "bad pivot_eps");
  if (!(h->opt.ir_tol > 0)) h->opt.ir_tol = h->opt.prec == NCL_PREC_FP64 ? 1e-12 : 1e-10;
  if (h->opt.ir_max_iter < 0) h->opt.ir_max_iter = h->opt.prec == NCL_PREC_FP64 ? 3 : 10;
  if (h->opt.wait_cycles <= 0) h->opt.wait_cycles = DEFAULT_WAIT_CYCLES;
  if (!(h->opt.ir_switch > 0.0) || !(h->opt.ir_switch <= 1.0)) h->opt.ir_switch = 0.5;
  if (h->opt.tc_min_pivots < 32) return fail(NCL_ERR_INVALID_ARG, "tc_min_pivots must be >= 32");
  if (h->opt.precision_fallback < 0 || h->opt.precision_fallback > 2)
    return fail(NCL_ERR_INVALID_ARG, "precision_fallback must be 0, 1 or 2");
  return NCL_OK;
}

// The cut-overs of a tuned table (written by the autotuner): the first line
// whose form, dimension range and instance-count range match the analysis
// sets persistent_fronts, subtree_sweeps, use_tensor_cores and
// tc_min_pivots.  Lines: form dim_lo dim_hi count_lo count_hi persistent
// subtree tensor_cores tc_min_pivots [comment]; '#' starts a comment line.
static ncl_status apply_tuned(ncl_kkt_s* h) {
  const char* path = h->opt.autotune_path;
  h->opt.autotune_path = nullptr;   // the caller's string is not kept
  if (!path) return NCL_OK;
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(NCL_ERR_INVALID_ARG, std::string("cannot read the tuned table ") + path);
  char line[512];
  ncl_status st = NCL_OK;
  int lineno = 0;
  while (std::fgets(line, sizeof(line), f)) {
    lineno++;
    const char* q = line;
    while (*q == ' ' || *q == '\t') q++;
    if (*q == '#' || *q == '\n' || *q == '\0') continue;
    long long v[9];
    if (std::sscanf(q, "%lld %lld %lld %lld %lld %lld %lld %lld %lld", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                    &v[7], &v[8]) != 9 ||
        v[5] < 0 || v[5] > 1 || v[6] < 0 || v[6] > 1 || v[7] < 0 || v[7] > 2 || v[8] < 32) {
      st = fail(NCL_ERR_INVALID_ARG, std::string("bad line ") + std::to_string(lineno) + " in the tuned table");
      break;
    }
    const int64_t cnt = (int64_t)h->plan.inst.size();
    if (v[0] == h->plan.form && h->plan.dim >= v[1] && h->plan.dim < v[2] && cnt >= v[3] && cnt <= v[4]) {
      h->opt.persistent_fronts = (int32_t)v[5];
      h->opt.subtree_sweeps = (int32_t)v[6];
      h->opt.use_tensor_cores = (int32_t)v[7];
      h->opt.tc_min_pivots = (int32_t)v[8];
      break;
    }
  }
  std::fclose(f);
  return st;
}

static ncl_status finish_handle(std::unique_ptr<ncl_kkt_s>& h, ncl_kkt_t* out);

ncl_status analyze_common(const AnalyzeInput& in, const ncl_kkt_options* opt, ncl_kkt_t* out) {
  if (!out) return fail(NCL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (in.form != 0 && in.form != 1) return fail(NCL_ERR_INVALID_ARG, "bad form");
  std::unique_ptr<ncl_kkt_s> h(new ncl_kkt_s());
  ncl_status so = init_options(h.get(), opt);
  if (so != NCL_OK) return so;
  AnalyzeInput a = in;
  a.leaf_size = h->opt.leaf_size;
  a.colpad = 4;
  std::string err = analyze(a, h->plan);
  if (!err.empty()) {
    if (err.rfind("pattern", 0) == 0) return fail(NCL_ERR_PATTERN, err);
    if (err.rfind("oom", 0) == 0) return fail(NCL_ERR_OOM, err);
    return fail(NCL_ERR_INVALID_ARG, err);
  }
  h->ninst = in.count;
  h->dp.ninst = in.count;
  ncl_status sa = apply_tuned(h.get());
  if (sa != NCL_OK) return sa;
  return finish_handle(h, out);
}

// A handle with new options on the analysis of an existing one (the plan is
// copied; the nested-dissection leaf size of the new options is not used).
ncl_status analyze_like(ncl_kkt_s* src, const ncl_kkt_options* opt, ncl_kkt_t* out) {
  if (!out) return fail(NCL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!src) return fail(NCL_ERR_INVALID_ARG, "NULL source handle");
  std::unique_ptr<ncl_kkt_s> h(new ncl_kkt_s());
  ncl_status so = init_options(h.get(), opt);
  if (so != NCL_OK) return so;
  h->plan = src->plan;
  h->ninst = src->ninst;
  h->dp.ninst = src->dp.ninst;
  ncl_status sa = apply_tuned(h.get());
  if (sa != NCL_OK) return sa;
  return finish_handle(h, out);
}

static ncl_status finish_handle(std::unique_ptr<ncl_kkt_s>& h, ncl_kkt_t* out) {
  try {
    build_schedule(h.get());
  } catch (const std::exception& e) {
    return fail(NCL_ERR_INVALID_ARG, e.what());
  }
  if (h->opt.host_only) {
    *out = h.release();
    return NCL_OK;
  }
  cudaGetDevice(&h->device);
  ncl_kkt_s* raw = h.get();
  ncl_status s = guarded(raw, [&] {
    build_device(raw);
    return NCL_OK;
  });
  if (s != NCL_OK) return s;
  *out = h.release();
  return NCL_OK;
}

}  // namespace

extern "C" {

void ncl_kkt_default_options(ncl_kkt_options* o) {
  if (!o) return;
  o->prec = NCL_PREC_FP32_IR;
  o->pivot_policy = NCL_PIVOT_PERTURB;
  o->pivot_eps = 1e-10;
  o->ir_tol = 0.0;
  o->ir_max_iter = -1;
  o->use_fgmres = 1;
  o->use_tensor_cores = 2;
  o->leaf_size = 96;
  o->host_only = 0;
  o->precision_fallback = 1;
  o->max_device_bytes = 0;
  o->wait_cycles = 0;
  o->persistent_fronts = 0;
  o->ir_switch = 0.5;
  o->subtree_sweeps = 1;
  o->tc_min_pivots = 256;
  o->autotune_path = nullptr;
}

ncl_status ncl_kkt_analyze(int32_t form, int32_t n, int32_t m, const int32_t* H_rowptr, const int32_t* H_colind,
                           const int32_t* J_rowptr, const int32_t* J_colind, const ncl_kkt_options* opt,
                           ncl_kkt_t* out) {
  if (n < 0 || m < 0) return fail(NCL_ERR_INVALID_ARG, "negative size");
  if ((n > 0 && !H_rowptr) || (m > 0 && !J_rowptr)) return fail(NCL_ERR_INVALID_ARG, "NULL pattern");
  AnalyzeInput in{};
  in.form = form;
  in.count = 1;
  in.n = &n;
  in.m = &m;
  in.H_rowptr = &H_rowptr;
  in.H_colind = &H_colind;
  in.J_rowptr = &J_rowptr;
  in.J_colind = &J_colind;
  return analyze_common(in, opt, out);
}

ncl_status ncl_kkt_analyze_like(ncl_kkt_t src, const ncl_kkt_options* opt, ncl_kkt_t* out) {
  return analyze_like(src, opt, out);
}

ncl_status ncl_kkt_batch_analyze(int32_t count, int32_t form, const int32_t* n, const int32_t* m,
                                 const int32_t* const* H_rowptr, const int32_t* const* H_colind,
                                 const int32_t* const* J_rowptr, const int32_t* const* J_colind,
                                 const ncl_kkt_options* opt, ncl_kkt_t* out) {
  if (count <= 0 || !n || !m || !H_rowptr || !H_colind || !J_rowptr || !J_colind)
    return fail(NCL_ERR_INVALID_ARG, "bad batch arguments");
  AnalyzeInput in{};
  in.form = form;
  in.count = count;
  in.n = n;
  in.m = m;
  in.H_rowptr = H_rowptr;
  in.H_colind = H_colind;
  in.J_rowptr = J_rowptr;
  in.J_colind = J_colind;
  return analyze_common(in, opt, out);
}

ncl_status ncl_kkt_factor(ncl_kkt_t h, const double* H_val, const double* J_val, const double* Sigma, double delta,
                          double rho, ncl_stream_t stream, ncl_kkt_factor_info* info) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (h->dp.ninst != 1) return fail(NCL_ERR_INVALID_ARG, "batch handle: use ncl_kkt_batch_factor");
  return guarded(h, [&] { return do_factor(h, H_val, J_val, Sigma, &delta, &rho, (cudaStream_t)stream, info); });
}

ncl_status ncl_kkt_batch_factor(ncl_kkt_t h, const double* H_val, const double* J_val, const double* Sigma,
                                const double* delta, const double* rho, ncl_stream_t stream,
                                ncl_kkt_factor_info* infos) {
  if (!h || !delta || !rho) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  return guarded(h, [&] { return do_factor(h, H_val, J_val, Sigma, delta, rho, (cudaStream_t)stream, infos); });
}

// The condensed form with slacks, Eq. K1s: the condensed factorisation with
// row weights rho Omega_r, Omega_r = Sigma_s,r / (rho + Sigma_s,r), from the
// caller's slack terms (+inf for a row without slack).
ncl_status ncl_kkt_factor_k1s(ncl_kkt_t h, const double* H_val, const double* J_val, const double* Sigma,
                              const double* Sigma_s, const double* delta, const double* rho, ncl_stream_t stream,
                              ncl_kkt_factor_info* infos) {
  if (!h || !delta || !rho) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (h->plan.form != 1) return fail(NCL_ERR_INVALID_ARG, "the slack form needs a condensed handle");
  if (h->dp.ncon > 0 && !Sigma_s) return fail(NCL_ERR_INVALID_ARG, "NULL Sigma_s");
  return guarded(h, [&] {
    return do_factor(h, H_val, J_val, Sigma, delta, rho, (cudaStream_t)stream, infos, Sigma_s);
  });
}

// Newton step around the factorisation: right-hand side of Eq. K2r / K1 and
// the recovery of Delta y, Delta r, Delta z_l, Delta z_u (Section 3.1-3.3).
static ncl_status newton_args(ncl_kkt_s* h, const ncl_kkt_newton_point* pt, const double* mu, NewtonDev* nd,
                              cudaStream_t st) {
  if (!h || !pt || !mu) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (!h->factored && !h->use_twin) return fail(NCL_ERR_STATE, "Newton step before a successful factor");
  const bool nv = h->dp.nvar > 0, nc = h->dp.ncon > 0;
  if (nv && (!pt->grad_phi || !pt->x || !pt->lower || !pt->upper || !pt->z_lower || !pt->z_upper))
    return fail(NCL_ERR_INVALID_ARG, "NULL n-vector of the Newton point");
  if (nc && (!pt->c || !pt->y || !pt->y_k || !pt->r)) return fail(NCL_ERR_INVALID_ARG, "NULL m-vector of the Newton point");
  const int ni = h->dp.ninst;
  for (int i = 0; i < ni; i++)
    if (!(mu[i] >= 0.0) || !std::isfinite(mu[i])) return fail(NCL_ERR_INVALID_ARG, "mu must be >= 0");
  double* hm = h->h_pinned + 7 * ni + 32;   // free slots of the pinned block (below the norms at 7 ni + 64)
  if (ni > 32) {
    std::vector<double> tmp(mu, mu + ni);
    CK(cudaMemcpy(h->d_mu, tmp.data(), ni * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    for (int i = 0; i < ni; i++) hm[i] = mu[i];
    CK(cudaMemcpyAsync(h->d_mu, hm, ni * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  *nd = NewtonDev{pt->grad_phi, pt->x, pt->lower, pt->upper, pt->z_lower, pt->z_upper, pt->c, pt->y, pt->y_k, pt->r};
  return NCL_OK;
}

ncl_status ncl_kkt_newton_rhs(ncl_kkt_t h, const ncl_kkt_newton_point* pt, const double* mu, double* B,
                              ncl_stream_t stream) {
  if (!B) return fail(NCL_ERR_INVALID_ARG, "NULL B");
  return guarded(h, [&]() -> ncl_status {
    NewtonDev nd;
    const cudaStream_t st = (cudaStream_t)stream;
    ncl_status s = newton_args(h, pt, mu, &nd, st);
    if (s != NCL_OK) return s;
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    launch_newton_rhs(h->dp, h->Jcopy, h->d_rho, h->d_mu, nd, B, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));   // the pinned mu slots are reused by the next call
    return NCL_OK;
  });
}

ncl_status ncl_kkt_newton_recover(ncl_kkt_t h, const ncl_kkt_newton_point* pt, const double* mu, const double* X,
                                  double* dx, double* dy, double* dr, double* dz_lower, double* dz_upper,
                                  ncl_stream_t stream) {
  if (!X) return fail(NCL_ERR_INVALID_ARG, "NULL X");
  return guarded(h, [&]() -> ncl_status {
    NewtonDev nd;
    const cudaStream_t st = (cudaStream_t)stream;
    ncl_status s = newton_args(h, pt, mu, &nd, st);
    if (s != NCL_OK) return s;
    g_kernel_launches.fetch_add(2, std::memory_order_relaxed);
    launch_newton_recover(h->dp, h->Jcopy, h->d_rho, h->d_mu, nd, X, dx, dy, dr, dz_lower, dz_upper, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return NCL_OK;
  });
}

// Right-hand side of Eq. K1s for the current condensed factorisation.
ncl_status ncl_kkt_k1s_rhs(ncl_kkt_t h, int32_t nrhs, const double* RT, int64_t ldt, const double* RS, int64_t ldr,
                           double* OUT, int64_t ldo, ncl_stream_t stream) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (h->plan.form != 1) return fail(NCL_ERR_INVALID_ARG, "the slack form needs a condensed handle");
  if (!h->factored && !h->use_twin) return fail(NCL_ERR_STATE, "right-hand side before a successful factor");
  const int64_t ncon = h->dp.ncon;
  if (nrhs <= 0 || !RT || !OUT || (ncon > 0 && !RS) || ldt < h->dp.dim || ldo < h->dp.dim || ldr < ncon)
    return fail(NCL_ERR_INVALID_ARG, "bad right-hand-side arguments");
  return guarded(h, [&]() -> ncl_status {
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    launch_k1s_rhs(h->dp, h->Jcopy, h->d_rho, h->d_ss, nrhs, RT, ldt, RS, ldr, OUT, ldo, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NCL_OK;
  });
}

// Slack recovery of Eq. K1s for the current condensed factorisation.
ncl_status ncl_kkt_k1s_slack_step(ncl_kkt_t h, int32_t nrhs, const double* DT, int64_t ldt, const double* RS,
                                  int64_t ldr, double* DS, int64_t lds, ncl_stream_t stream) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (h->plan.form != 1) return fail(NCL_ERR_INVALID_ARG, "the slack step needs a condensed handle");
  if (!h->factored && !h->use_twin) return fail(NCL_ERR_STATE, "slack step before a successful factor");
  const int64_t ncon = h->dp.ncon;
  if (nrhs <= 0 || (ncon > 0 && (!DT || !RS || !DS)) || ldt < h->dp.dim || ldr < ncon || lds < ncon)
    return fail(NCL_ERR_INVALID_ARG, "bad slack-step arguments");
  return guarded(h, [&]() -> ncl_status {
    if (ncon == 0) return NCL_OK;
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    launch_slack_step(h->dp, h->Jcopy, h->d_rho, h->d_ss, nrhs, DT, ldt, RS, ldr, DS, lds, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NCL_OK;
  });
}

// The inertia correction of Section 3.1: raise the primal regularisation of
// every instance whose inertia is irregular and refactor, rho-hat = rho +
// delta entering the matrix with it.
ncl_status ncl_kkt_factor_regularize(ncl_kkt_t h, const double* H_val, const double* J_val, const double* Sigma,
                                     double* delta, const double* rho, double delta_first, double growth,
                                     int32_t max_tries, ncl_stream_t stream, ncl_kkt_factor_info* infos,
                                     int32_t* tries) {
  if (!h || !delta || !rho) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (!(delta_first > 0.0) || !std::isfinite(delta_first) || !(growth > 1.0) || !std::isfinite(growth) ||
      max_tries < 1)
    return fail(NCL_ERR_INVALID_ARG, "bad regularisation schedule");
  const int ni = h->dp.ninst;
  for (int i = 0; i < ni; i++) {
    if (!(delta[i] >= 0.0) || !std::isfinite(delta[i])) return fail(NCL_ERR_INVALID_ARG, "delta must be >= 0");
    if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return fail(NCL_ERR_INVALID_ARG, "rho must be > 0");
  }
  if (tries) *tries = 0;
  std::vector<ncl_kkt_factor_info> own(ni);
  ncl_kkt_factor_info* inf = infos ? infos : own.data();
  return guarded(h, [&]() -> ncl_status {
    std::vector<double> rho_hat(ni), next(ni);
    for (int t = 1;; t++) {
      for (int i = 0; i < ni; i++) rho_hat[i] = rho[i] + delta[i];
      if (tries) *tries = t;
      const ncl_status s = do_factor(h, H_val, J_val, Sigma, delta, rho_hat.data(), (cudaStream_t)stream, inf);
      if (s != NCL_OK && s != NCL_ERR_ZERO_PIVOT) return s;
      bool regular = true;
      for (int i = 0; i < ni; i++) {
        const Instance& I = h->plan.inst[i];
        const int64_t want_neg = h->plan.form == 0 ? I.m : 0;
        const bool ok = inf[i].n_pos == I.n && inf[i].n_neg == want_neg && inf[i].n_zero == 0;
        next[i] = ok ? delta[i] : (delta[i] > 0.0 ? delta[i] * growth : delta_first);
        regular = regular && ok;
      }
      if (regular) return s;
      if (t >= max_tries) return fail(NCL_ERR_INERTIA, "inertia still irregular after max_tries factorisations");
      for (int i = 0; i < ni; i++) {
        if (!std::isfinite(next[i])) return fail(NCL_ERR_INERTIA, "the regularisation overflowed");
        delta[i] = next[i];
      }
    }
  });
}

ncl_status ncl_kkt_solve(ncl_kkt_t h, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                         ncl_stream_t stream, ncl_kkt_solve_info* info) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  return guarded(h, [&] { return do_solve(h, nrhs, B, ldb, X, ldx, (cudaStream_t)stream, info); });
}

ncl_status ncl_kkt_batch_factor_solve(ncl_kkt_t h, const double* H_val, const double* J_val, const double* Sigma,
                                      const double* delta, const double* rho, int32_t nrhs, const double* B,
                                      int64_t ldb, double* X, int64_t ldx, ncl_stream_t stream,
                                      ncl_kkt_factor_info* infos, ncl_kkt_solve_info* sinfo) {
  if (!h || !delta || !rho) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (nrhs <= 0 || !B || !X || ldb < h->dp.dim || ldx < h->dp.dim)
    return fail(NCL_ERR_INVALID_ARG, "bad right-hand side block");
  if (nrhs > MAX_RHS_SWEEP) {
    ncl_status s = ncl_kkt_batch_factor(h, H_val, J_val, Sigma, delta, rho, stream, infos);
    if (s != NCL_OK && s != NCL_ERR_ZERO_PIVOT) return s;
    ncl_status s2 = ncl_kkt_solve(h, nrhs, B, ldb, X, ldx, stream, sinfo);
    return s2 != NCL_OK ? s2 : s;
  }
  return guarded(h, [&] {
    return do_factor_solve(h, H_val, J_val, Sigma, delta, rho, nrhs, B, ldb, X, ldx, (cudaStream_t)stream, infos,
                           sinfo);
  });
}

ncl_status ncl_kkt_adjoint(ncl_kkt_t h, int32_t nrhs, const double* X, int64_t ldx, const double* GX, int64_t ldgx,
                           double* GB, int64_t ldgb, double* G_Hval, double* G_Jval, double* G_Sigma, double* G_scal,
                           ncl_stream_t stream, ncl_kkt_solve_info* info) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (!X || !GX || nrhs <= 0) return fail(NCL_ERR_INVALID_ARG, "bad adjoint arguments");
  return guarded(h, [&]() -> ncl_status {
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t dim = h->dp.dim;
    if (nrhs > MAX_RHS_SWEEP) return fail(NCL_ERR_INVALID_ARG, "adjoint supports at most 8 columns");
    double* gb = GB;
    int64_t ld = ldgb;
    if (!gb) {
      gb = h->GBtmp;
      ld = dim;
    }
    ncl_status s = do_solve(h, nrhs, GX, ldgx, gb, ld, st, info);
    if (s != NCL_OK && s != NCL_ERR_IR_NOT_CONVERGED) return s;
    g_kernel_launches.fetch_add(4, std::memory_order_relaxed);
    launch_adjoint_values(h->dp, h->Jcopy, h->d_w, X, ldx, gb, ld, nrhs, G_Hval, G_Jval, G_Sigma, G_scal,
                          h->jx, h->jg, st);
    if (G_scal) {
      launch_adjoint_scalars(h->dp, h->d_inst_n, h->d_inst_con_off, h->d_rho, h->d_dw, X, ldx, gb, ld, nrhs, h->jx, h->jg,
                             G_scal, st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return s;
  });
}

ncl_status ncl_kkt_get_options(ncl_kkt_t h, ncl_kkt_options* o) {
  if (!h || !o) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  *o = h->opt;
  return NCL_OK;
}

ncl_status ncl_kkt_get_analysis_info(ncl_kkt_t h, ncl_kkt_analysis_info* o) {
  if (!h || !o) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  const Plan& P = h->plan;
  o->dim = P.dim;
  o->nnz_A = P.nnzA;
  o->nnz_L = P.nnzL;
  o->nnz_L_stored = P.L_stored;
  o->update_entries = P.U_stored;
  o->n_supernodes = P.ns;
  o->n_levels = P.nlevels;
  o->max_front = P.max_front;
  o->max_pivots = P.max_pivots;
  o->device_bytes = h->device_bytes;
  o->flops = P.flops;
  o->analyze_ms = P.analyze_ms;
  return NCL_OK;
}

ncl_status ncl_kkt_get_permutation(ncl_kkt_t h, int32_t* perm) {
  if (!h || !perm) return fail(NCL_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(perm, h->plan.perm.data(), h->plan.perm.size() * sizeof(int32_t));
  return NCL_OK;
}

ncl_status ncl_kkt_get_supernodes(ncl_kkt_t h, int32_t* col0, int32_t* parent, int32_t* nrow) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  const Plan& P = h->plan;
  for (int32_t s = 0; s < P.ns; s++) {
    if (col0) col0[s] = P.sn_col0[s];
    if (parent) parent[s] = P.sn_parent[s];
    if (nrow) nrow[s] = P.sn_nrow[s];
  }
  if (col0) col0[P.ns] = (int32_t)P.dim;
  return NCL_OK;
}

int32_t ncl_kkt_instance_count(ncl_kkt_t h) { return h ? h->ninst : 0; }

int64_t ncl_kkt_kernel_launches(void) { return g_kernel_launches.load(); }

ncl_status ncl_kkt_profile(ncl_kkt_t h, int32_t enable) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (enable < 0) {
    h->prof.clear();
    return NCL_OK;
  }
  h->prof_on = enable ? 1 : 0;
  return NCL_OK;
}

ncl_status ncl_kkt_profile_report(ncl_kkt_t h, char* buf, int64_t buflen) {
  if (!h || !buf || buflen <= 0) return fail(NCL_ERR_INVALID_ARG, "bad arguments");
  std::string out = "{";
  bool first = true;
  for (const auto& kv : h->prof) {
    char tmp[512];
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
                  first ? "" : ", ", kv.first.c_str(), (long long)kv.second.launches, kv.second.ms, kv.second.flops,
                  kv.second.bytes);
    out += tmp;
    first = false;
  }
  out += "}";
  std::strncpy(buf, out.c_str(), (size_t)buflen - 1);
  buf[buflen - 1] = 0;
  return NCL_OK;
}

void ncl_kkt_destroy(ncl_kkt_t h) { delete h; }

const char* ncl_kkt_status_string(ncl_status st) {
  switch (st) {
    case NCL_OK: return "NCL_OK";
    case NCL_ERR_INVALID_ARG: return "NCL_ERR_INVALID_ARG";
    case NCL_ERR_PATTERN: return "NCL_ERR_PATTERN";
    case NCL_ERR_OOM: return "NCL_ERR_OOM";
    case NCL_ERR_CUDA: return "NCL_ERR_CUDA";
    case NCL_ERR_STATE: return "NCL_ERR_STATE";
    case NCL_ERR_ZERO_PIVOT: return "NCL_ERR_ZERO_PIVOT";
    case NCL_ERR_NUMERIC: return "NCL_ERR_NUMERIC";
    case NCL_ERR_IR_NOT_CONVERGED: return "NCL_ERR_IR_NOT_CONVERGED";
    case NCL_ERR_TIMEOUT: return "NCL_ERR_TIMEOUT";
    case NCL_ERR_INERTIA: return "NCL_ERR_INERTIA";
  }
  return "NCL_ERR_UNKNOWN";
}

const char* ncl_kkt_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without any device allocation.
//
// For callers that must not allocate memory at the point where they solve:
// real-time loops that cannot afford an allocator round trip, and processes
// whose device memory is fully committed to other pools (for instance after
// the factorisation was sized to the memory cap).  The workspace of the
// triangular sweeps, of the refinement and of its FGMRES stage lives in one
// file-scope device array of NCL_NOALLOC_SCRATCH_BYTES, which every GPU that
// loads this library keeps until the process exits, and the FGMRES host
// mirror in a file-scope host array.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t NCL_NOALLOC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB per GPU
__device__ __align__(256) unsigned char g_noalloc_scratch[NCL_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;       // the per-device address table
std::mutex g_noalloc_call_mu;  // one no-alloc solve at a time in the process
void* g_noalloc_base[256] = {};
// host mirror of the FGMRES partial sums and coefficients
double g_noalloc_host[(GM_M + 1) * 256 + GM_M + 8];

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not its address).
ncl_status noalloc_base(int dev, void** out) {
  if (dev < 0 || dev >= 256) return fail(NCL_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(NCL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return NCL_OK;
}

}  // namespace

extern "C" ncl_status ncl_kkt_solve_noalloc(ncl_kkt_t h, int32_t nrhs, const double* B, int64_t ldb, double* X,
                                            int64_t ldx, ncl_stream_t stream, ncl_kkt_solve_info* info) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (nrhs <= 0) return fail(NCL_ERR_INVALID_ARG, "nrhs must be positive");
  return guarded(h, [&]() -> ncl_status {
    if (h->prof_on) return fail(NCL_ERR_STATE, "turn profiling off before the no-alloc solve");
    {
      // the refinement reads residual norms back to the host between steps,
      // which a stream under capture cannot do
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      CK(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
      if (cs != cudaStreamCaptureStatusNone)
        return fail(NCL_ERR_STATE, "the no-alloc solve cannot run on a stream that is being captured");
    }
    std::lock_guard<std::mutex> serial(g_noalloc_call_mu);
    // the handle whose factors are in use (the FP64 twin after a precision
    // fallback; it exists already, and its workspace is swapped for the
    // static array as well)
    ncl_kkt_s* owner = h;
    if (h->use_twin) h = h->twin;
    void* base = nullptr;
    ncl_status s = noalloc_base(h->device, &base);
    if (s != NCL_OK) return s;
    const size_t g = (size_t)std::min(nrhs, MAX_RHS_SWEEP);
    const size_t esz = is_fp32(h) ? 4 : 8;
    const size_t dim = (size_t)h->dp.dim;
    const size_t b_xp = align256(dim * g * esz);
    const size_t b_w = align256((size_t)std::max<int64_t>(h->dp.Wtot, 1) * g * esz);
    const size_t b_pw = align256((size_t)std::max<int64_t>(h->dp.Ptot, 1) * g * esz);
    const size_t b_r = align256(dim * g * 8);
    const size_t b_n = align256(3 * (size_t)h->dp.ninst * MAX_RHS_SWEEP * 8);
    const size_t need = b_xp + b_w + b_pw + b_r + b_n;
    if (need > NCL_NOALLOC_SCRATCH_BYTES)
      return fail(NCL_ERR_INVALID_ARG, "problem too large for the no-alloc solve: needs " + std::to_string(need) +
                                           " bytes of workspace, the fixed scratch holds " +
                                           std::to_string(NCL_NOALLOC_SCRATCH_BYTES));
    // the FGMRES stage (single-instance handles, when Richardson stagnates)
    // works in the rest of the array when its Krylov vectors fit there, and
    // is left out of this call otherwise
    const int G = vec_grid();
    const size_t b_gv = align256((size_t)(GM_M + 1) * dim * 8), b_gz = align256((size_t)GM_M * dim * 8);
    const size_t b_gw = align256(dim * 8), b_gp = align256((size_t)(GM_M + 1) * G * 8);
    const size_t b_gc = align256((size_t)(GM_M + 1) * 8);
    const bool gm_fits = need + b_gv + b_gz + b_gw + b_gp + b_gc <= NCL_NOALLOC_SCRATCH_BYTES &&
                         (size_t)(GM_M + 1) * G + GM_M + 8 <= sizeof(g_noalloc_host) / sizeof(double);
    char* p = (char*)base;
    // run the regular solve on the static workspace, then give the handle
    // its own workspace back
    struct Swap {
      ncl_kkt_s* h;
      void *xp, *W, *Pw;
      double* R;
      unsigned long long* norms;
      double *gV, *gZ, *gw, *gpart, *gcoef, *ghost;
      int32_t use_fgmres;
      ~Swap() {
        h->xp = xp;
        h->W = W;
        h->Pw = Pw;
        h->R = R;
        h->d_norms = norms;
        h->gm_V = gV;
        h->gm_Z = gZ;
        h->gm_w = gw;
        h->gm_part = gpart;
        h->gm_coef = gcoef;
        h->gm_host = ghost;
        h->opt.use_fgmres = use_fgmres;
      }
    } keep{h, h->xp, h->W, h->Pw, h->R, h->d_norms, h->gm_V, h->gm_Z, h->gm_w, h->gm_part, h->gm_coef,
           h->gm_host, h->opt.use_fgmres};
    h->xp = p;
    h->W = p + b_xp;
    h->Pw = p + b_xp + b_w;
    h->R = (double*)(p + b_xp + b_w + b_pw);
    h->d_norms = (unsigned long long*)(p + b_xp + b_w + b_pw + b_r);
    if (gm_fits) {
      char* q = p + need;
      h->gm_V = (double*)q;
      h->gm_Z = (double*)(q + b_gv);
      h->gm_w = (double*)(q + b_gv + b_gz);
      h->gm_part = (double*)(q + b_gv + b_gz + b_gw);
      h->gm_coef = (double*)(q + b_gv + b_gz + b_gw + b_gp);
      h->gm_host = g_noalloc_host;
    } else {
      h->opt.use_fgmres = 0;
    }
    ncl_status r = do_solve(h, nrhs, B, ldb, X, ldx, (cudaStream_t)stream, info, false);
    if (info && h != owner) info->fp64_fallback = 1;
    return r;
  });
}

// ---------------------------------------------------------------------------
// Diagnostics: a bounded inter-CTA wait that runs out, on a real kernel
// ---------------------------------------------------------------------------
namespace {

template <typename T>
ncl_status selftest_timeout(ncl_kkt_s* h, DevNum<T>& N, int which, long long wait, cudaStream_t st) {
  static const int one = 1;
  const Plan& P = h->plan;
  const HostSched& hs = h->hs;
  int herr = 0;
  if (which == 0) {
    // the forward sweep's chain over the block-rows of a supernode with more
    // than one: its ticket counter starts at 1 and only nbr - 1 CTAs run, so
    // block-row 0 is never solved and its flag never published; the CTA of
    // block-row 1 waits for it until the limit
    int64_t i0 = -1;
    int nbr = 0, smem = 0;
    for (const Level& L : h->levels) {
      for (int64_t i = L.chain_off; i < L.chain_off + L.chain_cnt; i++) {
        const int s = hs.chainv[i].x;
        if (P.sn_ncol[s] > CHAIN_ROWS && (i == L.chain_off || hs.chainv[i - 1].x != s)) {
          i0 = i;
          nbr = (P.sn_ncol[s] + CHAIN_ROWS - 1) / CHAIN_ROWS;
          smem = (int)L.chain_smem;
          break;
        }
      }
      if (i0 >= 0) break;
    }
    if (i0 < 0) return fail(NCL_ERR_INVALID_ARG, "no supernode with more than one block-row");
    const int s = hs.chainv[i0].x;
    const int64_t ns = P.ns, nb = hs.nbrows;
    int* tk_f = h->d_chain_sync;
    int* fl_f = tk_f + 2 * ns;
    CK(cudaMemsetAsync(h->d_chain_sync, 0, (2 * ns + 2 * nb) * sizeof(int), st));
    CK(cudaMemcpyAsync(tk_f + s, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->d_err + 1, 0, sizeof(int), st));
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    launch_fwd_chain<T>(h->dp, N, h->d_chain + i0, nbr - 1, smem, true, h->d_chain_pptr, h->d_chain_pran,
                        (T*)h->own_xp, (const T*)h->W, 1, tk_f, fl_f, h->d_err + 1, wait, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&herr, h->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(h->d_err + 1, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
  } else {
    // the first macro panel of a large front with rows below it: its ticket
    // counter starts at 1, so no CTA takes the diagonal role and the
    // sub-block flags are never published; the row CTAs wait until the limit
    int64_t g0 = -1;
    int nrc = 0;
    for (size_t i = 0; i < hs.panelv.size();) {
      const int4 it = hs.panelv[i];
      const int qe = std::min(it.y + MACRO_NB, (int)P.sn_ncol[it.x]);
      const int n = (P.sn_nrow[it.x] - qe + MACRO_ROWS - 1) / MACRO_ROWS;
      if (n >= 1) {
        g0 = (int64_t)i;
        nrc = n;
        break;
      }
      i += 1 + (size_t)n;
    }
    if (g0 < 0) return fail(NCL_ERR_INVALID_ARG, "no macro panel with rows below it");
    CK(cudaMemsetAsync(h->d_panel_sync, 0, std::max<int64_t>(hs.panel_sync, 8) * sizeof(int), st));
    CK(cudaMemcpyAsync(h->d_panel_sync + hs.panelv[g0].z, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    launch_macro_panel<T>(h->dp, N, h->d_panel + g0, nrc, h->d_panel_sync, h->d_err,
                          h->opt.pivot_eps, h->opt.pivot_policy, wait, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    // the row CTAs went on without the diagonal block: the factors are void
    h->factored = false;
    h->use_twin = false;
  }
  if (herr) return fail(NCL_ERR_TIMEOUT, "the bounded wait ran out (as this self-test arranges)");
  return NCL_OK;
}

}  // namespace

extern "C" ncl_status ncl_kkt_selftest_wait_timeout(ncl_kkt_t h, int32_t which, int64_t wait_cycles,
                                                    ncl_stream_t stream) {
  if (!h) return fail(NCL_ERR_INVALID_ARG, "NULL handle");
  if (h->opt.host_only) return fail(NCL_ERR_STATE, "host-only handle");
  if (which != 0 && which != 1) return fail(NCL_ERR_INVALID_ARG, "which must be 0 (sweep) or 1 (panel)");
  if (wait_cycles <= 0) return fail(NCL_ERR_INVALID_ARG, "wait_cycles must be positive");
  if (which == 0 && !h->factored) return fail(NCL_ERR_STATE, "sweep self-test before a successful factor");
  return guarded(h, [&]() -> ncl_status {
    const cudaStream_t st = (cudaStream_t)stream;
    if (is_fp32(h)) return selftest_timeout<float>(h, h->nf, which, (long long)wait_cycles, st);
    return selftest_timeout<double>(h, h->nd, which, (long long)wait_cycles, st);
  });
}

// ---------------------------------------------------------------------------
// Diagnostics: the tensor-core update kernel on caller data
// ---------------------------------------------------------------------------
extern "C" ncl_status ncl_kkt_selftest_tensor_update(int32_t rows, int32_t ld, int32_t K, const float* L,
                                                     const float* d, int32_t row_a, int32_t row_b, int32_t M,
                                                     int32_t N, float* C, int32_t ldc, ncl_stream_t stream) {
  if (!L || !d || !C || rows <= 0 || K <= 0 || ld < K || ld % 4 != 0 || M <= 0 || N <= 0 || N > M ||
      row_a < 0 || row_b < 0 || row_a + M > rows || row_b + N > rows || ldc < N)
    return fail(NCL_ERR_INVALID_ARG, "bad self-test arguments");
  cudaStream_t st = (cudaStream_t)stream;
  float* S = nullptr;
  CUtensorMap* dmaps = nullptr;
  TcProb* dp = nullptr;
  int* derr = nullptr;
  int32_t* dtp = nullptr;
  auto release = [&] {
    if (S) cudaFree(S);
    if (dmaps) cudaFree(dmaps);
    if (dp) cudaFree(dp);
    if (derr) cudaFree(derr);
    if (dtp) cudaFree(dtp);
  };
  const size_t plane = (size_t)rows * ld;
  if (cudaMalloc(&S, 4 * plane * sizeof(float)) != cudaSuccess || cudaMalloc(&dmaps, 4 * sizeof(CUtensorMap)) ||
      cudaMalloc(&dp, sizeof(TcProb)) || cudaMalloc(&derr, sizeof(int))) {
    cudaGetLastError();
    release();
    return fail(NCL_ERR_OOM, "self-test allocation failed");
  }
  CUtensorMap maps[4];
  std::string why;
  if (!tc_encode_maps(S, rows, ld, maps, &why)) {
    release();
    return fail(NCL_ERR_CUDA, why);
  }
  TcProb q{};
  q.c_off = 0;
  q.ldc = ldc;
  q.c_in_u = 0;
  q.map = 0;
  q.row_a = row_a;
  q.row_b = row_b;
  q.k0 = 0;
  q.nk = (K + 31) / 32;
  q.M = M;
  q.N = N;
  q.tile0 = 0;
  const int64_t tiles = tc_tiles(M, N, &q.Nt);
  if (cudaMalloc(&dtp, tiles * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(NCL_ERR_OOM, "self-test allocation failed");
  }
  DevPlan P0{};
  DevNum<float> N0{};
  N0.L = C;
  N0.U = C;
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(dmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, &q, sizeof(q), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dtp, 0, tiles * sizeof(int32_t), st);
  if (e == cudaSuccess) {
    launch_split_rows(L, d, rows, ld, K, S, st);
    launch_update_tc(P0, N0, dp, dtp, tiles, 3, dmaps, derr, DEFAULT_WAIT_CYCLES, st);
    g_kernel_launches.fetch_add(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return fail(NCL_ERR_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
  if (herr) return fail(NCL_ERR_TIMEOUT, "self-test: a bounded wait ran out");
  return NCL_OK;
}
