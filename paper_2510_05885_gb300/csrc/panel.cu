// Dense front kernels (sm_103a): the per-step macro-panel kernel of large
// fronts (the roles are in panel_roles.cuh), and whole small fronts.
#include "panel_roles.cuh"

#include <algorithm>

namespace ncl {

// One launch per macro panel step of a level: for each large front, one
// CTA in the diagonal role and one per RB rows below the panel in the row
// role.  A CTA's role comes from the front's ticket counter (the first CTA
// to arrive takes the diagonal), so every CTA that waits waits for a CTA
// that is already running: the waits cannot deadlock, whatever the order
// in which CTAs are scheduled.  Waits are bounded (the factor's error flag
// is set past the limit).
// items: (front, q0, sync slot); sync[slot] = ticket counter, sync[slot + 1
// + j] = flag of sub-block j.
template <typename T, int NB>
__global__ void __launch_bounds__(256, 1) k_macro_panel(DevPlan P, DevNum<T> N, const int4* __restrict__ items,
                                                        int* sync, int* err, double eps, int policy,
                                                        long long wait) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int ticket;
  const int4 it = items[blockIdx.x];
  const int s = it.x, q0 = it.y;
  int* slot = sync + it.z;
  if (threadIdx.x == 0) ticket = atomicAdd(slot, 1);
  __syncthreads();
  if (ticket == 0) {
    panel_diag_role<T, NB>(P, N, s, q0, slot + 1, eps, policy, smem_raw);
  } else {
    const int qe = min(q0 + NB, P.sn_ncol[s]);
    panel_rows_role<T, NB>(P, N, s, q0, qe + RB * (ticket - 1), slot + 1, err, wait, smem_raw);
  }
}

// Small fronts (ncol <= 64): one CTA factors the pivot columns of the whole
// front in shared memory by 32-column sub-blocks, as the diagonal-block
// kernel does: one warp factors the sub-block (factor_sub32) and inverts it
// (for the triangular sweeps), the rows below it are solved by the blocked
// forward substitution, L21 = F21 L_jj^-T D^-1, and, when a second
// sub-block follows, the warps update its columns.  The update
// block F22 -= L21 D1 L21^T is left to the SIMT update kernel, which spreads
// it over many CTAs.
int small_front_smem(int nrow, int ncp, int esz) { return (nrow * (ncp + 1) + 32 * LDS + 64) * esz; }

// 256 threads per CTA (128 was measured slower on the 20 x 25, 300 x 300 and
// 700 x 700 systems: the rows below the sub-block take twice the passes)
constexpr int SMALL_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(SMALL_THREADS) k_factor_small(DevPlan P, DevNum<T> N,
                                                                const int32_t* __restrict__ list, double eps,
                                                                int policy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = list[blockIdx.x];
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int ldf = ncp + 1;   // odd: column accesses by lanes are conflict-free
  T* F = reinterpret_cast<T*>(smem_raw);
  T* Ls = F + nrow * ldf;     // the sub-block's unit lower factor, zero padded
  T* dsh = Ls + 32 * LDS;     // pivots
  T* Lg = N.L + P.sn_Loff[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  load_tile(F, ldf, Lg, ncp, nrow, ncp, [](int, int) { return true; });
  __syncthreads();
  constexpr int RW = 8;   // rows per register batch of a warp
  for (int c0 = 0; c0 < ncol; c0 += 32) {
    const int cw = min(32, ncol - c0);
    if (warp == 0) {
      int8_t st;
      const T d = factor_sub32<T, true>(F + c0 * ldf + c0, ldf, cw, lane < cw ? P.col_sign[col0 + c0 + lane] : 1, eps,
                                  policy, lane, st);
      dsh[c0 + lane] = d;
      if (lane < cw) {
        N.D[col0 + c0 + lane] = d;
        N.piv[col0 + c0 + lane] = st;
      }
      // the unit lower sub-block, zero above the diagonal and on the padding
#pragma unroll 4
      for (int u = 0; u < 32; u++) Ls[lane * LDS + u] = (u < lane && lane < cw) ? F[(c0 + lane) * ldf + c0 + u] : T(0);
      __syncwarp();
      invert_sub32<T>(Ls, LDS, cw, N.Linv + P.sn_Ioff[s] + (int64_t)(c0 >> 5) * 1024, lane);
    }
    __syncthreads();
    // rows below the sub-block: L21 = F21 L_jj^-T D^-1 (blocked forward
    // substitution, then the scaling)
    const int rb = c0 + cw;
    block_trsm32<T>(F + rb * ldf + c0, ldf, nrow - rb, cw, Ls, LDS);
    __syncthreads();
    for (int idx = tid; idx < (nrow - rb) * 32; idx += blockDim.x) {
      const int r = idx >> 5, c = idx & 31;
      if (c < cw) F[(rb + r) * ldf + c0 + c] /= dsh[c0 + c];
    }
    __syncthreads();
    // update the next sub-block's columns: F[r][c] -= sum_u L[r][u] d_u L[c][u]
    if (c0 + 32 < ncol) {
      const int c = c0 + 32 + lane;
      const bool cok = c < ncol;
      for (int r0 = c0 + 32 + warp * RW; r0 < nrow; r0 += (SMALL_THREADS / 32) * RW) {
        T acc[RW];
#pragma unroll
        for (int m = 0; m < RW; m++) acc[m] = T(0);
#pragma unroll 4
        for (int u = 0; u < 32; u++) {
          const T b = F[min(c, ncol - 1) * ldf + c0 + u] * dsh[c0 + u];
#pragma unroll
          for (int m = 0; m < RW; m++) acc[m] += F[min(r0 + m, nrow - 1) * ldf + c0 + u] * b;
        }
#pragma unroll
        for (int m = 0; m < RW; m++)
          if (cok && r0 + m < nrow && c <= r0 + m) F[(r0 + m) * ldf + c] -= acc[m];
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < nrow * ncp; idx += blockDim.x) Lg[idx] = F[(idx / ncp) * ldf + idx % ncp];
}

template <typename T>
void launch_factor_small(const DevPlan& P, const DevNum<T>& N, const int32_t* list, int count, int smem_bytes,
                         double eps, int policy, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_factor_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMALL_SMEM_MAX);
    attr = true;
  }
  k_factor_small<T><<<count, SMALL_THREADS, smem_bytes, st>>>(P, N, list, eps, policy);
}

// ---------------------------------------------------------------------------
// Factorisation of the subtrees of small fronts.
//
// The fronts of the small-subtree region (at most 32 pivots, small enough
// for the shared-memory front, and only such fronts below them) are
// factored by one CTA per maximal subtree, front by front in postorder, in
// one launch for the whole region; the level launches of the assembly, the
// small-front factorisation and the update blocks skip them.  Per front:
//   the front is assembled straight into shared memory (original entries,
//   then the children's update blocks child by child; a child's entries
//   that land below the pivot columns go to this front's update block in
//   global memory, zeroed first), the 32-column pivot block is factored by
//   one warp, the rows below by the blocked substitution, L21 = F21 L11^-T
//   D1^-1, the factor block written back, and the update block
//   F22 -= L21 D1 L21^T formed from the shared-memory front.
// The children's update blocks were written by the same CTA earlier, so a
// barrier orders them; nothing waits across CTAs.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void subtree_front(const DevPlan& P, const DevNum<T>& N, int s, double eps, int policy,
                                              unsigned char* smem_raw) {
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int nb = nrow - ncol;
  const int ldf = ncp + 1;
  T* F = reinterpret_cast<T*>(smem_raw);
  T* Ls = F + nrow * ldf;
  T* dsh = Ls + 32 * LDS;
  T* Lg = N.L + P.sn_Loff[s];
  T* Ub = N.U + P.sn_Uoff[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  // zero the front and the update block
  for (int idx = tid; idx < nrow * ldf; idx += blockDim.x) F[idx] = T(0);
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) Ub[idx] = T(0);
  __syncthreads();
  // original entries (each lands in its own position): the front's entries
  // spread over all threads, so that their loads are independent
  const int64_t rbase = P.sn_rows_off[s];
  {
    const int64_t q0 = P.amap_ptr[rbase], q1 = P.amap_ptr[rbase + nrow];
    for (int64_t q = q0 + tid; q < q1; q += blockDim.x)
      F[P.amap_row[q] * ldf + P.amap_col[q]] = (T)N.Klow[P.amap_src[q]];
  }
  // the children's update blocks, child by child (the targets of one child
  // are distinct: its relative map is increasing); each child's lower
  // triangle spread over all threads
  for (int k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
    __syncthreads();
    const int c = P.child_list[k];
    const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
    const int32_t* rel = P.relmap + P.relmap_off[c];
    const T* Uc = N.U + P.sn_Uoff[c];
    const int tot = nbc * (nbc + 1) / 2;
    for (int e = tid; e < tot; e += blockDim.x) {
      int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (a * (a + 1) / 2 > e) a--;
      while ((a + 1) * (a + 2) / 2 <= e) a++;
      const int b = e - a * (a + 1) / 2;
      const int ra = rel[a], rb = rel[b];
      const T v = Uc[(int64_t)a * nbc + b];
      if (rb < ncol) F[ra * ldf + rb] += v;
      else Ub[(int64_t)(ra - ncol) * nb + (rb - ncol)] += v;
    }
  }
  __syncthreads();
  // the pivot block (one 32-column sub-block) by warp 0: LDL^T, pivots,
  // statuses, the zero-padded unit lower block and its inverse
  if (warp == 0) {
    int8_t st;
    const T d = factor_sub32<T, true>(F, ldf, ncol, lane < ncol ? P.col_sign[col0 + lane] : 1, eps, policy, lane, st);
    dsh[lane] = d;
    if (lane < ncol) {
      N.D[col0 + lane] = d;
      N.piv[col0 + lane] = st;
    }
#pragma unroll 4
    for (int u = 0; u < 32; u++) Ls[lane * LDS + u] = (u < lane && lane < ncol) ? F[lane * ldf + u] : T(0);
    __syncwarp();
    invert_sub32<T>(Ls, LDS, ncol, N.Linv + P.sn_Ioff[s], lane);
  }
  __syncthreads();
  // rows below: L21 = F21 L11^-T D1^-1
  block_trsm32<T>(F + ncol * ldf, ldf, nb, ncol, Ls, LDS);
  __syncthreads();
  for (int idx = tid; idx < nb * 32; idx += blockDim.x) {
    const int r = idx >> 5, c = idx & 31;
    if (c < ncol) F[(ncol + r) * ldf + c] *= pivot_rcp(dsh[c]);
  }
  __syncthreads();
  // write the factor block back, and form the update block from it:
  // 4 x 4 register tiles of its lower triangle spread over all threads
  // (9 shared loads per 16 products), F22[a][b] -= sum_k (L[a][k] d_k) L[b][k]
  for (int idx = tid; idx < nrow * ncp; idx += blockDim.x) Lg[idx] = F[(idx / ncp) * ldf + idx % ncp];
  const int T4 = (nb + 3) / 4;
  const int ntl = T4 * (T4 + 1) / 2;
  for (int e = tid; e < ntl; e += blockDim.x) {
    int ti = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > e) ti--;
    while ((ti + 1) * (ti + 2) / 2 <= e) ti++;
    const int tj = e - ti * (ti + 1) / 2;
    const int a0 = 4 * ti, b0 = 4 * tj;
    const T* fa = F + (ncol + a0) * ldf;
    const T* fb = F + (ncol + b0) * ldf;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) acc[i][j] = T(0);
#pragma unroll 4
    for (int k = 0; k < ncol; k++) {
      const T dk = dsh[k];
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; i++) av[i] = a0 + i < nb ? fa[i * ldf + k] * dk : T(0);
#pragma unroll
      for (int j = 0; j < 4; j++) bv[j] = b0 + j < nb ? fb[j * ldf + k] : T(0);
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] += av[i] * bv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int a = a0 + i, b = b0 + j;
        if (a < nb && b <= a) Ub[(int64_t)a * nb + b] -= acc[i][j];
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_subtree_factor(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                        int count, const int32_t* __restrict__ nodes, int* counter,
                                                        double eps, int policy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= count) break;
    const int2 item = items[it];
    for (int q = 0; q < item.y; q++) {
      subtree_front<T>(P, N, nodes[item.x + q], eps, policy, smem_raw);
      __syncthreads();
    }
  }
}

template <typename T>
void launch_subtree_factor(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes,
                           int* counter, int smem, int nsm, double eps, int policy, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_subtree_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMALL_SMEM_MAX);
    attr = true;
  }
  // as many CTAs as fit on the device at once (they take subtrees from a counter)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_subtree_factor<T>, 256, smem) != cudaSuccess)
    per_sm = 4;
  const int grid = std::min(count, nsm * std::max(per_sm, 1));
  k_subtree_factor<T><<<grid, 256, smem, st>>>(P, N, items, count, nodes, counter, eps, policy);
}

template void launch_subtree_factor<float>(const DevPlan&, const DevNum<float>&, const int2*, int, const int32_t*,
                                           int*, int, int, double, int, cudaStream_t);
template void launch_subtree_factor<double>(const DevPlan&, const DevNum<double>&, const int2*, int, const int32_t*,
                                            int*, int, int, double, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Inverses of the unit lower 32 x 32 diagonal sub-blocks of the large
// fronts' pivot blocks (used by the triangular sweeps), one warp per
// sub-block, after the factorisation: items (supernode, sub-block).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_invert_blocks(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                       int count) {
  const int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (it >= count) return;
  const int s = items[it].x, b = items[it].y;
  const int ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s];
  const T* blk = N.L + P.sn_Loff[s] + (int64_t)(32 * b) * ncp + 32 * b;
  invert_sub32<T>(blk, ncp, min(32, ncol - 32 * b), N.Linv + P.sn_Ioff[s] + (int64_t)b * 1024, lane);
}

template <typename T>
void launch_invert_blocks(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, cudaStream_t st) {
  if (count <= 0) return;
  k_invert_blocks<T><<<(count + 7) / 8, 256, 0, st>>>(P, N, items, count);
}

template void launch_invert_blocks<float>(const DevPlan&, const DevNum<float>&, const int2*, int, cudaStream_t);
template void launch_invert_blocks<double>(const DevPlan&, const DevNum<double>&, const int2*, int, cudaStream_t);

template void launch_factor_small<float>(const DevPlan&, const DevNum<float>&, const int32_t*, int, int, double,
                                         int, cudaStream_t);
template void launch_factor_small<double>(const DevPlan&, const DevNum<double>&, const int32_t*, int, int, double,
                                          int, cudaStream_t);

template <typename T, int NB>
static void launch_macro_panel_nb(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int* sync,
                                  int* err, double eps, int policy, long long wait, cudaStream_t st) {
  static bool attr = false;
  const int smem = macro_panel_smem((int)sizeof(T), NB);
  if (!attr) {
    cudaFuncSetAttribute(k_macro_panel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  k_macro_panel<T, NB><<<count, 256, smem, st>>>(P, N, items, sync, err, eps, policy, wait);
}

// (a 192-column FP32 panel was measured slower than 128 columns on the
// condensed 300 x 300 and stabilized 700 x 700 grids: the diagonal role's
// serial chain of 32-column factorisations grows with the width)
template <typename T>
void launch_macro_panel(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int* sync, int* err,
                        double eps, int policy, long long wait, cudaStream_t st) {
  if (count <= 0) return;
  launch_macro_panel_nb<T, MACRO_NB>(P, N, items, count, sync, err, eps, policy, wait, st);
}

template void launch_macro_panel<float>(const DevPlan&, const DevNum<float>&, const int4*, int, int*, int*,
                                        double, int, long long, cudaStream_t);
template void launch_macro_panel<double>(const DevPlan&, const DevNum<double>&, const int4*, int, int*, int*,
                                         double, int, long long, cudaStream_t);

}  // namespace ncl
