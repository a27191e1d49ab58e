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
template <typename T>
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
    panel_diag_role<T>(P, N, s, q0, slot + 1, eps, policy, smem_raw);
  } else {
    const int qe = min(q0 + MNB, P.sn_ncol[s]);
    panel_rows_role<T>(P, N, s, q0, qe + RB * (ticket - 1), slot + 1, err, wait, smem_raw);
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

template <typename T>
__global__ void __launch_bounds__(256) k_factor_small(DevPlan P, DevNum<T> N, const int32_t* __restrict__ list,
                                                      double eps, int policy) {
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
      const T d = factor_sub32<T>(F + c0 * ldf + c0, ldf, cw, lane < cw ? P.col_sign[col0 + c0 + lane] : 1, eps,
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
      for (int r0 = c0 + 32 + warp * RW; r0 < nrow; r0 += 8 * RW) {
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
  k_factor_small<T><<<count, 256, smem_bytes, st>>>(P, N, list, eps, policy);
}

template void launch_factor_small<float>(const DevPlan&, const DevNum<float>&, const int32_t*, int, int, double,
                                         int, cudaStream_t);
template void launch_factor_small<double>(const DevPlan&, const DevNum<double>&, const int32_t*, int, int, double,
                                          int, cudaStream_t);

template <typename T>
void launch_macro_panel(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int* sync, int* err,
                        double eps, int policy, long long wait, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  const int smem = macro_panel_smem((int)sizeof(T));
  if (!attr) {
    cudaFuncSetAttribute(k_macro_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  k_macro_panel<T><<<count, 256, smem, st>>>(P, N, items, sync, err, eps, policy, wait);
}

template void launch_macro_panel<float>(const DevPlan&, const DevNum<float>&, const int4*, int, int*, int*, double,
                                        int, long long, cudaStream_t);
template void launch_macro_panel<double>(const DevPlan&, const DevNum<double>&, const int4*, int, int*, int*, double,
                                         int, long long, cudaStream_t);

}  // namespace ncl
