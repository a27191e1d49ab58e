// Static pivoting and the warp-level factorisation of a 32 x 32 diagonal
// block, shared by the assembly, panel and update kernels (internal).
#pragma once
#include "runtime.h"

namespace ncl {

// Static pivot (Section 3.1): no exchange; |d| <= eps is replaced by
// +-eps with the sign of the pivot's block before reordering (case (ii)),
// or counted as a zero eigenvalue (case (i), status 2).  Status 3 marks a
// non-finite pivot.
template <typename T>
__device__ __forceinline__ T static_pivot(T d, int sign, double eps, int policy, int8_t& st) {
  if (!isfinite((double)d)) {
    st = 3;
    return d;
  }
  if (fabs((double)d) <= eps) {
    st = policy == 0 ? 1 : 2;
    return sign < 0 ? (T)(-eps) : (T)eps;
  }
  st = 0;
  return d;
}

// One warp (all 32 lanes call it) factors in place the diagonal block of
// pivot columns [p0, min(p0 + 32, ncol)) of front s: lane i holds row i of
// the block in registers; right-looking LDL^T with column broadcasts by
// shuffles.  Writes L11 (unit lower, strictly below the diagonal), D on the
// diagonal, and the pivots and their status.
template <typename T>
__device__ __forceinline__ void factor_diag32(const DevPlan& P, const DevNum<T>& N, int s, int p0, double eps,
                                              int policy, int lane) {
  const int ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s];
  const int col0 = P.sn_col0[s];
  const int nbk = min(32, ncol - p0);
  T* Lb = N.L + P.sn_Loff[s];
  T r[32];
  const T* rp = Lb + (int64_t)(p0 + min(lane, nbk - 1)) * ncp + p0;
#pragma unroll
  for (int j = 0; j < 32; j++) r[j] = (j <= lane && lane < nbk) ? rp[j] : T(0);
  int8_t my_st = 0;
  T my_d = T(0);
  const int my_sign = lane < nbk ? P.col_sign[col0 + p0 + lane] : 1;
#pragma unroll
  for (int k = 0; k < 32; k++) {
    if (k < nbk) {
      int8_t stt;
      const int sg = __shfl_sync(0xffffffffu, my_sign, k);
      const T dk = static_pivot<T>(__shfl_sync(0xffffffffu, r[k], k), sg, eps, policy, stt);
      const T wk = r[k];
      const T li = wk / dk;
#pragma unroll
      for (int j = k + 1; j < 32; j++) {
        const T wj = __shfl_sync(0xffffffffu, wk, j);
        if (lane >= j) r[j] -= li * wj;
      }
      if (lane > k) r[k] = li;
      if (lane == k) {
        r[k] = dk;
        my_d = dk;
        my_st = stt;
      }
    }
  }
  if (lane < nbk) {
    T* wp = Lb + (int64_t)(p0 + lane) * ncp + p0;
#pragma unroll
    for (int j = 0; j < 32; j++)
      if (j <= lane) wp[j] = r[j];
    N.D[col0 + p0 + lane] = my_d;
    N.piv[col0 + p0 + lane] = my_st;
  }
}

}  // namespace ncl
