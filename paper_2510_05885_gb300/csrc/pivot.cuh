// Static pivoting (internal), shared by the small-front and macro-panel kernels.
#pragma once
#include "runtime.h"

namespace ncl {

// finite (not NaN, not infinite) in the value's own precision
__device__ __forceinline__ bool finite_val(float x) { return fabsf(x) <= 3.402823466e38f; }
__device__ __forceinline__ bool finite_val(double x) { return fabs(x) <= 1.7976931348623157e308; }

// Static pivot (Section 3.1): no exchange; |d| <= eps is replaced by
// +-eps with the sign of the pivot's block before reordering (case (ii)),
// or counted as a zero eigenvalue (case (i), status 2).  Status 3 marks a
// non-finite pivot.
template <typename T>
__device__ __forceinline__ T static_pivot(T d, int sign, double eps, int policy, int8_t& st) {
  // compared in the factor's own precision: FP64 arithmetic is slow on this
  // part, and a pivot of the FP32 factor is an FP32 number
  if (!finite_val(d)) {
    st = 3;
    return d;
  }
  const T e = (T)eps;
  if ((d < T(0) ? -d : d) <= e) {
    st = policy == 0 ? 1 : 2;
    return sign < 0 ? -e : e;
  }
  st = 0;
  return d;
}

}  // namespace ncl
