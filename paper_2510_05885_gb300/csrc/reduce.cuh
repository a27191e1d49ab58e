// Per-instance reductions of the norm and inertia kernels (internal).
//
// Each thread keeps a running maximum (or count) for the instance of the
// rows it is visiting and flushes it with one atomic when the instance
// changes; at the end the warp combines the lanes that share an instance
// and issues one atomic for them.  (One atomic per row on a single address
// serialises in L2.)
#pragma once
#include <cuda_runtime.h>

namespace ncl {

constexpr unsigned FULL_MASK = 0xffffffffu;

// bit pattern of a non-negative double: atomicMax on it orders the values
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// warp-aggregated atomicMax(dst[key], v); key < 0 contributes nothing.
// Called by all 32 lanes.
__device__ __forceinline__ void warp_flush_max(unsigned long long* dst, int key, unsigned long long v) {
  const int k0 = __shfl_sync(FULL_MASK, key, 0);
  const bool same = key == k0;
  unsigned long long w = same ? v : 0ull;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(FULL_MASK, w, o);
    w = u > w ? u : w;
  }
  if ((threadIdx.x & 31) == 0 && k0 >= 0) atomicMax(dst + k0, w);
  if (!same && key >= 0) atomicMax(dst + key, v);
}

// warp-aggregated atomicAdd(dst[key], v); called by all 32 lanes
__device__ __forceinline__ void warp_flush_add(unsigned long long* dst, int key, unsigned v) {
  const int k0 = __shfl_sync(FULL_MASK, key, 0);
  const bool same = key == k0;
  const unsigned w = __reduce_add_sync(FULL_MASK, same ? v : 0u);
  if ((threadIdx.x & 31) == 0 && k0 >= 0 && w) atomicAdd(dst + k0, (unsigned long long)w);
  if (!same && key >= 0 && v) atomicAdd(dst + key, (unsigned long long)v);
}

}  // namespace ncl
