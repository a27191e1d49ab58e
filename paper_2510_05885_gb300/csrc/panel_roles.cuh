// Device roles of the dense front factorisation (internal), shared by the
// per-step macro-panel kernel (panel.cu) and the persistent front kernel
// (front_dag.cu): the 32-column sub-block LDL^T, the blocked substitution,
// the diagonal role and the row role of a 128-column macro panel.
//
// The pivot columns of a large front are processed NB = 128 at a time
// (right-looking blocked LDL^T with D diagonal and static pivoting, Section
// 3.1).  For macro panel [q0, qe) one launch (k_macro_panel) runs, for every
// large front of the level:
//   the diagonal role  one CTA: the w x w diagonal block (w <= 128) is
//                      factored in shared memory by 32-column sub-blocks,
//                      each published as soon as it is done;
//   the row role       one CTA per 64 rows below the panel: as the
//                      sub-blocks appear, the blocked forward substitution
//                      L21 = F21 L11^-T D1^-1; for a tensor-core front also
//                      the split TF32 operands of L21 and W = L21 D1.
// Then the trailing update of the remaining pivot columns with K = w runs on
// the SIMT or the tensor-core update kernel.
#pragma once
#include "runtime.h"
#include "pivot.cuh"

#include <algorithm>

namespace ncl {

namespace {

constexpr int RB = MACRO_ROWS;     // rows per row CTA
constexpr int LDS = 33;            // stride of the 32 x 32 shared blocks

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace

// Copy a rows x cols tile from global memory (row stride lds) into shared
// memory (row stride ldd), zero where keep(r, c) is false, with 8 loads in
// flight per thread before the shared stores.
template <typename T, typename Keep>
__device__ __forceinline__ void load_tile(T* dst, int ldd, const T* src, int64_t lds, int rows, int cols, Keep keep) {
  const int n = rows * cols;
  for (int base = threadIdx.x; base < n; base += 8 * blockDim.x) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = base + k * blockDim.x;
      const int r = idx / cols, c = idx - r * cols;
      v[k] = (idx < n && keep(r, c)) ? src[(int64_t)r * lds + c] : T(0);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = base + k * blockDim.x;
      const int r = idx / cols, c = idx - r * cols;
      if (idx < n) dst[r * ldd + c] = v[k];
    }
  }
}

// shared memory of the two roles of a panel nb columns wide (row stride nb + 1)
inline int macro_diag_smem(int esz, int nb) { return (nb * (nb + 1) + (nb - 32) * LDS + nb) * esz + 2 * nb; }
inline int macro_rows_smem(int esz, int nb) {
  const int k = nb / 32;   // the diagonal sub-blocks of L11 and those below them
  return (RB * (nb + 1) + (k + k * (k - 1) / 2) * 32 * LDS + nb) * esz;
}
inline int macro_panel_smem(int esz, int nb) { return std::max(macro_diag_smem(esz, nb), macro_rows_smem(esz, nb)); }

// LDL^T of a 32 x 32 diagonal sub-block in shared memory (row stride ld,
// cw <= 32 valid rows) by one warp, lane i holding row i in registers:
// right-looking with column broadcasts by shuffles.  Writes the unit lower
// factor (strictly below the diagonal) and D on the diagonal back; returns
// lane's pivot (1 on the padding) and its status in st.
// reciprocal of a pivot: correctly rounded in FP32 without the general
// division's slow path (pivots are normal numbers: |d| > eps or replaced)
__device__ __forceinline__ float pivot_rcp(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double pivot_rcp(double d) { return 1.0 / d; }

// One column step of the 32 x 32 factorisation in registers: rows above the
// pivot get a zero multiplier, so the update needs no per-column select or
// branch; entries above a lane's diagonal are never read.
template <typename T>
__device__ __forceinline__ void factor_step(T (&r)[32], int k, T dk, int lane, T& my_d) {
  const T wk = r[k];
  const T li = lane > k ? wk * pivot_rcp(dk) : T(0);
#pragma unroll
  for (int j = k + 1; j < 32; j++)
    if (j > k) r[j] -= li * __shfl_sync(0xffffffffu, wk, j);
  r[k] = lane > k ? li : (lane == k ? dk : r[k]);
  my_d = lane == k ? dk : my_d;
}

// LDL^T of a 32 x 32 diagonal sub-block in shared memory (row stride ld,
// cw <= 32 valid rows) by one warp, lane i holding row i in registers:
// right-looking with column broadcasts by shuffles.  Writes the unit lower
// factor (strictly below the diagonal) and D on the diagonal back; returns
// lane's pivot (1 on the padding) and its status in st.  Static pivoting
// (Section 3.1): a pivot with |d| <= eps becomes +-eps by the sign of its
// block (status 1 perturbed, or 2 zero under the stop policy), a non-finite
// pivot is kept (status 3).  The common case has no such pivot: the columns
// run without any pivot test, the tests run once afterwards on the pivots
// the lanes kept, and only when one fired does the block run again from
// shared memory with the replacement at each step.
// EARLY: stop after column cw (narrow blocks of small fronts); otherwise
// all 32 steps run on the identity-padded block (no branch between steps).
template <typename T, bool EARLY>
__device__ __noinline__ T factor_sub32(T* blk, int ld, int cw, int my_sign, double eps, int policy, int lane,
                                       int8_t& st) {
  T r[32];
  auto load = [&] {
#pragma unroll
    for (int j = 0; j < 32; j++)
      r[j] = lane < cw ? ((j <= lane) ? blk[lane * ld + j] : T(0)) : (j == lane ? T(1) : T(0));
  };
  load();
  const T e = (T)eps;
  T my_d = T(1);
#pragma unroll
  for (int k = 0; k < 32; k++) {
    if (EARLY && k >= cw) break;
    factor_step(r, k, __shfl_sync(0xffffffffu, r[k], k), lane, my_d);
  }
  // the pivot tests, once at the end: lane k's my_d is the pivot of step k
  // (1 on the padding and beyond cw)
  const T ad = my_d < T(0) ? -my_d : my_d;
  unsigned tiny_mask = __ballot_sync(0xffffffffu, ad <= e);   // NaN compares false
  unsigned bad_mask = __ballot_sync(0xffffffffu, !finite_val(my_d));
  if (tiny_mask | bad_mask) {
    // again, with the static pivot applied at each step
    const unsigned neg = __ballot_sync(0xffffffffu, my_sign < 0);
    load();
    tiny_mask = bad_mask = 0u;
    my_d = T(1);
#pragma unroll
    for (int k = 0; k < 32; k++) {
      if (EARLY && k >= cw) break;
      const T d0 = __shfl_sync(0xffffffffu, r[k], k);
      const T a = d0 < T(0) ? -d0 : d0;
      const bool fin = finite_val(d0);
      const bool tiny = fin && a <= e;
      tiny_mask |= (unsigned)tiny << k;
      bad_mask |= (unsigned)(!fin) << k;
      factor_step(r, k, tiny ? (((neg >> k) & 1u) ? -e : e) : d0, lane, my_d);
    }
  }
  if (lane < cw) {
#pragma unroll
    for (int j = 0; j < 32; j++)
      if (j <= lane) blk[lane * ld + j] = r[j];
  }
  __syncwarp();
  st = (lane >= cw) ? 0 : (((bad_mask >> lane) & 1u) ? 3 : (((tiny_mask >> lane) & 1u) ? (policy == 0 ? 1 : 2) : 0));
  return my_d;
}

// Inverse of the unit lower 32 x 32 block blk (row stride ld, cw valid
// rows; identity on the padding) by one warp, written row-major to out:
// lane j forms column j by forward substitution in registers,
// x_i = -sum_{k<i} L[i][k] x_k, x_j = 1, x_i = 0 for i < j.
template <typename T>
__device__ __noinline__ void invert_sub32(const T* blk, int ld, int cw, T* out, int lane) {
  T x[32];
#pragma unroll
  for (int i = 0; i < 32; i++) {
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int k = 0; k + 1 < i; k += 2) {
      a0 += blk[i * ld + k] * x[k];
      a1 += blk[i * ld + k + 1] * x[k + 1];
    }
    if (i & 1) a0 += blk[i * ld + i - 1] * x[i - 1];
    x[i] = (i == lane) ? T(1) : ((i > lane && i < cw) ? -(a0 + a1) : T(0));
  }
#pragma unroll
  for (int i = 0; i < 32; i++) out[i * 32 + lane] = x[i];
}

// X = R L^-T for the rows [0, nrows) of R (shared, row stride ldr, ncols <=
// 32 columns) and the unit lower 32 x 32 block L (shared, row stride ldl;
// only the entries strictly below its diagonal are read, zero beyond
// ncols): blocked forward
// substitution with 8-column groups, four threads per row (thread g holds
// columns 8g..8g+7).  Stage s: group s substitutes with the 8 x 8 diagonal
// block, its 8 values go to the row's other threads by shuffles, and the
// later groups subtract their products with the (g, s) block.  No inverse is
// formed.  Called by all threads of the CTA (blockDim a multiple of 32).
template <typename T>
__device__ __forceinline__ void block_trsm32(T* R, int ldr, int nrows, int ncols, const T* L, int ldl, int t0 = 0,
                                             int nthr = -1) {
  // the threads [t0, t0 + nthr) of the CTA (whole warps; all of them by default)
  if (nthr < 0) nthr = blockDim.x;
  const int t = threadIdx.x - t0;
  const int lane = threadIdx.x & 31, g = threadIdx.x & 3;
  const int src0 = lane & ~3;
  for (int r0 = 0; r0 < nrows; r0 += nthr >> 2) {
    const int row = r0 + (t >> 2);
    const bool act = row < nrows;
    T* rp = R + (act ? row : 0) * ldr + 8 * g;
    T q[8];
#pragma unroll
    for (int t = 0; t < 8; t++) q[t] = (act && 8 * g + t < ncols) ? rp[t] : T(0);
#pragma unroll
    for (int st = 0; st < 4; st++) {
      if (g == st) {
        const T* Ld = L + (8 * st) * ldl + 8 * st;
#pragma unroll
        for (int u = 0; u < 7; u++)
#pragma unroll
          for (int t = u + 1; t < 8; t++) q[t] -= Ld[t * ldl + u] * q[u];
      }
      T xs[8];
#pragma unroll
      for (int u = 0; u < 8; u++) xs[u] = __shfl_sync(0xffffffffu, q[u], src0 | st);
      if (g > st) {
        const T* Lg = L + (8 * g) * ldl + 8 * st;
#pragma unroll
        for (int t = 0; t < 8; t++) {
          T acc = T(0);
#pragma unroll
          for (int u = 0; u < 8; u++) acc += Lg[t * ldl + u] * xs[u];
          q[t] -= acc;
        }
      }
    }
    if (act) {
#pragma unroll
      for (int t = 0; t < 8; t++)
        if (8 * g + t < ncols) rp[t] = q[t];
    }
  }
}

// Copy a tile from shared memory back to global memory (stores where
// keep(r, c)), 8 shared loads in flight per thread before the stores.
template <typename T, typename Keep>
__device__ __forceinline__ void store_tile(T* dst, int64_t ldd, const T* src, int lds, int rows, int cols, Keep keep) {
  const int n = rows * cols;
  for (int base = threadIdx.x; base < n; base += 8 * blockDim.x) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = min(base + k * blockDim.x, n - 1);
      const int r = idx / cols, c = idx - r * cols;
      v[k] = src[r * lds + c];
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = base + k * blockDim.x;
      const int r = idx / cols, c = idx - r * cols;
      if (idx < n && keep(r, c)) dst[(int64_t)r * ldd + c] = v[k];
    }
  }
}

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// barrier among warps 1..7 of a 256-thread CTA (warp 0 is busy meanwhile)
__device__ __forceinline__ void bar_warps_1_7() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

// A[r][c] -= sum_u X[r - rb][u] L21[c][u] (L21 in the columns c0..c0+31 of
// A) for rows [r_begin, w) and columns [c_begin, c_end) (at most 64), c <= r;
// done by the nw warps wfirst.. of the CTA, lane = column, register tiles of
// up to 8 rows per warp and trip
template <typename T, int MRW = 8>
__device__ __forceinline__ void block_update(T* A, int LDM, const T* Xs, int c0, int rb, int w, int r_begin,
                                             int c_begin, int c_end, int wfirst, int nw) {
  const int warp = (threadIdx.x >> 5) - wfirst, lane = threadIdx.x & 31;
  if (warp < 0 || warp >= nw || c_begin >= c_end) return;
  const int ng = (c_end - c_begin + 31) / 32;   // 1 or 2
  for (int rr0 = r_begin + warp * MRW; rr0 < w; rr0 += nw * MRW) {
    T acc[MRW][2];
#pragma unroll
    for (int m = 0; m < MRW; m++) acc[m][0] = acc[m][1] = T(0);
#pragma unroll 2
    for (int u = 0; u < 32; u++) {
      T bv[2];
#pragma unroll
      for (int g = 0; g < 2; g++) bv[g] = g < ng ? A[min(c_begin + 32 * g + lane, c_end - 1) * LDM + c0 + u] : T(0);
#pragma unroll
      for (int m = 0; m < MRW; m++) {
        const T a = Xs[(min(rr0 + m, w - 1) - rb) * LDS + u];
        acc[m][0] += a * bv[0];
        acc[m][1] += a * bv[1];
      }
    }
#pragma unroll
    for (int m = 0; m < MRW; m++) {
      const int r = rr0 + m;
#pragma unroll
      for (int g = 0; g < 2; g++) {
        const int c = c_begin + 32 * g + lane;
        if (g < ng && r < w && c < c_end && c <= r) A[r * LDM + c] -= acc[m][g];
      }
    }
  }
}

// Diagonal role of a macro panel (one CTA of 256 threads): factors the w x w
// diagonal block (w <= 128) in shared memory by 32-column sub-blocks.  For
// sub-block j: the rows below it inside the block are solved by the blocked
// forward substitution, X = F21 L_jj^-T, and scaled, L21 = X D^-1; the next
// sub-block's columns are updated by all warps; then warp 0 factors the
// next sub-block (factor_sub32) while warps 1..7 publish sub-block j (its
// columns and pivots to global memory, fence, release flag j, for the row
// CTAs) and update the columns beyond the next sub-block.  The rows below
// the first sub-block are loaded while warp 0 factors it.  At the end four
// warps invert the four unit lower sub-blocks (for the triangular sweeps).
template <typename T, int MNB>
__device__ __forceinline__ void panel_diag_role(const DevPlan& P, const DevNum<T>& N, int s, int q0, int* flags,
                                                double eps, int policy, unsigned char* smem_raw) {
  constexpr int LDM = MNB + 1;   // shared row stride of the diagonal block
  T* A = reinterpret_cast<T*>(smem_raw);   // w x w block, row stride LDM
  T* Xs = A + MNB * LDM;                   // X of the rows below the sub-block
  T* dsh = Xs + (MNB - 32) * LDS;          // pivots of the block (MNB)
  int8_t* sg = reinterpret_cast<int8_t*>(dsh + MNB);   // block signs, then pivot status
  int8_t* pst = sg + MNB;
  const int ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int w = min(MNB, ncol - q0);
  const int nbk = (w + 31) / 32;
  T* Lb = N.L + P.sn_Loff[s] + (int64_t)q0 * ncp + q0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the first sub-block's rows, then its factorisation by warp 0 while the
  // other warps load the rest of the block
  load_tile(A, LDM, Lb, ncp, min(32, w), MNB, [&](int r, int c) { return c <= r; });
  for (int c = tid; c < MNB; c += blockDim.x) sg[c] = c < w ? P.col_sign[col0 + q0 + c] : 1;
  __syncthreads();
  auto factor = [&](int c0) {
    int8_t st;
    const T d = factor_sub32<T, false>(A + c0 * LDM + c0, LDM, min(32, w - c0), sg[c0 + lane], eps, policy, lane, st);
    dsh[c0 + lane] = d;
    pst[c0 + lane] = st;
  };
  if (warp == 0) {
    factor(0);
  } else if (w > 32) {
    // (eight loads in flight per thread before the shared stores)
    const int n = (w - 32) * MNB;
    for (int base = tid - 32; base < n; base += 8 * 224) {
      T v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int idx = base + k * 224;
        const int r = 32 + idx / MNB, c = idx % MNB;
        v[k] = (idx < n && c <= r) ? Lb[(int64_t)r * ncp + c] : T(0);
      }
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int idx = base + k * 224;
        if (idx < n) A[(32 + idx / MNB) * LDM + idx % MNB] = v[k];
      }
    }
  }
  __syncthreads();
  for (int j = 0; j < nbk; j++) {
    const int c0 = 32 * j, cw = min(32, w - c0);
    const int rb = c0 + 32, nr = w - rb;
    const int nn = min(32, max(nr, 0));   // rows of the next sub-block
    if (nr > 0) {
      // the critical path: only the next sub-block's rows are solved,
      // X = F21 L_jj^-T (kept), L21 = X D^-1, and its diagonal block updated
      block_trsm32<T>(A + rb * LDM + c0, LDM, nn, 32, A + c0 * LDM + c0, LDM);
      __syncthreads();
      for (int idx = tid; idx < nn * 32; idx += blockDim.x) {
        const int r = idx >> 5, c = idx & 31;
        const T x = A[(rb + r) * LDM + c0 + c];
        Xs[r * LDS + c] = x;
        A[(rb + r) * LDM + c0 + c] = x * pivot_rcp(dsh[c0 + c]);
      }
      __syncthreads();
      block_update<T, 4>(A, LDM, Xs, c0, rb, rb + nn, rb, rb, rb + nn, 0, 8);   // 32 rows: 4 per warp
      __syncthreads();
    }
    if (warp == 0) {
      if (j + 1 < nbk) factor(rb);
    } else {
      // warps 1..7, while warp 0 factors the next sub-block: the remaining
      // rows below it, the publication of sub-block j (columns [c0, c0 + cw)
      // of rows [c0, w), pivots; one fence after the warps' barrier, then
      // the release flag) and the rest of sub-block j's update
      if (nr > 32) {
        block_trsm32<T>(A + (rb + 32) * LDM + c0, LDM, nr - 32, 32, A + c0 * LDM + c0, LDM, 32, 224);
        bar_warps_1_7();
        for (int idx = tid - 32; idx < (nr - 32) * 32; idx += 224) {
          const int r = 32 + (idx >> 5), c = idx & 31;
          const T x = A[(rb + r) * LDM + c0 + c];
          Xs[r * LDS + c] = x;
          A[(rb + r) * LDM + c0 + c] = x * pivot_rcp(dsh[c0 + c]);
        }
        bar_warps_1_7();
      }
      const int n = (w - c0) * cw;
      for (int idx = tid - 32; idx < n; idx += 224) {
        const int r = idx / cw, c = idx - r * cw;
        if (c <= r) Lb[(int64_t)(c0 + r) * ncp + c0 + c] = A[(c0 + r) * LDM + c0 + c];
      }
      if (tid - 32 < cw) N.D[col0 + q0 + c0 + tid - 32] = dsh[c0 + tid - 32];
      bar_warps_1_7();
      if (tid == 32) {
        __threadfence();
        st_release_i32(flags + j, 1);
      }
      if (nr > 32) {
        // (block_update covers at most 64 columns per call)
        for (int cb = rb; cb < w; cb += 64) block_update<T>(A, LDM, Xs, c0, rb, w, rb + 32, cb, min(cb + 64, w), 1, 7);
      }
    }
    __syncthreads();
  }
  // (the inverses of the unit lower diagonal sub-blocks, which only the
  // triangular sweeps use, are formed by one launch after the factorisation)
  for (int c = tid; c < w; c += blockDim.x) N.piv[col0 + q0 + c] = pst[c];
}

// Row role of a macro panel (one CTA of 256 threads per RB rows below it): stages its rows
// while the diagonal role works, then for each 32-column sub-block j, as
// soon as it is published, X_j = R_j L_jj^-T by the blocked forward
// substitution and R_i -= X_j L_ij^T for the later sub-blocks (lane =
// column, the rows of a warp in registers); finally L21 = X D1^-1, and for a
// tensor-core front the split TF32 operands of L21 and of W = L21 D1 = X.
template <typename T, int MNB>
__device__ __forceinline__ void panel_rows_role(const DevPlan& P, const DevNum<T>& N, int s, int q0, int r0,
                                                const int* flags, int* err, long long wait,
                                                unsigned char* smem_raw) {
  constexpr int LDM = MNB + 1;
  constexpr int KB = MNB / 32;             // sub-blocks of the panel
  T* R = reinterpret_cast<T*>(smem_raw);   // RB rows x w columns, stride LDM
  T* Ld = R + RB * LDM;                    // the KB unit lower diagonal sub-blocks of L11
  T* Lo = Ld + KB * 32 * LDS;              // the KB (KB - 1) / 2 off-diagonal sub-blocks (i > j) of L11
  T* dsh = Lo + (KB * (KB - 1) / 2) * 32 * LDS;   // D1
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int w = min(MNB, ncol - q0);
  const int nbk = (w + 31) / 32;
  const int nr = min(RB, nrow - r0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T* Lb = N.L + P.sn_Loff[s];
  load_tile(R, LDM, Lb + (int64_t)r0 * ncp + q0, ncp, RB, MNB, [&](int r, int c) { return r < nr && c < w; });
  constexpr int KR = RB / 8;   // rows per warp in the updates (lane = column)
  T* Rw = R + warp * LDM;      // row warp + 8 k is Rw[8 k LDM + ...]
  for (int j = 0; j < nbk; j++) {
    // wait (bounded) for sub-block j, then fetch its published columns
    if (tid == 0) {
      if (!ld_acquire_i32(flags + j) && !ld_acquire_i32(err)) {
        const long long t0 = clock64();
        while (!ld_acquire_i32(flags + j)) {
          if (clock64() - t0 > wait || ld_acquire_i32(err)) {
            atomicExch(err, 1);
            break;
          }
          __nanosleep(64);
        }
      }
    }
    __syncthreads();
    {
      // the published blocks (i, j), i >= j, and D_j: every load in flight
      // before the shared stores (256 threads, four entries of each block)
      T v[KB][4];
#pragma unroll
      for (int q = 0; q < KB; q++) {
        const int i = j + q;
        const int rows = min(32, w - 32 * i);
        const T* src = Lb + (int64_t)(q0 + 32 * i) * ncp + q0 + 32 * j;
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int e = tid + 256 * t, rr = e >> 5, cc = e & 31;
          v[q][t] = (i < nbk && rr < rows && (i > j || cc < rr)) ? __ldcg(src + (int64_t)rr * ncp + cc) : T(0);
        }
      }
      const T dv = (tid < 32 && 32 * j + tid < w) ? __ldcg(N.D + col0 + q0 + 32 * j + tid) : T(1);
#pragma unroll
      for (int q = 0; q < KB; q++) {
        const int i = j + q;
        if (i >= nbk) break;
        T* dst = (i == j) ? Ld + i * 32 * LDS : Lo + (i * (i - 1) / 2 + j) * 32 * LDS;
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int e = tid + 256 * t;
          dst[(e >> 5) * LDS + (e & 31)] = v[q][t];
        }
      }
      if (tid < 32) dsh[32 * j + tid] = dv;
    }
    __syncthreads();
    block_trsm32<T>(R + 32 * j, LDM, nr, min(32, w - 32 * j), Ld + j * 32 * LDS, LDS);
    __syncthreads();
    for (int i = j + 1; i < nbk; i++) {
      const T* lij = Lo + (i * (i - 1) / 2 + j) * 32 * LDS;
      T x[KR];
#pragma unroll
      for (int k = 0; k < KR; k++) x[k] = T(0);
#pragma unroll 4
      for (int u = 0; u < 32; u++) {
        const T b = lij[lane * LDS + u];
#pragma unroll
        for (int k = 0; k < KR; k++) x[k] += Rw[8 * k * LDM + 32 * j + u] * b;
      }
#pragma unroll
      for (int k = 0; k < KR; k++) Rw[8 * k * LDM + 32 * i + lane] -= x[k];
    }
    __syncthreads();
  }
  // L21 = X D1^-1 (+ split operands of L21 and W = X for a tensor-core front)
  int64_t so = -1;
  if constexpr (sizeof(T) == 4) so = (N.S && P.sn_Soff) ? P.sn_Soff[s] : -1;
  const int64_t plane = (int64_t)nrow * ncp;
  const int cend = (q0 + w == ncol) ? ncp - q0 : w;   // the last panel also clears the padding columns
  for (int j = 0; 32 * j < cend; j++) {
    const int c = 32 * j + lane;
    if (c >= cend) continue;
    const T invd = c < w ? T(1) / dsh[c] : T(0);
#pragma unroll
    for (int k = 0; k < KR; k++) {
      const int r = warp + 8 * k;
      if (r >= nr) continue;
      const T xv = c < w ? R[r * LDM + c] : T(0);
      const T l = xv * invd;
      if (c < w) Lb[(int64_t)(r0 + r) * ncp + q0 + c] = l;
      if constexpr (sizeof(T) == 4) {
        if (so >= 0) {
          float* sp = N.S + so + (int64_t)(r0 + r) * ncp + q0 + c;
          const float lh = tf32_round(l), wh = tf32_round(xv);
          sp[0] = lh;
          sp[plane] = tf32_round(l - lh);
          sp[2 * plane] = wh;
          sp[3 * plane] = tf32_round(xv - wh);
        }
      }
    }
  }
}

}  // namespace ncl
