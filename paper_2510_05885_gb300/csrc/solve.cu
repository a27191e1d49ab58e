// Triangular solves, FP64 residual and adjoint kernels (sm_103a).
//
// Solve with the supernodal factors of P K P^T = L D L^T:
//   forward  L y = P b   leaves to root, level by level,
//   diagonal z = D^-1 y,
//   backward L^T w = z   root to leaves,   x = P^T w.
// Forward updates flow to ancestors through per-supernode update vectors
// W_s = (rows below s) - L21 y_s, pulled by the parent in a fixed order
// (no atomics, bitwise reproducible).  The FP64 residual r = b - K x is
// computed on the FP64 KKT values for iterative refinement (Section 4.3).
#include "runtime.h"
#include "reduce.cuh"

#include <algorithm>

namespace ncl {

// ---------------------------------------------------------------------------
// permutations
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_perm_in(DevPlan P, T* __restrict__ xp, const double* __restrict__ B, int64_t ldb, int nrhs) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.dim; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t src = P.perm[k];
    for (int r = 0; r < nrhs; r++) xp[r * P.dim + k] = (T)B[r * ldb + src];
  }
}

template <typename T>
__global__ void k_perm_out(DevPlan P, const T* __restrict__ xp, double* __restrict__ X, int64_t ldx, int nrhs,
                           int accumulate) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.dim; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t dst = P.perm[k];
    for (int r = 0; r < nrhs; r++) {
      const double v = (double)xp[r * P.dim + k];
      if (accumulate) X[r * ldx + dst] += v;
      else X[r * ldx + dst] = v;
    }
  }
}

static unsigned grid_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T>
void launch_perm_in(const DevPlan& P, T* xp, const double* B, int64_t ldb, int nrhs, cudaStream_t st) {
  if (P.dim) k_perm_in<T><<<grid_for(P.dim), 256, 0, st>>>(P, xp, B, ldb, nrhs);
}
template <typename T>
void launch_perm_out(const DevPlan& P, const T* xp, double* X, int64_t ldx, int nrhs, int acc, cudaStream_t st) {
  if (P.dim) k_perm_out<T><<<grid_for(P.dim), 256, 0, st>>>(P, xp, X, ldx, nrhs, acc);
}

// ---------------------------------------------------------------------------
// Pivot blocks of the sweeps, chained over 128-row block-rows.
//
// Every supernode's pivot block L11 is cut into block-rows of CHAIN_ROWS =
// 128 rows, one CTA (4 warps) each; warp w owns the block-row's 32-row
// sub-block w.  A CTA takes its block-row from the supernode's ticket
// counter, in order, so every block-row it waits for belongs to a CTA that is
// already running: the waits cannot deadlock, whatever the order in which
// CTAs are scheduled.  Waits are bounded: past the limit the CTA sets the
// sweep's error flag, goes on with what it has and still publishes, so that
// nobody waits on it; the host then reports the sweep as failed.
//   forward:  y_B = L_BB^-1 (t_B - sum_{J<B} L_BJ y_J),
//             t_B = the block-row's right-hand side plus the children's updates;
//   backward: x_B = L_BB^-T (z_B - sum_{I>B} L_IB^T x_I),
//             z_B = D^-1 y_B - the partial sums of L21^T x of the rows below.
// The sums over published block-rows are formed by every warp for its rows
// (lane = row, the published values by shuffles); the diagonal block-row
// L_BB is then solved inside the CTA sub-block by sub-block with the
// inverted 32 x 32 diagonal blocks, its strictly lower part staged in shared
// memory while the CTA waits (only when it has more than one sub-block).
// Levels whose supernodes all have a single block-row launch the
// instantiation without the cross-block-row part (MULTI = false), which
// needs far fewer registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// lane 0 waits (bounded by `limit` clock cycles) for the flag; the warp then
// proceeds together.  err is the sweep's error flag: once set, nobody waits
// any more.
__device__ __forceinline__ void chain_wait(const int* flag, int* err, long long limit) {
  if ((threadIdx.x & 31) == 0 && !ld_acquire(flag) && !ld_acquire(err)) {
    const long long t0 = clock64();
    while (!ld_acquire(flag)) {
      if (clock64() - t0 > limit || ld_acquire(err)) {
        atomicExch(err, 1);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncwarp();
}

// after a CTA barrier: thread 0 publishes the CTA's results (the release
// store orders every write the barrier made visible to thread 0 before the
// flag, so no separate fence is needed)
__device__ __forceinline__ void chain_publish(int* flag) {
  if (threadIdx.x == 0) st_release(flag, 1);
}

int chain_smem(int rows, int esz) {
  return (rows * (rows + 1) + 2 * MAX_RHS_SWEEP * (CHAIN_ROWS + 1) + ((rows + 31) / 32) * 32 * 33) * esz;
}

// strictly lower part of the diagonal block-row tile (rows and columns
// [R0, R0 + nr)) into shared memory, row stride nr + 1
template <typename T>
__device__ __forceinline__ void chain_stage_tile(T* Ls, const T* Lb, int64_t ncp, int R0, int nr) {
  const int n = nr * nr, ld = nr + 1;
  for (int base = threadIdx.x; base < n; base += 8 * blockDim.x) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = base + k * blockDim.x;
      const int i = idx / nr, c = idx - i * nr;
      v[k] = (idx < n && c < i) ? Lb[(int64_t)(R0 + i) * ncp + R0 + c] : T(0);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int idx = base + k * blockDim.x;
      const int i = idx / nr, c = idx - i * nr;
      if (idx < n) Ls[i * ld + c] = v[k];
    }
  }
}

template <typename T, bool MULTI>
__global__ void __launch_bounds__(128) k_fwd_chain(DevPlan P, DevNum<T> N, const int4* __restrict__ items,
                                                   const int32_t* __restrict__ pptr, const int4* __restrict__ pran,
                                                   T* __restrict__ xp, const T* __restrict__ W, int nrhs,
                                                   int* tickets, int* flags, int* err, long long wait) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sb;
  const int4 it = items[blockIdx.x];
  const int s = it.x, broff = it.y, boff = it.z;
  if (threadIdx.x == 0) sb = atomicAdd(&tickets[s], 1);
  __syncthreads();
  const int B = sb;
  const int ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int R0 = CHAIN_ROWS * B, nr = min(CHAIN_ROWS, ncol - R0), nsub = (nr + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ldt = nr + 1;
  T* Ls = reinterpret_cast<T*>(smem_raw);              // nr x nr, strictly lower
  T* tb = Ls + nr * ldt;                               // [MAX_RHS_SWEEP][CHAIN_ROWS + 1]
  T* ys = tb + MAX_RHS_SWEEP * (CHAIN_ROWS + 1);
  T* Iv = ys + MAX_RHS_SWEEP * (CHAIN_ROWS + 1);      // the inverted 32 x 32 diagonal blocks, stride 33
  const T* Lb = N.L + P.sn_Loff[s];
  if (nsub > 1) chain_stage_tile(Ls, Lb, ncp, R0, nr);
  const int rw = 32 * warp + lane;                     // this lane's row in the block-row
  const bool mine = warp < nsub;
  const bool valid = rw < nr;
  if (mine) {
    // the inverted diagonal block of this warp's sub-block (for the end)
    const T* ip = N.Linv + P.sn_Ioff[s] + (int64_t)(4 * B + warp) * 1024;
    T* iw = Iv + warp * 32 * 33;
#pragma unroll 8
    for (int i = 0; i < 32; i++) iw[i * 33 + lane] = ip[i * 32 + lane];
    // t: the rows' entries plus the children's updates, child by child
#pragma unroll
    for (int r = 0; r < MAX_RHS_SWEEP; r++)
      tb[r * (CHAIN_ROWS + 1) + rw] = (r < nrhs && valid) ? xp[(int64_t)r * P.dim + col0 + R0 + rw] : T(0);
    __syncwarp();
    const int k = 4 * B + warp;
    for (int e = pptr[boff + k]; e < pptr[boff + k + 1]; e++) {
      const int4 pr = pran[e];
      const int c = pr.x;
      const int32_t* rel = P.relmap + P.relmap_off[c];
      for (int a = pr.y + lane; a < pr.z; a += 32)
        for (int r = 0; r < nrhs; r++) tb[r * (CHAIN_ROWS + 1) + rel[a] - R0] += W[r * P.Wtot + P.sn_Woff[c] + a];
      __syncwarp();
    }
  }
  // sum over the published block-rows J < B (all 128 columns of J exist):
  // the warp reads its 32 rows 32 columns at a time (one coalesced segment
  // per row; the next segment is loaded before the current one is used and
  // before waiting for its block-row), and a butterfly reduce-scatter leaves
  // row rr's sum in lane rr.  Once J is published, its 128 values are loaded
  // together.  (Levels whose supernodes all have one block-row compile
  // without this part.)
  T acc[MAX_RHS_SWEEP];
#pragma unroll
  for (int r = 0; r < MAX_RHS_SWEEP; r++) acc[r] = T(0);
  if (MULTI && mine && B > 0) {
    const T* wrow = Lb + (int64_t)(R0 + 32 * warp) * ncp + lane;
    const int nrw = min(32, nr - 32 * warp);
    // FP32: two chunks in flight ahead of the one in use, so that after the
    // wait for a block-row its first two chunks are already in registers
    // (FP64: one, for registers)
    constexpr bool PF2 = sizeof(T) == 4;
    T lv[32], ln[32], ln2[32];
    const int nchunk = 4 * B;
#pragma unroll
    for (int rr = 0; rr < 32; rr++) ln[rr] = rr < nrw ? wrow[(int64_t)rr * ncp] : T(0);
    if (PF2) {
#pragma unroll
      for (int rr = 0; rr < 32; rr++) ln2[rr] = rr < nrw ? wrow[(int64_t)rr * ncp + 32] : T(0);
    }
    // the right-hand sides of the four chunks of a block-row, loaded
    // together once it is published and rotated chunk by chunk (FP64: the
    // first right-hand side only, for registers)
    constexpr int YQ = sizeof(T) == 4 ? MAX_RHS_SWEEP : 1;
    T yq[4][YQ];
    for (int q = 0; q < nchunk; q++) {
      const int c0 = 32 * q;
      if (PF2) {
#pragma unroll
        for (int rr = 0; rr < 32; rr++) {
          lv[rr] = ln[rr];
          ln[rr] = ln2[rr];
        }
        if (q + 2 < nchunk) {
#pragma unroll
          for (int rr = 0; rr < 32; rr++) ln2[rr] = rr < nrw ? wrow[(int64_t)rr * ncp + c0 + 64] : T(0);
        }
      } else {
#pragma unroll
        for (int rr = 0; rr < 32; rr++) lv[rr] = ln[rr];
        if (q + 1 < nchunk) {
#pragma unroll
          for (int rr = 0; rr < 32; rr++) ln[rr] = rr < nrw ? wrow[(int64_t)rr * ncp + c0 + 32] : T(0);
        }
      }
      if ((q & 3) == 0) {
        chain_wait(flags + broff + (q >> 2), err, wait);
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
          for (int r = 0; r < YQ; r++)
            yq[c][r] = r < nrhs ? __ldcg(xp + (int64_t)r * P.dim + col0 + c0 + 32 * c + lane) : T(0);
      }
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        const T yu = r < YQ ? yq[0][r] : __ldcg(xp + (int64_t)r * P.dim + col0 + c0 + lane);
        T v[32];
#pragma unroll
        for (int rr = 0; rr < 32; rr++) v[rr] = lv[rr] * yu;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          const bool upper = (lane & o) != 0;
#pragma unroll
          for (int k = 0; k < o; k++) {
            const T send = upper ? v[k] : v[k + o];
            const T recv = __shfl_xor_sync(0xffffffffu, send, o);
            v[k] = (upper ? v[k + o] : v[k]) + recv;
          }
        }
        acc[r] += v[0];
      }
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int r = 0; r < YQ; r++) yq[c][r] = yq[c + 1][r];
    }
  }
  __syncthreads();
  // the diagonal block-row, sub-block by sub-block
  for (int w2 = 0; w2 < nsub; w2++) {
    if (warp == w2) {
      const T* iw = Iv + warp * 32 * 33 + lane * 33;   // row lane of the inverted block
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        const T z = valid ? tb[r * (CHAIN_ROWS + 1) + rw] - acc[r] : T(0);
        T v = T(0);
#pragma unroll
        for (int u = 0; u < 32; u++) v += iw[u] * __shfl_sync(0xffffffffu, z, u);
        ys[r * (CHAIN_ROWS + 1) + rw] = valid ? v : T(0);
        if (valid) xp[(int64_t)r * P.dim + col0 + R0 + rw] = v;
      }
    }
    __syncthreads();
    if (warp > w2 && mine) {
      const T* lr = Ls + min(rw, nr - 1) * ldt + 32 * w2;
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        const T* y = ys + r * (CHAIN_ROWS + 1) + 32 * w2;
        T a = T(0);
#pragma unroll 8
        for (int u = 0; u < 32; u++) a += lr[u] * y[u];
        acc[r] += a;
      }
    }
  }
  chain_publish(flags + broff + B);
}

template <typename T, bool MULTI>
__global__ void __launch_bounds__(128) k_bwd_chain(DevPlan P, DevNum<T> N, const int4* __restrict__ items,
                                                   T* __restrict__ xp, const T* __restrict__ Pw, int nrhs,
                                                   int* tickets, int* flags, int* err, long long wait) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sb;
  const int4 it = items[blockIdx.x];
  const int s = it.x, broff = it.y;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int nbr = (ncol + CHAIN_ROWS - 1) / CHAIN_ROWS;
  if (threadIdx.x == 0) sb = nbr - 1 - atomicAdd(&tickets[s], 1);
  __syncthreads();
  const int B = sb;
  const int R0 = CHAIN_ROWS * B, nr = min(CHAIN_ROWS, ncol - R0), nsub = (nr + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ldt = nr + 1;
  T* Ls = reinterpret_cast<T*>(smem_raw);
  T* zb = Ls + nr * ldt;
  T* xs = zb + MAX_RHS_SWEEP * (CHAIN_ROWS + 1);
  T* Iv = xs + MAX_RHS_SWEEP * (CHAIN_ROWS + 1);      // the inverted 32 x 32 diagonal blocks, stride 33
  const T* Lb = N.L + P.sn_Loff[s];
  if (nsub > 1) chain_stage_tile(Ls, Lb, ncp, R0, nr);
  const int rw = 32 * warp + lane;                     // this lane's column (unknown) in the block-row
  const bool mine = warp < nsub;
  const bool valid = rw < nr;
  if (mine) {
    // the inverted diagonal block of this warp's sub-block (for the end)
    const T* ip = N.Linv + P.sn_Ioff[s] + (int64_t)(4 * B + warp) * 1024;
    T* iw = Iv + warp * 32 * 33;
#pragma unroll 8
    for (int i = 0; i < 32; i++) iw[i * 33 + lane] = ip[i * 32 + lane];
    // z = D^-1 y - the partial sums of the rows below
    const int nb = nrow - ncol, nch = (nb + SOLVE_ROWS - 1) / SOLVE_ROWS;
    const T dk = valid ? N.D[col0 + R0 + rw] : T(1);
    for (int r = 0; r < MAX_RHS_SWEEP; r++) {
      T z = T(0);
      if (r < nrhs && valid) {
        z = xp[(int64_t)r * P.dim + col0 + R0 + rw] / dk;
        for (int ch = 0; ch < nch; ch++) z -= Pw[r * P.Ptot + P.sn_Poff[s] + (int64_t)ch * ncol + R0 + rw];
      }
      zb[r * (CHAIN_ROWS + 1) + rw] = z;
    }
  }
  // sum over the published block-rows I > B: L_IB^T x_I (lane = column);
  // once I is published, its values are loaded together.  (Levels whose
  // supernodes all have one block-row compile without this part.)
  T acc[MAX_RHS_SWEEP];
#pragma unroll
  for (int r = 0; r < MAX_RHS_SWEEP; r++) acc[r] = T(0);
  if (MULTI && mine && B < nbr - 1) {
    // chunks q = 0, 1, ...: 32 rows of block-row I = nbr - 1 - q / 4, the
    // next chunk loaded before the current one is used and before waiting
    const T* lcol = Lb + R0 + min(rw, nr - 1);
    const int nchunk = 4 * (nbr - 1 - B);
    auto rows_of = [&](int q, int& q0, int& bwi) {
      const int I = nbr - 1 - (q >> 2);
      q0 = CHAIN_ROWS * I + 32 * (q & 3);
      bwi = max(0, min(32, ncol - q0));
    };
    // FP32: two chunks in flight ahead of the one in use (FP64: one, for registers)
    constexpr bool PF2 = sizeof(T) == 4;
    T lv[32], ln[32], ln2[32];
    int nq0, nbw, nq2 = 0, nbw2 = 0;
    rows_of(0, nq0, nbw);
#pragma unroll
    for (int v = 0; v < 32; v++) ln[v] = v < nbw ? lcol[(int64_t)(nq0 + v) * ncp] : T(0);
    if (PF2 && nchunk > 1) {
      rows_of(1, nq2, nbw2);
#pragma unroll
      for (int v = 0; v < 32; v++) ln2[v] = v < nbw2 ? lcol[(int64_t)(nq2 + v) * ncp] : T(0);
    }
    // the values of the four chunks of a block-row, loaded together once it
    // is published and rotated chunk by chunk (FP64: the first right-hand
    // side only, for registers)
    constexpr int XQ = sizeof(T) == 4 ? MAX_RHS_SWEEP : 1;
    T xq[4][XQ];
    for (int q = 0; q < nchunk; q++) {
      const int q0 = nq0, bwi = nbw;
      if (PF2) {
#pragma unroll
        for (int v = 0; v < 32; v++) {
          lv[v] = ln[v];
          ln[v] = ln2[v];
        }
        nq0 = nq2;
        nbw = nbw2;
        if (q + 2 < nchunk) {
          rows_of(q + 2, nq2, nbw2);
#pragma unroll
          for (int v = 0; v < 32; v++) ln2[v] = v < nbw2 ? lcol[(int64_t)(nq2 + v) * ncp] : T(0);
        }
      } else {
#pragma unroll
        for (int v = 0; v < 32; v++) lv[v] = ln[v];
        if (q + 1 < nchunk) {
          rows_of(q + 1, nq0, nbw);
#pragma unroll
          for (int v = 0; v < 32; v++) ln[v] = v < nbw ? lcol[(int64_t)(nq0 + v) * ncp] : T(0);
        }
      }
      if ((q & 3) == 0) {
        chain_wait(flags + broff + nbr - 1 - (q >> 2), err, wait);
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const int bw = max(0, min(32, ncol - (q0 + 32 * c)));
#pragma unroll
          for (int r = 0; r < XQ; r++)
            xq[c][r] = (r < nrhs && lane < bw) ? __ldcg(xp + (int64_t)r * P.dim + col0 + q0 + 32 * c + lane) : T(0);
        }
      }
      if (bwi > 0) {
#pragma unroll
        for (int r = 0; r < MAX_RHS_SWEEP; r++) {
          if (r >= nrhs) break;
          const T xv = r < XQ ? xq[0][r]
                              : (lane < bwi ? __ldcg(xp + (int64_t)r * P.dim + col0 + q0 + lane) : T(0));
#pragma unroll
          for (int v = 0; v < 32; v++) acc[r] += lv[v] * __shfl_sync(0xffffffffu, xv, v);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int r = 0; r < XQ; r++) xq[c][r] = xq[c + 1][r];
    }
  }
  __syncthreads();
  // the diagonal block-row, sub-block by sub-block from the last
  for (int w2 = nsub - 1; w2 >= 0; w2--) {
    if (warp == w2) {
      const T* iw = Iv + warp * 32 * 33 + lane;        // column lane of the inverted block
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        const T w = valid ? zb[r * (CHAIN_ROWS + 1) + rw] - acc[r] : T(0);
        T v = T(0);
#pragma unroll
        for (int q = 0; q < 32; q++) v += iw[q * 33] * __shfl_sync(0xffffffffu, w, q);
        xs[r * (CHAIN_ROWS + 1) + rw] = valid ? v : T(0);
        if (valid) xp[(int64_t)r * P.dim + col0 + R0 + rw] = v;
      }
    }
    __syncthreads();
    if (warp < w2) {
      // acc[col rw] += sum_v L[32 w2 + v][rw] x[32 w2 + v]
      const int nv = min(32, nr - 32 * w2);
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        const T* x = xs + r * (CHAIN_ROWS + 1) + 32 * w2;
        T a = T(0);
        for (int v = 0; v < nv; v++) a += Ls[(32 * w2 + v) * ldt + rw] * x[v];
        acc[r] += a;
      }
    }
  }
  chain_publish(flags + broff + B);
}

// 16-byte vectors of factor entries (rows of L start 16-byte aligned: the
// blocks start at multiples of 32 elements and the row stride is a multiple
// of 4 elements)
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

// forward: rows below supernode s, SOLVE_ROWS per CTA:
//   W_s[a] = (children's updates landing on row a) - L21[a,:] y_s
// The products use tpr = 4..32 threads per row (by the supernode's width),
// each reading 16-byte vectors of its row, and RPT rows per thread at a time,
// so that a narrow supernode still has many loads in flight; the partial
// sums are reduced by shuffles inside each group of tpr lanes.
template <typename T>
__global__ void __launch_bounds__(256) k_fwd_below(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                   const int32_t* __restrict__ cptr, const int4* __restrict__ cran,
                                                   const T* __restrict__ xp, T* __restrict__ W, int nrhs) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
  constexpr int RPT = 4;
  __shared__ T t[SOLVE_ROWS * 8];
  const int2 it = items[blockIdx.x];
  const int s = it.x, a0 = it.y;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int nb = nrow - ncol;
  const int a1 = min(a0 + SOLVE_ROWS, nb);
  const T* Lb = N.L + P.sn_Loff[s];
  for (int idx = threadIdx.x; idx < SOLVE_ROWS * nrhs; idx += blockDim.x) t[idx] = T(0);
  __syncthreads();
  // children's updates landing on these rows (ranges found on the host),
  // child by child
  for (int e = cptr[blockIdx.x]; e < cptr[blockIdx.x + 1]; e++) {
    const int4 cr = cran[e];
    const int c = cr.x;
    const int32_t* rel = P.relmap + P.relmap_off[c];
    for (int a = cr.y + threadIdx.x; a < cr.z; a += blockDim.x)
      for (int r = 0; r < nrhs; r++) t[r * SOLVE_ROWS + rel[a] - ncol - a0] += W[r * P.Wtot + P.sn_Woff[c] + a];
    __syncthreads();
  }
  const int nv = (ncol + VW - 1) / VW;                 // vectors per row
  int tpr = 4;
  while (tpr < 32 && 2 * tpr < nv) tpr *= 2;
  const int q = threadIdx.x & (tpr - 1);
  const int slots = blockDim.x / tpr, slot = threadIdx.x / tpr;
  const int64_t ysz = (int64_t)P.dim;
  // every thread runs the same number of passes (the shuffles below are
  // warp-wide)
  for (int base = a0; base < a1; base += RPT * slots) {
    int ar[RPT];
    bool ok[RPT];
#pragma unroll
    for (int j = 0; j < RPT; j++) {
      ar[j] = base + j * slots + slot;
      ok[j] = ar[j] < a1;
    }
    T acc[RPT][MAX_RHS_SWEEP];
#pragma unroll
    for (int j = 0; j < RPT; j++)
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) acc[j][r] = T(0);
    for (int v = q; v < nv; v += tpr) {
      V lv[RPT];
#pragma unroll
      for (int j = 0; j < RPT; j++) {
        if (ok[j]) lv[j] = __ldg(reinterpret_cast<const V*>(Lb + (int64_t)(ncol + ar[j]) * ncp) + v);
        else lv[j] = V{};
      }
#pragma unroll
      for (int e = 0; e < VW; e++) {
        const int k = v * VW + e;
        if (k >= ncol) break;
#pragma unroll
        for (int r = 0; r < MAX_RHS_SWEEP; r++) {
          if (r >= nrhs) break;
          const T y = __ldg(xp + r * ysz + col0 + k);
#pragma unroll
          for (int j = 0; j < RPT; j++) acc[j][r] += reinterpret_cast<const T*>(&lv[j])[e] * y;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < RPT; j++) {
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) {
        if (r >= nrhs) break;
        T a = acc[j][r];
        for (int o = tpr >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (q == 0 && ok[j]) W[r * P.Wtot + P.sn_Woff[s] + ar[j]] = t[r * SOLVE_ROWS + ar[j] - a0] - a;
      }
    }
  }
}

// backward: partial sums of L21^T x_below over a run of SOLVE_ROWS rows and
// a run of up to 256 columns (item (s, a0, k0)).  The level's first `narrow`
// items (supernodes of at most 32 columns) take one warp each, eight to a
// CTA (lane = column, the rows in order); the others one CTA each, where
// for 33..128 columns G = 256 / (columns rounded up to 32) groups of threads
// split the rows and their sums are added in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_below(DevPlan P, DevNum<T> N, const int4* __restrict__ items,
                                                   int narrow, const T* __restrict__ xp, T* __restrict__ Pw,
                                                   int nrhs) {
  __shared__ T xb[SOLVE_ROWS * MAX_RHS_SWEEP];
  __shared__ T red[256];
  const int nnc = (narrow + 7) / 8;   // CTAs of the narrow items
  if ((int)blockIdx.x < nnc) {
    __shared__ T xw[8][SOLVE_ROWS * MAX_RHS_SWEEP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + w;
    if (i >= narrow) return;   // the whole warp; no CTA barrier in this branch
    const int4 it = items[i];
    const int s = it.x, a0 = it.y;
    const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
    const int nb = nrow - ncol;
    const int a1 = min(a0 + SOLVE_ROWS, nb), na = a1 - a0;
    const int chunk = a0 / SOLVE_ROWS;
    const int32_t* rows = P.sn_rows + P.sn_rows_off[s] + ncol;
    T* x = xw[w];
    for (int idx = lane; idx < na * nrhs; idx += 32) {
      const int r = idx / na, a = idx - r * na;
      x[r * SOLVE_ROWS + a] = xp[r * P.dim + rows[a0 + a]];
    }
    __syncwarp();
    const T* col = N.L + P.sn_Loff[s] + (int64_t)ncol * ncp + min(lane, ncol - 1);
    for (int r = 0; r < nrhs; r++) {
      const T* xr = x + r * SOLVE_ROWS - a0;
      T acc = T(0);
      if (lane < ncol) {
#pragma unroll 16
        for (int a = a0; a < a1; a++) acc += col[(int64_t)a * ncp] * xr[a];
        Pw[r * P.Ptot + P.sn_Poff[s] + (int64_t)chunk * ncol + lane] = acc;
      }
    }
    return;
  }
  const int4 it = items[narrow + (blockIdx.x - nnc)];
  const int s = it.x, a0 = it.y, k0 = it.z;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
  const int nb = nrow - ncol;
  const int a1 = min(a0 + SOLVE_ROWS, nb);
  const int chunk = a0 / SOLVE_ROWS;
  const int kc = min(256, ncol - k0);
  const T* Lb = N.L + P.sn_Loff[s];
  const int32_t* rows = P.sn_rows + P.sn_rows_off[s] + ncol;
  for (int idx = threadIdx.x; idx < (a1 - a0) * nrhs; idx += blockDim.x) {
    const int r = idx / (a1 - a0), a = idx % (a1 - a0);
    xb[r * SOLVE_ROWS + a] = xp[r * P.dim + rows[a0 + a]];
  }
  __syncthreads();
  // G thread groups of blockDim / G >= kc threads each
  const int cols = (kc + 31) & ~31;
  const int G = (cols > 128 || cols <= 32) ? 1 : blockDim.x / cols;
  const int tpg = blockDim.x / G, g = threadIdx.x / tpg, kl = threadIdx.x - g * tpg;
  const int per = (a1 - a0 + G - 1) / G;
  const int ga0 = a0 + g * per, ga1 = min(a1, ga0 + per);
  const T* col = Lb + (int64_t)ncol * ncp + k0 + min(kl, kc - 1);
  for (int r = 0; r < nrhs; r++) {
    const T* x = xb + r * SOLVE_ROWS - a0;
    T acc = T(0);
    if (kl < kc) {
#pragma unroll 16
      for (int a = ga0; a < ga1; a++) acc += col[(int64_t)a * ncp] * x[a];
    }
    T* out = Pw + r * P.Ptot + P.sn_Poff[s] + (int64_t)chunk * ncol + k0;
    if (G == 1) {
      if (kl < kc) out[kl] = acc;
    } else {
      red[g * tpg + kl] = acc;
      __syncthreads();
      if (threadIdx.x < kc) {
        T t = T(0);
        for (int q = 0; q < G; q++) t += red[q * tpg + threadIdx.x];
        out[threadIdx.x] = t;
      }
      __syncthreads();
    }
  }
}

template <typename T>
void launch_fwd_chain(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int smem, bool multi,
                      const int32_t* pptr, const int4* pran, T* xp, const T* W, int nrhs, int* tickets, int* flags,
                      int* err, long long wait, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fwd_chain<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         chain_smem(CHAIN_ROWS, sizeof(T)));
    cudaFuncSetAttribute(k_fwd_chain<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         chain_smem(CHAIN_ROWS, sizeof(T)));
    attr = true;
  }
  if (multi)
    k_fwd_chain<T, true><<<count, 128, smem, st>>>(P, N, items, pptr, pran, xp, W, nrhs, tickets, flags, err, wait);
  else
    k_fwd_chain<T, false><<<count, 128, smem, st>>>(P, N, items, pptr, pran, xp, W, nrhs, tickets, flags, err, wait);
}
template <typename T>
void launch_fwd_below(const DevPlan& P, const DevNum<T>& N, const int2* items, const int32_t* cptr, const int4* cran,
                      int count, T* xp, T* W, int nrhs, cudaStream_t st) {
  if (count > 0) k_fwd_below<T><<<count, 256, 0, st>>>(P, N, items, cptr, cran, xp, W, nrhs);
}
template <typename T>
void launch_bwd_below(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int narrow, const T* xp,
                      T* Pw, int nrhs, cudaStream_t st) {
  if (count <= 0) return;
  const int grid = (narrow + 7) / 8 + (count - narrow);
  k_bwd_below<T><<<grid, 256, 0, st>>>(P, N, items, narrow, xp, Pw, nrhs);
}
template <typename T>
void launch_bwd_chain(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, int smem, bool multi, T* xp,
                      const T* Pw, int nrhs, int* tickets, int* flags, int* err, long long wait, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bwd_chain<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         chain_smem(CHAIN_ROWS, sizeof(T)));
    cudaFuncSetAttribute(k_bwd_chain<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         chain_smem(CHAIN_ROWS, sizeof(T)));
    attr = true;
  }
  if (multi)
    k_bwd_chain<T, true><<<count, 128, smem, st>>>(P, N, items, xp, Pw, nrhs, tickets, flags, err, wait);
  else
    k_bwd_chain<T, false><<<count, 128, smem, st>>>(P, N, items, xp, Pw, nrhs, tickets, flags, err, wait);
}

// ---------------------------------------------------------------------------
// Sweeps over the subtrees of small supernodes.
//
// Near the leaves the assembly tree holds very many supernodes of a few
// columns (at the 700 x 700 grid 170k of 184k supernodes have at most 32
// pivots); per-level launches with one CTA per supernode or per 64 rows keep
// most lanes idle there.  A supernode with at most 32 pivots all of whose
// descendants have at most 32 as well belongs to a region of small
// subtrees; each maximal subtree of it is swept by ONE warp, supernode by
// supernode in postorder (forward) or in reverse (backward), so no flags or
// launches separate a supernode from its children.  The region's forward
// sweep runs before the level launches of the rest of the tree, its
// backward sweep after them.  Lane c holds column c of the supernode; the
// 32 x 32 inverse of its unit lower pivot block is staged in the warp's
// shared memory (row stride 33).
//   forward:  t = own entries + children's updates (in child order),
//             y = L11^-1 t, W_s = children's updates below - L21 y;
//   backward: z = D^-1 y - L21^T x_below, x = L11^-T z.
// ---------------------------------------------------------------------------
constexpr int REG_WARPS = 8;

template <typename T>
__device__ __forceinline__ void region_stage_inverse(const DevPlan& P, const DevNum<T>& N, int s, T* iv, int lane) {
  const T* ip = N.Linv + P.sn_Ioff[s];
#pragma unroll 8
  for (int i = 0; i < 32; i++) iv[i * 33 + lane] = ip[i * 32 + lane];
}

template <typename T>
__global__ void __launch_bounds__(256) k_region_fwd(DevPlan P, DevNum<T> N, const int2* __restrict__ items, int count,
                                                    const int32_t* __restrict__ nodes, T* __restrict__ xp,
                                                    T* __restrict__ W, int nrhs, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* iv = reinterpret_cast<T*>(smem_raw) + warp * (32 * 33 + MAX_RHS_SWEEP * 33);
  T* tb = iv + 32 * 33;                              // [MAX_RHS_SWEEP][33]
  const int64_t dim = P.dim, Wtot = P.Wtot;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= count) break;
    const int2 item = items[it];
    for (int q = 0; q < item.y; q++) {
      const int s = nodes[item.x + q];
      const int ncol = P.sn_ncol[s], nb = P.sn_nrow[s] - ncol, ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
      T* Ws = W + P.sn_Woff[s];
      region_stage_inverse(P, N, s, iv, lane);
      for (int r = 0; r < nrhs; r++) tb[r * 33 + lane] = lane < ncol ? xp[r * dim + col0 + lane] : T(0);
      for (int a = lane; a < nb; a += 32)
        for (int r = 0; r < nrhs; r++) Ws[r * Wtot + a] = T(0);
      __syncwarp();
      // the children's updates, child by child (distinct rows within a child)
      for (int k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
        const int c = P.child_list[k];
        const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
        const int32_t* rel = P.relmap + P.relmap_off[c];
        const T* Wc = W + P.sn_Woff[c];
        for (int a = lane; a < nbc; a += 32) {
          const int row = rel[a];
          for (int r = 0; r < nrhs; r++) {
            const T v = Wc[r * Wtot + a];
            if (row < ncol) tb[r * 33 + row] += v;
            else Ws[r * Wtot + row - ncol] += v;
          }
        }
        __syncwarp();
      }
      // y = L11^-1 t (unit lower inverse, lane = row)
      for (int r = 0; r < nrhs; r++) {
        T y = T(0);
#pragma unroll 8
        for (int u = 0; u < 32; u++) y += iv[lane * 33 + u] * tb[r * 33 + u];
        __syncwarp();
        tb[r * 33 + lane] = lane < ncol ? y : T(0);
        if (lane < ncol) xp[r * dim + col0 + lane] = y;
      }
      __syncwarp();
      // W_s -= L21 y (lane = row below, 16-byte vectors of its row)
      using V = typename Vec16<T>::type;
      constexpr int VW = Vec16<T>::n;
      const int nv = (ncol + VW - 1) / VW;
      for (int a = lane; a < nb; a += 32) {
        const V* row = reinterpret_cast<const V*>(N.L + P.sn_Loff[s] + (int64_t)(ncol + a) * ncp);
        T acc[MAX_RHS_SWEEP];
#pragma unroll
        for (int r = 0; r < MAX_RHS_SWEEP; r++) acc[r] = T(0);
        for (int v = 0; v < nv; v++) {
          const V lv = __ldg(row + v);
#pragma unroll
          for (int e = 0; e < VW; e++) {
            const int k = v * VW + e;
            if (k >= ncol) break;
            const T l = reinterpret_cast<const T*>(&lv)[e];
#pragma unroll
            for (int r = 0; r < MAX_RHS_SWEEP; r++)
              if (r < nrhs) acc[r] += l * tb[r * 33 + k];
          }
        }
#pragma unroll
        for (int r = 0; r < MAX_RHS_SWEEP; r++)
          if (r < nrhs) Ws[r * Wtot + a] -= acc[r];
      }
      __syncwarp();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_region_bwd(DevPlan P, DevNum<T> N, const int2* __restrict__ items, int count,
                                                    const int32_t* __restrict__ nodes, T* __restrict__ xp, int nrhs,
                                                    int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* iv = reinterpret_cast<T*>(smem_raw) + warp * (32 * 33 + MAX_RHS_SWEEP * 33);
  T* zb = iv + 32 * 33;                              // [MAX_RHS_SWEEP][33]
  const int64_t dim = P.dim;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= count) break;
    const int2 item = items[it];
    for (int q = item.y - 1; q >= 0; q--) {
      const int s = nodes[item.x + q];
      const int ncol = P.sn_ncol[s], nb = P.sn_nrow[s] - ncol, ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
      const T* Lb = N.L + P.sn_Loff[s] + (int64_t)ncol * ncp;
      const int32_t* rows = P.sn_rows + P.sn_rows_off[s] + ncol;
      region_stage_inverse(P, N, s, iv, lane);
      // z = D^-1 y - L21^T x_below (lane = column): x_below is gathered 32
      // rows at a time (lane = row, the gathers of a chunk independent), then
      // each row of L21 is read whole by the warp and its x value taken from
      // the row's lane by a shuffle
      const T dk = lane < ncol ? N.D[col0 + lane] : T(1);
      T acc[MAX_RHS_SWEEP];
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++) acc[r] = T(0);
      const int cl = min(lane, max(ncol - 1, 0));
      for (int a0 = 0; a0 < nb; a0 += 32) {
        const int a = a0 + lane;
        const int row = a < nb ? rows[a] : 0;
        T xb[MAX_RHS_SWEEP];
#pragma unroll
        for (int r = 0; r < MAX_RHS_SWEEP; r++) xb[r] = (r < nrhs && a < nb) ? xp[r * dim + row] : T(0);
        const int cnt = min(32, nb - a0);
        const T* lr = Lb + (int64_t)a0 * ncp + cl;
#pragma unroll 8
        for (int u = 0; u < cnt; u++) {
          const T l = lr[(int64_t)u * ncp];
#pragma unroll
          for (int r = 0; r < MAX_RHS_SWEEP; r++)
            if (r < nrhs) acc[r] += l * __shfl_sync(0xffffffffu, xb[r], u);
        }
      }
#pragma unroll
      for (int r = 0; r < MAX_RHS_SWEEP; r++)
        if (r < nrhs) zb[r * 33 + lane] = lane < ncol ? xp[r * dim + col0 + lane] / dk - acc[r] : T(0);
      __syncwarp();
      // x = L11^-T z (lane = column of the inverse)
      for (int r = 0; r < nrhs; r++) {
        T x = T(0);
#pragma unroll 8
        for (int u = 0; u < 32; u++) x += iv[u * 33 + lane] * zb[r * 33 + u];
        if (lane < ncol) xp[r * dim + col0 + lane] = x;
      }
      __syncwarp();
    }
  }
}

int region_smem(int esz) { return REG_WARPS * (32 * 33 + MAX_RHS_SWEEP * 33) * esz; }

template <typename T>
void launch_region_fwd(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes, T* xp,
                       T* W, int nrhs, int* counter, int nsm, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  const int smem = region_smem((int)sizeof(T));
  if (!attr) {
    cudaFuncSetAttribute(k_region_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  // as many CTAs as fit on the device at once (the warps take subtrees from a counter)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_region_fwd<T>, 32 * REG_WARPS, smem) != cudaSuccess)
    per_sm = 4;
  const int grid = std::min((count + REG_WARPS - 1) / REG_WARPS, nsm * std::max(per_sm, 1));
  k_region_fwd<T><<<grid, 32 * REG_WARPS, smem, st>>>(P, N, items, count, nodes, xp, W, nrhs, counter);
}

template <typename T>
void launch_region_bwd(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const int32_t* nodes, T* xp,
                       int nrhs, int* counter, int nsm, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  const int smem = region_smem((int)sizeof(T));
  if (!attr) {
    cudaFuncSetAttribute(k_region_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_region_bwd<T>, 32 * REG_WARPS, smem) != cudaSuccess)
    per_sm = 4;
  const int grid = std::min((count + REG_WARPS - 1) / REG_WARPS, nsm * std::max(per_sm, 1));
  k_region_bwd<T><<<grid, 32 * REG_WARPS, smem, st>>>(P, N, items, count, nodes, xp, nrhs, counter);
}

// ---------------------------------------------------------------------------
// FP64 residual R = B - K X on the FP64 KKT values (4 lanes per row, 8 rows
// per warp trip), with per-instance ||R||_inf and ||X||_inf (bit patterns,
// atomicMax).  Kf holds the values of the full pattern in its row order
// (written before ||K||), so the entries and column indices are read
// contiguously and only X is gathered; an entry is read once for all NR
// right-hand sides, and every load of a trip that does not depend on
// another (row bounds, B, the row's own X) is issued before the products.
// Each warp takes a contiguous run of rows, so that its running maxima
// change instance (and go to the atomics) only at an instance boundary.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(256) k_residual(DevPlan P, const double* __restrict__ Kf,
                                                  const double* __restrict__ B, int64_t ldb,
                                                  const double* __restrict__ X, int64_t ldx, double* __restrict__ R,
                                                  int64_t ldr, int nrhs, unsigned long long* rnorm,
                                                  unsigned long long* xnorm, int64_t rows_per_warp) {
  constexpr int LPR = 4;   // lanes per row
  const int lane = threadIdx.x & 31, sub = lane & (LPR - 1);
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t r_begin = gwarp * rows_per_warp;
  const int64_t r_end = min(P.dim, r_begin + rows_per_warp);
  // running maxima of |r| and |x| for the instance of this lane's rows
  int cur = -1;
  unsigned long long rmx[NR], xmx[NR];
#pragma unroll
  for (int r = 0; r < NR; r++) rmx[r] = xmx[r] = 0ull;
  // the trip count is uniform across the warp so that the full-mask
  // shuffles are safe
  for (int64_t rb = r_begin; rb < r_end; rb += 32 / LPR) {
    const int64_t row = rb + lane / LPR;
    const bool valid = row < r_end;
    const int64_t q0 = valid ? P.F_rowptr[row] : 0, q1 = valid ? P.F_rowptr[row + 1] : 0;
    const int inst = valid ? P.row_inst[row] : -1;
    double bv[NR], xv[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
      const bool use = valid && sub == 0 && r < nrhs;
      bv[r] = use ? B[r * ldb + row] : 0.0;
      xv[r] = use ? X[r * ldx + row] : 0.0;
    }
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) acc[r] = 0.0;
    int64_t q = q0 + sub;
    for (; q + LPR < q1; q += 2 * LPR) {
      const double k0 = Kf[q], k1 = Kf[q + LPR];
      const int64_t c0 = P.F_col[q], c1 = P.F_col[q + LPR];
#pragma unroll
      for (int r = 0; r < NR; r++)
        if (r < nrhs) acc[r] = fma(k1, X[r * ldx + c1], fma(k0, X[r * ldx + c0], acc[r]));
    }
    if (q < q1) {
      const double k0 = Kf[q];
      const int64_t c0 = P.F_col[q];
#pragma unroll
      for (int r = 0; r < NR; r++)
        if (r < nrhs) acc[r] = fma(k0, X[r * ldx + c0], acc[r]);
    }
    if (valid && sub == 0 && inst != cur) {
      if (cur >= 0)
#pragma unroll
        for (int r = 0; r < NR; r++)
          if (r < nrhs) {
            atomicMax(&rnorm[cur * nrhs + r], rmx[r]);
            atomicMax(&xnorm[cur * nrhs + r], xmx[r]);
          }
#pragma unroll
      for (int r = 0; r < NR; r++) rmx[r] = xmx[r] = 0ull;
      cur = inst;
    }
#pragma unroll
    for (int r = 0; r < NR; r++) {
      if (r >= nrhs) break;
      double a = acc[r];
      a += __shfl_xor_sync(FULL_MASK, a, 2);
      a += __shfl_xor_sync(FULL_MASK, a, 1);
      if (valid && sub == 0) {
        const double res = bv[r] - a;
        R[r * ldr + row] = res;
        const unsigned long long u = dbits(fabs(res)), v = dbits(fabs(xv[r]));
        rmx[r] = u > rmx[r] ? u : rmx[r];
        xmx[r] = v > xmx[r] ? v : xmx[r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; r++) {
    if (r >= nrhs) break;
    warp_flush_max(rnorm + r, cur < 0 ? -1 : cur * nrhs, rmx[r]);
    warp_flush_max(xnorm + r, cur < 0 ? -1 : cur * nrhs, xmx[r]);
  }
}

void launch_residual(const DevPlan& P, const double* Kf, const double* B, int64_t ldb, const double* X,
                     int64_t ldx, double* R, int64_t ldr, int nrhs, unsigned long long* rnorm,
                     unsigned long long* xnorm, cudaStream_t st) {
  if (P.dim == 0) return;
  const unsigned grid = grid_for(P.dim * 8);
  const int64_t nwarp = (int64_t)grid * 8;
  const int64_t rpw = ((P.dim + nwarp - 1) / nwarp + 7) / 8 * 8;
  if (nrhs <= 1)
    k_residual<1><<<grid, 256, 0, st>>>(P, Kf, B, ldb, X, ldx, R, ldr, nrhs, rnorm, xnorm, rpw);
  else if (nrhs <= 2)
    k_residual<2><<<grid, 256, 0, st>>>(P, Kf, B, ldb, X, ldx, R, ldr, nrhs, rnorm, xnorm, rpw);
  else if (nrhs <= 4)
    k_residual<4><<<grid, 256, 0, st>>>(P, Kf, B, ldb, X, ldx, R, ldr, nrhs, rnorm, xnorm, rpw);
  else
    k_residual<MAX_RHS_SWEEP><<<grid, 256, 0, st>>>(P, Kf, B, ldb, X, ldx, R, ldr, nrhs, rnorm, xnorm, rpw);
}

// per-instance ||B||_inf; each CTA takes a contiguous run of rows (see k_knorm)
__global__ void k_vec_norm(DevPlan P, const double* __restrict__ B, int64_t ldb, int nrhs, unsigned long long* out,
                           int64_t rows_per_cta) {
  const int64_t i_begin = blockIdx.x * rows_per_cta, i_end = min(P.dim, i_begin + rows_per_cta);
  for (int r = 0; r < nrhs; r++) {
    int cur = -1;
    unsigned long long mx = 0ull;
    for (int64_t i = i_begin + threadIdx.x; i < i_end; i += blockDim.x) {
      const int inst = P.row_inst[i];
      const unsigned long long v = dbits(fabs(B[r * ldb + i]));
      if (inst != cur) {
        if (cur >= 0) atomicMax(&out[cur * nrhs + r], mx);
        cur = inst;
        mx = 0ull;
      }
      mx = v > mx ? v : mx;
    }
    warp_flush_max(out + r, cur < 0 ? -1 : cur * nrhs, mx);
  }
}

void launch_vec_norm(const DevPlan& P, const double* B, int64_t ldb, int nrhs, unsigned long long* out,
                     cudaStream_t st) {
  if (P.dim == 0) return;
  const unsigned grid = grid_for(P.dim);
  k_vec_norm<<<grid, 256, 0, st>>>(P, B, ldb, nrhs, out, (P.dim + grid - 1) / grid);
}

__global__ void k_axpy(double* X, int64_t ldx, const double* Y, int64_t ldy, double a, int64_t dim, int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; r++) X[r * ldx + i] += a * Y[r * ldy + i];
}

void launch_axpy_inplace(double* X, int64_t ldx, const double* Y, int64_t ldy, double a, int64_t dim, int nrhs,
                         cudaStream_t st) {
  if (dim) k_axpy<<<grid_for(dim), 256, 0, st>>>(X, ldx, Y, ldy, a, dim, nrhs);
}

// ---------------------------------------------------------------------------
// FP64 vector kernels of the FGMRES refinement (single instance).
// Reductions are two-pass with a fixed grid: per-block partial sums here,
// summed on the host in block order (bitwise reproducible).
// ---------------------------------------------------------------------------
constexpr int VGRID = 256;

// Y = K X (full FP64 CSR)
__global__ void k_spmv(DevPlan P, const double* __restrict__ Klow, const double* __restrict__ X,
                       double* __restrict__ Y) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t rb = gwarp * 4; rb < P.dim; rb += nwarp * 4) {
    const int64_t row = rb + (lane >> 3);
    const bool valid = row < P.dim;
    const int64_t q0 = valid ? P.F_rowptr[row] : 0, q1 = valid ? P.F_rowptr[row + 1] : 0;
    double acc = 0.0;
    for (int64_t q = q0 + sub; q < q1; q += 8) acc = fma(Klow[P.F_src[q]], X[P.F_col[q]], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (valid && sub == 0) Y[row] = acc;
  }
}

// partial[i * VGRID + block] = sum over the block's slice of V_i . w  (i < nv)
__global__ void __launch_bounds__(256) k_multidot(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                                                  const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double red[256];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (int i = 0; i < nv; i++) {
    double acc = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc = fma(V[i * ldv + e], w[e], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[i * VGRID + blockIdx.x] = red[0];
    __syncthreads();
  }
}

// w = a * w + sum_i c[i] V_i   (c on the device)
__global__ void k_multi_axpy(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                             const double* __restrict__ c, double a, double* __restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = a != 0.0 ? a * w[e] : 0.0;
    for (int i = 0; i < nv; i++) acc = fma(c[i], V[i * ldv + e], acc);
    w[e] = acc;
  }
}

void launch_spmv(const DevPlan& P, const double* Klow, const double* X, double* Y, cudaStream_t st) {
  if (P.dim) k_spmv<<<grid_for(P.dim * 8), 256, 0, st>>>(P, Klow, X, Y);
}
void launch_multidot(int64_t n, const double* V, int64_t ldv, int nv, const double* w, double* partial,
                     cudaStream_t st) {
  if (nv > 0) k_multidot<<<VGRID, 256, 0, st>>>(n, V, ldv, nv, w, partial);
}
void launch_multi_axpy(int64_t n, const double* V, int64_t ldv, int nv, const double* c, double a, double* w,
                       cudaStream_t st) {
  k_multi_axpy<<<grid_for(n), 256, 0, st>>>(n, V, ldv, nv, c, a, w);
}
int vec_grid() { return VGRID; }

// ---------------------------------------------------------------------------
// Adjoint: dl/dK = -GB X^T folded onto the stored values (see ncl_kkt.h).
// ---------------------------------------------------------------------------
__global__ void k_adj_H(DevPlan P, const double* X, int64_t ldx, const double* GB, int64_t ldgb, int nrhs,
                        double* G_H) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.nnzH; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = P.H_row[q], j = P.H_col[q];
    double g = 0.0;
    for (int r = 0; r < nrhs; r++) {
      g -= GB[r * ldgb + i] * X[r * ldx + j];
      if (i != j) g -= GB[r * ldgb + j] * X[r * ldx + i];
    }
    G_H[q] = g;
  }
}

__global__ void k_adj_S(DevPlan P, const double* X, int64_t ldx, const double* GB, int64_t ldgb, int nrhs,
                        double* G_S) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < P.nvar; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = P.var_row[v];
    double g = 0.0;
    for (int r = 0; r < nrhs; r++) g -= GB[r * ldgb + i] * X[r * ldx + i];
    G_S[v] = g;
  }
}

// (J x)_con and (J gb)_con for the condensed form
__global__ void k_jmul(DevPlan P, const double* Jv, const double* X, int64_t ldx, const double* GB, int64_t ldgb,
                       int nrhs, double* jx, double* jg) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.ncon; c += (int64_t)gridDim.x * blockDim.x) {
    for (int r = 0; r < nrhs; r++) {
      double a = 0.0, b = 0.0;
      for (int64_t q = P.J_rowptr[c]; q < P.J_rowptr[c + 1]; q++) {
        a = fma(Jv[q], X[r * ldx + P.J_col[q]], a);
        b = fma(Jv[q], GB[r * ldgb + P.J_col[q]], b);
      }
      jx[r * P.ncon + c] = a;
      jg[r * P.ncon + c] = b;
    }
  }
}

// dl/dJ: K2r from the (2,1) block; K from the product sum_r w_r J_r^T J_r
// (w_r = rho, or rho Omega_r with slacks, Eq. K1s)
__global__ void k_adj_J(DevPlan P, const double* w, const double* X, int64_t ldx, const double* GB, int64_t ldgb,
                        int nrhs, const double* jx, const double* jg, double* G_J) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.nnzJ; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t con = P.J_con[q], c = P.J_col[q];
    double g = 0.0;
    if (P.form == 0) {
      const int32_t rr = P.con_row[con];
      for (int r = 0; r < nrhs; r++) g -= GB[r * ldgb + rr] * X[r * ldx + c] + GB[r * ldgb + c] * X[r * ldx + rr];
    } else {
      const double rh = w[con];
      for (int r = 0; r < nrhs; r++)
        g -= rh * (jg[r * P.ncon + con] * X[r * ldx + c] + jx[r * P.ncon + con] * GB[r * ldgb + c]);
    }
    G_J[q] = g;
  }
}

// per-instance scalar gradients (one CTA per instance, fixed reduction order)
// (dl/drho of K uses dw_r/drho: 1 without slacks, Sigma_s^2/(rho+Sigma_s)^2 with)
__global__ void __launch_bounds__(256) k_adj_scal(DevPlan P, const int64_t* inst_n, const int64_t* inst_con_off,
                                                  const double* rho, const double* dw, const double* X,
                                                  int64_t ldx, const double* GB, int64_t ldgb, int nrhs,
                                                  const double* jx, const double* jg, double* G_scal) {
  __shared__ double red[2][256];
  const int inst = blockIdx.x;
  const int64_t r0 = P.inst_row_off[inst], r1 = P.inst_row_off[inst + 1];
  const int64_t n = inst_n[inst];
  double gd = 0.0, gr = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < nrhs; r++) s += GB[r * ldgb + i] * X[r * ldx + i];
    if (i - r0 < n) gd -= s;
    else gr -= s;  // dual rows (K2r only)
  }
  if (P.form == 0) {
    const double rh = rho[inst];
    gr = gr / (rh * rh);
  } else {
    gr = 0.0;
    for (int64_t c = inst_con_off[inst] + threadIdx.x; c < inst_con_off[inst + 1]; c += blockDim.x)
      for (int r = 0; r < nrhs; r++) gr -= dw[c] * jg[r * P.ncon + c] * jx[r * P.ncon + c];
  }
  red[0][threadIdx.x] = gd;
  red[1][threadIdx.x] = gr;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    G_scal[2 * inst] = red[0][0];
    G_scal[2 * inst + 1] = red[1][0];
  }
}

void launch_adjoint_values(const DevPlan& P, const double* Jv, const double* w, const double* X, int64_t ldx,
                           const double* GB, int64_t ldgb, int nrhs, double* G_H, double* G_J, double* G_S,
                           double* G_scal, double* jx, double* jg, cudaStream_t st) {
  if (G_H && P.nnzH) k_adj_H<<<grid_for(P.nnzH), 256, 0, st>>>(P, X, ldx, GB, ldgb, nrhs, G_H);
  if (G_S && P.nvar) k_adj_S<<<grid_for(P.nvar), 256, 0, st>>>(P, X, ldx, GB, ldgb, nrhs, G_S);
  const bool need_j = P.form == 1 && P.ncon && (G_J || G_scal);
  if (need_j) k_jmul<<<grid_for(P.ncon), 256, 0, st>>>(P, Jv, X, ldx, GB, ldgb, nrhs, jx, jg);
  if (G_J && P.nnzJ) k_adj_J<<<grid_for(P.nnzJ), 256, 0, st>>>(P, w, X, ldx, GB, ldgb, nrhs, jx, jg, G_J);
  (void)G_scal;
}

void launch_adjoint_scalars(const DevPlan& P, const int64_t* inst_n, const int64_t* inst_con_off, const double* rho,
                            const double* dw, const double* X, int64_t ldx, const double* GB, int64_t ldgb,
                            int nrhs, const double* jx, const double* jg, double* G_scal, cudaStream_t st) {
  k_adj_scal<<<P.ninst, 256, 0, st>>>(P, inst_n, inst_con_off, rho, dw, X, ldx, GB, ldgb, nrhs, jx, jg, G_scal);
}

// Slack step of the condensed form with slacks (Section 3.3, proof of the
// proposition on Eq. K1s):  Delta s_r = (rho (J Delta t)_r + r_s,r) /
// (Sigma_s,r + rho) for an inequality row; 0 for a row without slack
// (Sigma_s = +inf).  rho is the penalty of the factored matrix (rho-hat).
// One thread per (row, right-hand side).
__global__ void k_slack_step(DevPlan P, const double* __restrict__ Jv, const double* __restrict__ rho,
                             const double* __restrict__ ss, int nrhs, const double* __restrict__ DT, int64_t ldt,
                             const double* __restrict__ RS, int64_t ldr, double* __restrict__ DS, int64_t lds) {
  const int64_t total = P.ncon * (int64_t)nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx % P.ncon;
    const int r = (int)(idx / P.ncon);
    const double s = ss[c];
    if (isinf(s) && s > 0) {
      DS[r * lds + c] = 0.0;
      continue;
    }
    double jt = 0.0;
    for (int64_t q = P.J_rowptr[c]; q < P.J_rowptr[c + 1]; q++) jt = fma(Jv[q], DT[r * ldt + P.J_col[q]], jt);
    const double rh = rho[P.con_inst[c]];
    DS[r * lds + c] = fma(rh, jt, RS[r * ldr + c]) / (s + rh);
  }
}

// Right-hand side of Eq. K1s as the proof's elimination of Delta s gives it:
//   OUT = RT + rho J_I^T (Sigma_s + rho I)^{-1} RS,
// one thread per (variable, right-hand side), the variable's J values in
// constraint order (deterministic; OUT may alias RT).
__global__ void k_k1s_rhs(DevPlan P, const double* __restrict__ Jv, const double* __restrict__ rho,
                          const double* __restrict__ ss, int nrhs, const double* RT, int64_t ldt,
                          const double* __restrict__ RS, int64_t ldr, double* OUT, int64_t ldo) {
  const int64_t total = P.dim * (int64_t)nrhs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = idx % P.dim;
    const int r = (int)(idx / P.dim);
    double acc = 0.0;
    for (int64_t q = P.JT_ptr[v]; q < P.JT_ptr[v + 1]; q++) {
      const int32_t e = P.JT_idx[q];
      const int32_t c = P.J_con[e];
      const double s = ss[c];
      if (isinf(s) && s > 0) continue;
      const double rh = rho[P.con_inst[c]];
      acc = fma(rh * Jv[e], RS[r * ldr + c] / (s + rh), acc);
    }
    OUT[r * ldo + v] = RT[r * ldt + v] + acc;
  }
}

void launch_k1s_rhs(const DevPlan& P, const double* Jv, const double* rho, const double* ss, int nrhs,
                    const double* RT, int64_t ldt, const double* RS, int64_t ldr, double* OUT, int64_t ldo,
                    cudaStream_t st) {
  const int64_t total = P.dim * (int64_t)nrhs;
  if (total == 0) return;
  k_k1s_rhs<<<grid_for(total), 256, 0, st>>>(P, Jv, rho, ss, nrhs, RT, ldt, RS, ldr, OUT, ldo);
}

// ---------------------------------------------------------------------------
// Newton step of Algorithm NCL around the factorisation (Section 3.1-3.3):
// the right-hand side of Eq. K2r (unknown [Delta x; -Delta y]) or Eq. K1
// (unknown Delta x), and the recovery of the other components from Eq. K3:
//   Delta y   = -(second block of the K2r solution), or
//             = -rho (J Delta x + c) + y_k - y          (Eq. K1, elimination)
//   Delta r   = (Delta y - y_k + y) / rho - r            (Eq. K2, elimination)
//   Delta z_l = -(X - L)^{-1} (Z_l Delta x - mu e) - z_l (eliminated from Eq. K3)
//   Delta z_u =  (U - X)^{-1} (Z_u Delta x + mu e) - z_u
// rho is the penalty of the factored matrix (rho-hat).  An infinite bound
// gives (x - l)^{-1} = 0 (IEEE), so its barrier terms vanish.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double barrier_grad(const NewtonDev& pt, int64_t v, double mu) {
  // -(X - L)^{-1} mu e + (U - X)^{-1} mu e, component v
  return -mu / (pt.x[v] - pt.lo[v]) + mu / (pt.up[v] - pt.x[v]);
}

__global__ void k_newton_rhs(DevPlan P, const double* __restrict__ Jv, const double* __restrict__ rho,
                             const double* __restrict__ mu, NewtonDev pt, double* __restrict__ B) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.dim;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t inst = P.row_inst[k];
    const double rh = rho[inst], m = mu[inst];
    const int32_t v = P.row_var[k];
    if (v >= 0) {
      // J^T y (K2r) or J^T (y_k - rho c) (K), the variable's J values in constraint order
      double jt = 0.0;
      for (int64_t q = P.JT_ptr[k]; q < P.JT_ptr[k + 1]; q++) {
        const int32_t e = P.JT_idx[q], c = P.J_con[e];
        const double wv = P.form == 0 ? pt.y[c] : pt.yk[c] - rh * pt.c[c];
        jt = fma(Jv[e], wv, jt);
      }
      const double gb = pt.g[v] + barrier_grad(pt, v, m);
      B[k] = P.form == 0 ? -(gb - jt) : jt - gb;
    } else {
      const int32_t c = P.row_con[k];
      B[k] = -(pt.c[c] - (pt.yk[c] - pt.y[c]) / rh);
    }
  }
}

__global__ void k_newton_recover_var(DevPlan P, const double* __restrict__ mu, NewtonDev pt,
                                     const double* __restrict__ X, double* __restrict__ dx,
                                     double* __restrict__ dzl, double* __restrict__ dzu) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < P.nvar;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = P.var_row[v];
    const double m = mu[P.row_inst[k]];
    const double d = X[k];
    if (dx) dx[v] = d;
    if (dzl) dzl[v] = -(pt.zl[v] * d - m) / (pt.x[v] - pt.lo[v]) - pt.zl[v];
    if (dzu) dzu[v] = (pt.zu[v] * d + m) / (pt.up[v] - pt.x[v]) - pt.zu[v];
  }
}

__global__ void k_newton_recover_con(DevPlan P, const double* __restrict__ Jv, const double* __restrict__ rho,
                                     NewtonDev pt, const double* __restrict__ X, double* __restrict__ dy,
                                     double* __restrict__ dr) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.ncon;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double rh = rho[P.con_inst[c]];
    double d;
    if (P.form == 0) {
      d = -X[P.con_row[c]];
    } else {
      double jx = 0.0;
      for (int64_t q = P.J_rowptr[c]; q < P.J_rowptr[c + 1]; q++) jx = fma(Jv[q], X[P.J_col[q]], jx);
      d = -rh * (jx + pt.c[c]) + pt.yk[c] - pt.y[c];
    }
    if (dy) dy[c] = d;
    if (dr) dr[c] = (d - pt.yk[c] + pt.y[c]) / rh - pt.r[c];
  }
}

void launch_newton_rhs(const DevPlan& P, const double* Jv, const double* rho, const double* mu, NewtonDev pt,
                       double* B, cudaStream_t st) {
  if (P.dim) k_newton_rhs<<<grid_for(P.dim), 256, 0, st>>>(P, Jv, rho, mu, pt, B);
}

void launch_newton_recover(const DevPlan& P, const double* Jv, const double* rho, const double* mu, NewtonDev pt,
                           const double* X, double* dx, double* dy, double* dr, double* dzl, double* dzu,
                           cudaStream_t st) {
  if (P.nvar) k_newton_recover_var<<<grid_for(P.nvar), 256, 0, st>>>(P, mu, pt, X, dx, dzl, dzu);
  if (P.ncon && (dy || dr)) k_newton_recover_con<<<grid_for(P.ncon), 256, 0, st>>>(P, Jv, rho, pt, X, dy, dr);
}

void launch_slack_step(const DevPlan& P, const double* Jv, const double* rho, const double* ss, int nrhs,
                       const double* DT, int64_t ldt, const double* RS, int64_t ldr, double* DS, int64_t lds,
                       cudaStream_t st) {
  const int64_t total = P.ncon * (int64_t)nrhs;
  if (total == 0) return;
  k_slack_step<<<grid_for(total), 256, 0, st>>>(P, Jv, rho, ss, nrhs, DT, ldt, RS, ldr, DS, lds);
}

#define NCL_INST(T)                                                                                               \
  template void launch_perm_in<T>(const DevPlan&, T*, const double*, int64_t, int, cudaStream_t);                 \
  template void launch_perm_out<T>(const DevPlan&, const T*, double*, int64_t, int, int, cudaStream_t);           \
  template void launch_fwd_chain<T>(const DevPlan&, const DevNum<T>&, const int4*, int, int, bool,               \
                                    const int32_t*, const int4*, T*, const T*, int, int*, int*, int*,            \
                                    long long, cudaStream_t);                                                     \
  template void launch_fwd_below<T>(const DevPlan&, const DevNum<T>&, const int2*, const int32_t*, const int4*,  \
                                    int, T*, T*, int, cudaStream_t);                                              \
  template void launch_bwd_below<T>(const DevPlan&, const DevNum<T>&, const int4*, int, int, const T*, T*, int,   \
                                    cudaStream_t);                                                                \
  template void launch_bwd_chain<T>(const DevPlan&, const DevNum<T>&, const int4*, int, int, bool, T*, const T*, \
                                    int, int*, int*, int*, long long, cudaStream_t);                            \
  template void launch_region_fwd<T>(const DevPlan&, const DevNum<T>&, const int2*, int, const int32_t*, T*, T*, \
                                     int, int*, int, cudaStream_t);                                              \
  template void launch_region_bwd<T>(const DevPlan&, const DevNum<T>&, const int2*, int, const int32_t*, T*, int, \
                                     int*, int, cudaStream_t);
NCL_INST(float)
NCL_INST(double)
#undef NCL_INST

}  // namespace ncl
