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

namespace ncl {

__device__ __forceinline__ int lb_i32(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

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
// forward: pivot block of supernode s (one CTA): pull the children's updates
// that land on the pivot rows, then L11 y = t by 32-column blocks: warp 0
// solves the 32 x 32 diagonal block with shuffles (its row of the block
// prefetched into registers), then every thread updates whole rows below
// it (one 128-byte row segment per row, y of the block from shared memory).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) k_fwd_diag(DevPlan P, DevNum<T> N, const int32_t* __restrict__ list,
                                                   T* __restrict__ xp, const T* __restrict__ W, int nrhs) {
  __shared__ T ys[8][32];
  const int s = list[blockIdx.x];
  const int ncol = P.sn_ncol[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const T* Lb = N.L + P.sn_Loff[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
    const int c = P.child_list[k];
    const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
    const int32_t* rel = P.relmap + P.relmap_off[c];
    const int ahi = lb_i32(rel, nbc, ncol);
    for (int a = threadIdx.x; a < ahi; a += blockDim.x)
      for (int r = 0; r < nrhs; r++) xp[r * P.dim + col0 + rel[a]] += W[r * P.Wtot + P.sn_Woff[c] + a];
    __syncthreads();
  }
  for (int kb = 0; kb < ncol; kb += 32) {
    const int bw = min(32, ncol - kb);
    if (warp == 0) {
      // y_blk = L_blk^-1 t_blk with the inverted diagonal block (row lane)
      T lrow[32];
      const T* ip = N.Linv + P.sn_Ioff[s] + (int64_t)(kb / 32) * 1024 + lane * 32;
#pragma unroll
      for (int u = 0; u < 32; u++) lrow[u] = ip[u];
      for (int r = 0; r < nrhs; r++) {
        T* x = xp + r * P.dim + col0;
        const T t = lane < bw ? x[kb + lane] : T(0);
        T v = T(0);
#pragma unroll
        for (int u = 0; u < 32; u++) v += lrow[u] * __shfl_sync(0xffffffffu, t, u);
        if (lane < bw) x[kb + lane] = v;
        ys[r][lane] = lane < bw ? v : T(0);
      }
    }
    __syncthreads();
    // rows below the block, 32 per warp: lane u reads column kb+u of each
    // row (coalesced), and a butterfly reduce-scatter leaves row r's sum in
    // lane r (31 shuffles per 32 rows)
    const int nw = blockDim.x >> 5;
    for (int i0 = kb + bw + warp * 32; i0 < ncol; i0 += nw * 32) {
      T lv[32];
#pragma unroll
      for (int rr = 0; rr < 32; rr++)
        lv[rr] = (lane < bw && i0 + rr < ncol) ? Lb[(int64_t)(i0 + rr) * ncp + kb + lane] : T(0);
      for (int r = 0; r < nrhs; r++) {
        const T yu = ys[r][lane];
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
        if (i0 + lane < ncol) xp[r * P.dim + col0 + i0 + lane] -= v[0];
      }
    }
    __syncthreads();
  }
}

// forward: rows below supernode s, SOLVE_ROWS per CTA:
//   W_s[a] = (children's updates landing on row a) - L21[a,:] y_s
template <typename T>
__global__ void __launch_bounds__(256) k_fwd_below(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                   const T* __restrict__ xp, T* __restrict__ W, int nrhs) {
  __shared__ T t[SOLVE_ROWS * 8];
  const int2 it = items[blockIdx.x];
  const int s = it.x, a0 = it.y;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int nb = nrow - ncol;
  const int a1 = min(a0 + SOLVE_ROWS, nb);
  const T* Lb = N.L + P.sn_Loff[s];
  for (int idx = threadIdx.x; idx < SOLVE_ROWS * nrhs; idx += blockDim.x) t[idx] = T(0);
  __syncthreads();
  for (int k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
    const int c = P.child_list[k];
    const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
    const int32_t* rel = P.relmap + P.relmap_off[c];
    const int lo = lb_i32(rel, nbc, ncol + a0), hi = lb_i32(rel, nbc, ncol + a1);
    for (int a = lo + threadIdx.x; a < hi; a += blockDim.x)
      for (int r = 0; r < nrhs; r++) t[r * SOLVE_ROWS + rel[a] - ncol - a0] += W[r * P.Wtot + P.sn_Woff[c] + a];
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = a0 + warp; a < a1; a += nw) {
    const T* row = Lb + (int64_t)(ncol + a) * ncp;
    for (int r = 0; r < nrhs; r++) {
      const T* y = xp + r * P.dim + col0;
      T acc = T(0);
      for (int k = lane; k < ncol; k += 32) acc += row[k] * y[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) W[r * P.Wtot + P.sn_Woff[s] + a] = t[r * SOLVE_ROWS + a - a0] - acc;
    }
  }
}

// backward: partial sums of L21^T x_below over a run of SOLVE_ROWS rows
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_below(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                   const T* __restrict__ xp, T* __restrict__ Pw, int nrhs) {
  __shared__ T xb[SOLVE_ROWS * 8];
  const int2 it = items[blockIdx.x];
  const int s = it.x, a0 = it.y;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
  const int nb = nrow - ncol;
  const int a1 = min(a0 + SOLVE_ROWS, nb);
  const int chunk = a0 / SOLVE_ROWS;
  const T* Lb = N.L + P.sn_Loff[s];
  const int32_t* rows = P.sn_rows + P.sn_rows_off[s] + ncol;
  for (int idx = threadIdx.x; idx < (a1 - a0) * nrhs; idx += blockDim.x) {
    const int r = idx / (a1 - a0), a = idx % (a1 - a0);
    xb[r * SOLVE_ROWS + a] = xp[r * P.dim + rows[a0 + a]];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ncol; k += blockDim.x) {
    for (int r = 0; r < nrhs; r++) {
      T acc = T(0);
      for (int a = a0; a < a1; a++) acc += Lb[(int64_t)(ncol + a) * ncp + k] * xb[r * SOLVE_ROWS + a - a0];
      Pw[r * P.Ptot + P.sn_Poff[s] + (int64_t)chunk * ncol + k] = acc;
    }
  }
}

// backward: pivot block (one CTA): z = D^-1 y - sum of partials, then
// L11^T x = z by 32-column blocks from the last one: warp 0 solves the
// diagonal block (lane u holds column u of the block in registers), then
// every thread updates one earlier column u with the block's 32 rows.
template <typename T>
__global__ void __launch_bounds__(512) k_bwd_diag(DevPlan P, DevNum<T> N, const int32_t* __restrict__ list,
                                                   T* __restrict__ xp, const T* __restrict__ Pw, int nrhs) {
  __shared__ T xs[8][32];
  const int s = list[blockIdx.x];
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s], col0 = P.sn_col0[s];
  const int nb = nrow - ncol;
  const int nch = (nb + SOLVE_ROWS - 1) / SOLVE_ROWS;
  const T* Lb = N.L + P.sn_Loff[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < ncol; k += blockDim.x) {
    const T dk = N.D[col0 + k];
    for (int r = 0; r < nrhs; r++) {
      T z = xp[r * P.dim + col0 + k] / dk;
      for (int ch = 0; ch < nch; ch++) z -= Pw[r * P.Ptot + P.sn_Poff[s] + (int64_t)ch * ncol + k];
      xp[r * P.dim + col0 + k] = z;
    }
  }
  __syncthreads();
  const int nblk = (ncol + 31) / 32;
  for (int bi = nblk - 1; bi >= 0; bi--) {
    const int kb = bi * 32;
    const int bw = min(32, ncol - kb);
    if (warp == 0) {
      // x_blk = L_blk^-T z_blk with the inverted diagonal block (column lane)
      T lcol[32];
      const T* ip = N.Linv + P.sn_Ioff[s] + (int64_t)(kb / 32) * 1024 + lane;
#pragma unroll
      for (int v = 0; v < 32; v++) lcol[v] = ip[v * 32];
      for (int r = 0; r < nrhs; r++) {
        T* x = xp + r * P.dim + col0;
        const T z = lane < bw ? x[kb + lane] : T(0);
        T acc = T(0);
#pragma unroll
        for (int v = 0; v < 32; v++) acc += lcol[v] * __shfl_sync(0xffffffffu, z, v);
        if (lane < bw) x[kb + lane] = acc;
        xs[r][lane] = lane < bw ? acc : T(0);
      }
    }
    __syncthreads();
    for (int u = threadIdx.x; u < kb; u += blockDim.x) {
      T lv[32];
#pragma unroll
      for (int v = 0; v < 32; v++) lv[v] = (v < bw) ? Lb[(int64_t)(kb + v) * ncp + u] : T(0);
      for (int r = 0; r < nrhs; r++) {
        T acc = T(0);
#pragma unroll
        for (int v = 0; v < 32; v++) acc += lv[v] * xs[r][v];
        xp[r * P.dim + col0 + u] -= acc;
      }
    }
    __syncthreads();
  }
}

template <typename T>
void launch_fwd_diag(const DevPlan& P, const DevNum<T>& N, const int32_t* list, int count, T* xp, T* W, int nrhs,
                     cudaStream_t st) {
  if (count > 0) k_fwd_diag<T><<<count, sizeof(T) == 4 ? 512 : 256, 0, st>>>(P, N, list, xp, W, nrhs);
}
template <typename T>
void launch_fwd_below(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, T* xp, T* W, int nrhs,
                      cudaStream_t st) {
  if (count > 0) k_fwd_below<T><<<count, 256, 0, st>>>(P, N, items, xp, W, nrhs);
}
template <typename T>
void launch_bwd_below(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, const T* xp, T* Pw,
                      int nrhs, cudaStream_t st) {
  if (count > 0) k_bwd_below<T><<<count, 256, 0, st>>>(P, N, items, xp, Pw, nrhs);
}
template <typename T>
void launch_bwd_diag(const DevPlan& P, const DevNum<T>& N, const int32_t* list, int count, T* xp, const T* Pw,
                     int nrhs, cudaStream_t st) {
  if (count > 0) k_bwd_diag<T><<<count, 512, 0, st>>>(P, N, list, xp, Pw, nrhs);
}

// ---------------------------------------------------------------------------
// FP64 residual R = B - K X on the FP64 KKT values (8 lanes per row), with
// per-instance ||R||_inf and ||X||_inf (bit patterns, atomicMax).
// ---------------------------------------------------------------------------
__global__ void k_residual(DevPlan P, const double* __restrict__ Klow, const double* __restrict__ B, int64_t ldb,
                           const double* __restrict__ X, int64_t ldx, double* __restrict__ R, int64_t ldr, int nrhs,
                           unsigned long long* rnorm, unsigned long long* xnorm) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // each warp takes 4 rows per trip (8 lanes per row); the trip count is
  // uniform across the warp so that the full-mask shuffles are safe
  for (int64_t rb = gwarp * 4; rb < P.dim; rb += nwarp * 4) {
    const int64_t row = rb + (lane >> 3);
    const bool valid = row < P.dim;
    const int64_t q0 = valid ? P.F_rowptr[row] : 0, q1 = valid ? P.F_rowptr[row + 1] : 0;
    const int inst = valid ? P.row_inst[row] : 0;
    for (int r = 0; r < nrhs; r++) {
      const double* x = X + r * ldx;
      double acc = 0.0;
      for (int64_t q = q0 + sub; q < q1; q += 8) acc = fma(Klow[P.F_src[q]], x[P.F_col[q]], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (valid && sub == 0) {
        const double res = B[r * ldb + row] - acc;
        R[r * ldr + row] = res;
        atomicMax(&rnorm[inst * nrhs + r], (unsigned long long)__double_as_longlong(fabs(res)));
        atomicMax(&xnorm[inst * nrhs + r], (unsigned long long)__double_as_longlong(fabs(x[row])));
      }
    }
  }
}

void launch_residual(const DevPlan& P, const double* Klow, const double* B, int64_t ldb, const double* X,
                     int64_t ldx, double* R, int64_t ldr, int nrhs, unsigned long long* rnorm,
                     unsigned long long* xnorm, cudaStream_t st) {
  if (P.dim == 0) return;
  k_residual<<<grid_for(P.dim * 8), 256, 0, st>>>(P, Klow, B, ldb, X, ldx, R, ldr, nrhs, rnorm, xnorm);
}

__global__ void k_vec_norm(DevPlan P, const double* __restrict__ B, int64_t ldb, int nrhs, unsigned long long* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.dim; i += (int64_t)gridDim.x * blockDim.x) {
    const int inst = P.row_inst[i];
    for (int r = 0; r < nrhs; r++)
      atomicMax(&out[inst * nrhs + r], (unsigned long long)__double_as_longlong(fabs(B[r * ldb + i])));
  }
}

void launch_vec_norm(const DevPlan& P, const double* B, int64_t ldb, int nrhs, unsigned long long* out,
                     cudaStream_t st) {
  if (P.dim) k_vec_norm<<<grid_for(P.dim), 256, 0, st>>>(P, B, ldb, nrhs, out);
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

__global__ void k_adj_J(DevPlan P, const double* rho, const double* X, int64_t ldx, const double* GB, int64_t ldgb,
                        int nrhs, const double* jx, const double* jg, double* G_J) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.nnzJ; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t con = P.J_con[q], c = P.J_col[q];
    double g = 0.0;
    if (P.form == 0) {
      const int32_t rr = P.con_row[con];
      for (int r = 0; r < nrhs; r++) g -= GB[r * ldgb + rr] * X[r * ldx + c] + GB[r * ldgb + c] * X[r * ldx + rr];
    } else {
      const double rh = rho[P.J_inst[q]];
      for (int r = 0; r < nrhs; r++)
        g -= rh * (jg[r * P.ncon + con] * X[r * ldx + c] + jx[r * P.ncon + con] * GB[r * ldgb + c]);
    }
    G_J[q] = g;
  }
}

// per-instance scalar gradients (one CTA per instance, fixed reduction order)
__global__ void __launch_bounds__(256) k_adj_scal(DevPlan P, const int64_t* inst_n, const int64_t* inst_con_off,
                                                  const double* rho, const double* X, int64_t ldx,
                                                  const double* GB, int64_t ldgb, int nrhs, const double* jx,
                                                  const double* jg, double* G_scal) {
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
      for (int r = 0; r < nrhs; r++) gr -= jg[r * P.ncon + c] * jx[r * P.ncon + c];
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

void launch_adjoint_values(const DevPlan& P, const double* Jv, const double* rho, const double* X, int64_t ldx,
                           const double* GB, int64_t ldgb, int nrhs, double* G_H, double* G_J, double* G_S,
                           double* G_scal, double* jx, double* jg, cudaStream_t st) {
  if (G_H && P.nnzH) k_adj_H<<<grid_for(P.nnzH), 256, 0, st>>>(P, X, ldx, GB, ldgb, nrhs, G_H);
  if (G_S && P.nvar) k_adj_S<<<grid_for(P.nvar), 256, 0, st>>>(P, X, ldx, GB, ldgb, nrhs, G_S);
  const bool need_j = P.form == 1 && P.ncon && (G_J || G_scal);
  if (need_j) k_jmul<<<grid_for(P.ncon), 256, 0, st>>>(P, Jv, X, ldx, GB, ldgb, nrhs, jx, jg);
  if (G_J && P.nnzJ) k_adj_J<<<grid_for(P.nnzJ), 256, 0, st>>>(P, rho, X, ldx, GB, ldgb, nrhs, jx, jg, G_J);
  (void)G_scal;
}

void launch_adjoint_scalars(const DevPlan& P, const int64_t* inst_n, const int64_t* inst_con_off, const double* rho,
                            const double* X, int64_t ldx, const double* GB, int64_t ldgb, int nrhs,
                            const double* jx, const double* jg, double* G_scal, cudaStream_t st) {
  k_adj_scal<<<P.ninst, 256, 0, st>>>(P, inst_n, inst_con_off, rho, X, ldx, GB, ldgb, nrhs, jx, jg, G_scal);
}

#define NCL_INST(T)                                                                                               \
  template void launch_perm_in<T>(const DevPlan&, T*, const double*, int64_t, int, cudaStream_t);                 \
  template void launch_perm_out<T>(const DevPlan&, const T*, double*, int64_t, int, int, cudaStream_t);           \
  template void launch_fwd_diag<T>(const DevPlan&, const DevNum<T>&, const int32_t*, int, T*, T*, int,            \
                                   cudaStream_t);                                                                 \
  template void launch_fwd_below<T>(const DevPlan&, const DevNum<T>&, const int2*, int, T*, T*, int,              \
                                    cudaStream_t);                                                                \
  template void launch_bwd_below<T>(const DevPlan&, const DevNum<T>&, const int2*, int, const T*, T*, int,        \
                                    cudaStream_t);                                                                \
  template void launch_bwd_diag<T>(const DevPlan&, const DevNum<T>&, const int32_t*, int, T*, const T*, int,      \
                                   cudaStream_t);
NCL_INST(float)
NCL_INST(double)
#undef NCL_INST

}  // namespace ncl
