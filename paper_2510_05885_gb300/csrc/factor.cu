// Numeric multifrontal LDL^T kernels (sm_103a).
//
// A front of supernode s is the dense lower matrix on its rows:
//   [ F11   .  ]   F11: ncol x ncol pivot block   (stored in the L block)
//   [ F21  F22 ]   F21: nbelow x ncol             (stored in the L block)
//                  F22: nbelow x nbelow update    (stored in the U block)
// assembled from the original entries and the children's update blocks
// (extend-add), then partially factored:
//   F11 = L11 D1 L11^T,  L21 = F21 L11^-T D1^-1,  F22 -= L21 D1 L21^T.
// This is the LDL^T with D diagonal and static pivoting of Section 3.1: no
// row or column is ever exchanged; a pivot with |d| <= eps is replaced by
// +-eps with the sign of its block before reordering (case (ii)), or counted
// as a zero eigenvalue (case (i)).
#include "runtime.h"
#include "pivot.cuh"
#include "reduce.cuh"

#include <math_constants.h>

#include <cmath>
#include <cstdio>

namespace ncl {

// ---------------------------------------------------------------------------
// Row weights of the condensed form (Section 3.3): w_r = rho for a row
// without slack (an equality row: Sigma_s = +inf, or no Sigma_s given), and
// for an inequality row with slack barrier term Sigma_s,r (Eq. K1s)
//   w_r = rho Omega_r,  Omega_r = Sigma_s,r / (rho + Sigma_s,r),
// which tends to rho as Sigma_s,r -> inf.  dw_r = dw_r/drho (1, or
// Sigma_s^2 / (rho + Sigma_s)^2) is kept for the adjoint, and the slack term
// for the slack recovery.  rho is the penalty of the matrix (rho-hat).
// ---------------------------------------------------------------------------
__global__ void k_row_weights(DevPlan P, const double* const* __restrict__ vals, const double* __restrict__ rho,
                              double* __restrict__ w, double* __restrict__ dw, double* __restrict__ ss) {
  const double* __restrict__ Ss = vals[3];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.ncon;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double s = Ss ? Ss[c] : CUDART_INF;
    ss[c] = s;
    const double rh = rho[P.con_inst[c]];
    if (isinf(s) && s > 0) {
      w[c] = rh;
      dw[c] = 1.0;
    } else {
      const double den = rh + s;
      w[c] = rh * s / den;
      dw[c] = (s / den) * (s / den);
    }
  }
}

void launch_row_weights(const DevPlan& P, const double* const* vals, const double* rho, double* w, double* dw,
                        double* ss, cudaStream_t st) {
  if (P.ncon == 0) return;
  int64_t blocks = (P.ncon + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_row_weights<<<(unsigned)blocks, 256, 0, st>>>(P, vals, rho, w, dw, ss);
}

// ---------------------------------------------------------------------------
// FP64 values of the lower KKT entries:
//   K2r (Eq. K2r): H_ij, Sigma_i + delta on the primal diagonal, J_ri in the
//                  (2,1) block, -1/rho on the dual diagonal;
//   K   (Eq. K1 / K1s): H_ij + (Sigma_i + delta) [i=j] + sum_r w_r J_ri J_rj,
//                  the product summed over the constraint rows shared by i, j
//                  in a fixed order (no atomics); w_r = rho without slacks.
// ---------------------------------------------------------------------------
__global__ void k_kkt_values(DevPlan P, const double* const* __restrict__ vals, const double* __restrict__ delta,
                             const double* __restrict__ rho, const double* __restrict__ w,
                             double* __restrict__ Klow) {
  // vals = {H values, J values, Sigma}: read from device memory so that a
  // captured graph stays valid when the caller passes new arrays
  const double* __restrict__ Hv = vals[0];
  const double* __restrict__ Jv = vals[1];
  const double* __restrict__ S = vals[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.nnzA;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    int32_t h = P.e_h[e], j = P.e_j[e];
    if (h >= 0) v += Hv[h];
    if (j >= 0) v += Jv[j];
    int8_t kind = P.e_kind[e];
    int32_t inst = P.e_inst[e];
    if (kind == 1) v += S[P.e_var[e]] + delta[inst];
    else if (kind == 2) v += -1.0 / rho[inst];
    int64_t p0 = P.pair_ptr[e], p1 = P.pair_ptr[e + 1];
    if (p1 > p0) {
      double s = 0.0;
      for (int64_t p = p0; p < p1; p++) {
        const int32_t a = P.pair_p[p];
        s = fma(w[P.J_con[a]] * Jv[a], Jv[P.pair_q[p]], s);
      }
      v += s;
    }
    Klow[e] = v;
  }
}

void launch_kkt_values(const DevPlan& P, const double* const* vals, const double* delta, const double* rho,
                       const double* w, double* Klow, cudaStream_t st) {
  if (P.nnzA == 0) return;
  int64_t blocks = (P.nnzA + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_kkt_values<<<(unsigned)blocks, 256, 0, st>>>(P, vals, delta, rho, w, Klow);
}

// The values of the full (both triangles) pattern in its row order, Kf[q] =
// Klow[F_src[q]], which the residual reads contiguously.
__global__ void k_full_values(DevPlan P, const double* __restrict__ Klow, double* __restrict__ Kf, int64_t nnzF) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnzF; q += (int64_t)gridDim.x * blockDim.x)
    Kf[q] = Klow[P.F_src[q]];
}

// ||K||_inf per instance (max absolute row sum), as the bit pattern of a
// non-negative double so that atomicMax on the integer orders it.  Each CTA
// takes a contiguous run of rows (its threads stride through it), so that a
// thread's running maximum changes instance (and goes to an atomic) only at
// an instance boundary: batches of many instances would otherwise contend
// on a few addresses.
__global__ void k_knorm(DevPlan P, const double* __restrict__ Kf, unsigned long long* knorm, int64_t rows_per_cta) {
  int cur = -1;
  unsigned long long mx = 0ull;
  const int64_t r_begin = blockIdx.x * rows_per_cta, r_end = min(P.dim, r_begin + rows_per_cta);
  for (int64_t r = r_begin + threadIdx.x; r < r_end; r += blockDim.x) {
    double s = 0.0;
    for (int64_t q = P.F_rowptr[r]; q < P.F_rowptr[r + 1]; q++) s += fabs(Kf[q]);
    const int inst = P.row_inst[r];
    if (inst != cur) {
      if (cur >= 0) atomicMax(&knorm[cur], mx);
      cur = inst;
      mx = 0ull;
    }
    const unsigned long long v = dbits(s);
    mx = v > mx ? v : mx;
  }
  warp_flush_max(knorm, cur, mx);
}

void launch_full_values(const DevPlan& P, const double* Klow, double* Kf, int64_t nnzF, cudaStream_t st) {
  if (nnzF <= 0) return;
  int64_t qb = (nnzF + 255) / 256;
  if (qb > 152 * 16) qb = 152 * 16;
  k_full_values<<<(unsigned)qb, 256, 0, st>>>(P, Klow, Kf, nnzF);
}

void launch_knorm(const DevPlan& P, const double* Kf, unsigned long long* knorm, cudaStream_t st) {
  if (P.dim == 0) return;
  int64_t blocks = (P.dim + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const int64_t rpc = (P.dim + blocks - 1) / blocks;
  k_knorm<<<(unsigned)blocks, 256, 0, st>>>(P, Kf, knorm, rpc);
}

// ---------------------------------------------------------------------------
// Front assembly.  One CTA per (supernode, run of ASM_ROWS front rows):
// zero the rows, store the original entries, then add the children's update
// blocks child by child (a child's rows map to distinct parent rows, so the
// threads of one child never collide; children are added in a fixed order).
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_assemble(DevPlan P, DevNum<T> N, const int2* __restrict__ items,
                                                  const int32_t* __restrict__ cptr, const int4* __restrict__ cran) {
  const int2 it = items[blockIdx.x];
  const int s = it.x, r0 = it.y;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
  const int nb = nrow - ncol;
  const int r1 = min(r0 + ASM_ROWS, nrow);
  T* Lb = N.L + P.sn_Loff[s];
  T* Ub = N.U + P.sn_Uoff[s];
  // zero
  for (int idx = threadIdx.x; idx < (r1 - r0) * ncp; idx += blockDim.x) Lb[(int64_t)r0 * ncp + idx] = T(0);
  for (int r = max(r0, ncol); r < r1; r++) {
    int a = r - ncol;
    for (int b = threadIdx.x; b <= a; b += blockDim.x) Ub[(int64_t)a * nb + b] = T(0);
  }
  __syncthreads();
  // original entries (each lands in its own position)
  const int64_t rbase = P.sn_rows_off[s];
  for (int r = r0 + (threadIdx.x >> 5); r < r1; r += (blockDim.x >> 5)) {
    int64_t q0 = P.amap_ptr[rbase + r], q1 = P.amap_ptr[rbase + r + 1];
    for (int64_t q = q0 + (threadIdx.x & 31); q < q1; q += 32)
      Lb[(int64_t)r * ncp + P.amap_col[q]] = (T)N.Klow[P.amap_src[q]];
  }
  // children, in a fixed order: the rows [alo, ahi) of child c's update
  // block land on this CTA's rows (ranges found on the host).  Loads are
  // batched four per lane before the read-modify-writes: the targets of one
  // child row are distinct, and each warp owns whole rows.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = cptr[blockIdx.x]; e < cptr[blockIdx.x + 1]; e++) {
    __syncthreads();
    const int4 cr = cran[e];
    const int c = cr.x, alo = cr.y, ahi = cr.z;
    const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
    const int32_t* rel = P.relmap + P.relmap_off[c];
    const T* Uc = N.U + P.sn_Uoff[c];
    for (int a = alo + warp; a < ahi; a += nw) {
      const int ra = rel[a];
      const T* urow = Uc + (int64_t)a * nbc;
      T* lrow = Lb + (int64_t)ra * ncp;
      T* urow_p = ra >= ncol ? Ub + (int64_t)(ra - ncol) * nb - ncol : Ub;   // indexed by rb >= ncol
      for (int b0 = 0; b0 <= a; b0 += 128) {
        int rb[4];
        T v[4], old[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int b = b0 + lane + 32 * t;
          rb[t] = b <= a ? rel[b] : -1;
          v[t] = b <= a ? urow[b] : T(0);
        }
#pragma unroll
        for (int t = 0; t < 4; t++)
          if (rb[t] >= 0) old[t] = rb[t] < ncol ? lrow[rb[t]] : urow_p[rb[t]];
#pragma unroll
        for (int t = 0; t < 4; t++)
          if (rb[t] >= 0) {
            if (rb[t] < ncol) lrow[rb[t]] = old[t] + v[t];
            else urow_p[rb[t]] = old[t] + v[t];
          }
      }
    }
  }
}

template <typename T>
void launch_assemble(const DevPlan& P, const DevNum<T>& N, const int2* items, const int32_t* cptr, const int4* cran,
                     int count, cudaStream_t st) {
  if (count <= 0) return;
  k_assemble<T><<<count, 256, 0, st>>>(P, N, items, cptr, cran);
}

// ---------------------------------------------------------------------------
// SIMT update C -= A diag(d) B^T (lower part), 64 x 64 tiles, 256 threads,
// 4 x 4 outputs per thread: rows 4 ty .. 4 ty + 3 (one 16-byte shared load
// of A per k) and columns tx + 16 b (four conflict-free loads of B, and
// coalesced row segments of C).  FP64 uses DFMA, FP32 FFMA.
// ---------------------------------------------------------------------------
// four consecutive entries of a 16-byte aligned shared array
__device__ __forceinline__ void ld4_shared(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ld4_shared(const double* p, double (&v)[4]) {
  const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

__device__ __forceinline__ void decode_tile(int64_t t, int Nt, int& ti, int& tj) {
  const int64_t tri = (int64_t)Nt * (Nt + 1) / 2;
  if (t < tri) {
    int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((int64_t)a * (a + 1) / 2 > t) a--;
    while ((int64_t)(a + 1) * (a + 2) / 2 <= t) a++;
    ti = a;
    tj = (int)(t - (int64_t)a * (a + 1) / 2);
  } else {
    const int64_t u = t - tri;
    ti = Nt + (int)(u / Nt);
    tj = (int)(u % Nt);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(DevPlan P, DevNum<T> N, const GemmProb* __restrict__ probs,
                                                   const int32_t* __restrict__ tile_prob) {
  constexpr int TB = GEMM_TILE, KC = 16;
  __shared__ __align__(16) T As[KC][TB + 4];   // rows 16-byte aligned
  __shared__ T Bs[KC][TB + 1];
  const int64_t gt = blockIdx.x;
  const GemmProb pb = probs[tile_prob[gt]];
  int ti, tj;
  decode_tile(gt - pb.tile0, pb.Nt, ti, tj);
  const int i0 = ti * TB, j0 = tj * TB;
  const T* A = N.L + pb.a_off;
  const T* B = N.L + pb.b_off;
  const T* d = N.D + pb.d_off;
  T* C = (pb.c_in_u ? N.U : N.L) + pb.c_off;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = T(0);
  // the next K chunk is fetched into registers while the current one is
  // multiplied (thread: k = kk, rows rr + 16 q of A and of B)
  const int kk = threadIdx.x & 15, rr = threadIdx.x >> 4;
  T fa[4], fb[4];
  auto fetch = [&](int k0) {
    const int k = k0 + kk;
    const bool kin = k < pb.K;
    const T dk = kin ? d[k] : T(0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int ia = i0 + rr + 16 * q, jb = j0 + rr + 16 * q;
      fa[q] = (ia < pb.M && kin) ? A[(int64_t)ia * pb.lda + k] : T(0);
      fb[q] = (jb < pb.N && kin) ? B[(int64_t)jb * pb.lda + k] * dk : T(0);
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < pb.K; k0 += KC) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      As[kk][rr + 16 * q] = fa[q];
      Bs[kk][rr + 16 * q] = fb[q];
    }
    __syncthreads();
    if (k0 + KC < pb.K) fetch(k0 + KC);
#pragma unroll
    for (int k2 = 0; k2 < KC; k2++) {
      T av[4], bv[4];
      ld4_shared(&As[k2][4 * ty], av);
#pragma unroll
      for (int b = 0; b < 4; b++) bv[b] = Bs[k2][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  // all 16 loads of C first, then the stores
  T cv[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + 4 * ty + a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      cv[a][b] = (i < pb.M && j < pb.N && j <= i) ? C[(int64_t)i * pb.ldc + j] : T(0);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + 4 * ty + a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      if (i < pb.M && j < pb.N && j <= i) C[(int64_t)i * pb.ldc + j] = cv[a][b] - acc[a][b];
    }
  }
}

template <typename T>
void launch_gemm_simt(const DevPlan& P, const DevNum<T>& N, const GemmProb* probs, const int32_t* tile_prob,
                      int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return;
  k_gemm_simt<T><<<(unsigned)ntiles, 256, 0, st>>>(P, N, probs, tile_prob);
}

// ---------------------------------------------------------------------------
// Inertia and perturbed-pivot counts per instance:
// counts[4*inst + {0,1,2,3}] = (n_pos, n_neg, n_zero, n_perturbed), plus
// counts[4*ninst] = number of non-finite pivots.
// ---------------------------------------------------------------------------
// (each CTA takes a contiguous run of columns, see k_knorm)
template <typename T>
__global__ void k_inertia(DevPlan P, DevNum<T> N, unsigned long long* counts, int64_t cols_per_cta) {
  int cur = -1;
  unsigned c[4] = {0u, 0u, 0u, 0u}, nonfin = 0u;
  const int64_t k_begin = blockIdx.x * cols_per_cta, k_end = min(P.dim, k_begin + cols_per_cta);
  for (int64_t k = k_begin + threadIdx.x; k < k_end; k += blockDim.x) {
    const int inst = P.col_inst[k];
    if (inst != cur) {
      if (cur >= 0)
        for (int j = 0; j < 4; j++)
          if (c[j]) atomicAdd(&counts[4 * cur + j], (unsigned long long)c[j]);
      cur = inst;
      c[0] = c[1] = c[2] = c[3] = 0u;
    }
    const int8_t st = N.piv[k];
    const T d = N.D[k];
    if (st == 3) {
      nonfin++;
      continue;
    }
    if (st == 2) c[2]++;
    else if (d > T(0)) c[0]++;
    else if (d < T(0)) c[1]++;
    else c[2]++;
    if (st == 1) c[3]++;
  }
#pragma unroll
  for (int j = 0; j < 4; j++) warp_flush_add(counts + j, cur < 0 ? -1 : 4 * cur, c[j]);
  warp_flush_add(counts + 4 * P.ninst, 0, nonfin);
}

template <typename T>
void launch_inertia(const DevPlan& P, const DevNum<T>& N, long long* counts, cudaStream_t st) {
  static_assert(sizeof(long long) == sizeof(unsigned long long), "count width");
  if (P.dim == 0) return;
  int64_t blocks = (P.dim + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_inertia<T><<<(unsigned)blocks, 256, 0, st>>>(P, N, reinterpret_cast<unsigned long long*>(counts),
                                                 (P.dim + blocks - 1) / blocks);
}

#define NCL_INST(T)                                                                                     \
  template void launch_assemble<T>(const DevPlan&, const DevNum<T>&, const int2*, const int32_t*,       \
                                   const int4*, int, cudaStream_t);                                     \
  template void launch_gemm_simt<T>(const DevPlan&, const DevNum<T>&, const GemmProb*, const int32_t*,  \
                                    int64_t, cudaStream_t);                                             \
  template void launch_inertia<T>(const DevPlan&, const DevNum<T>&, long long*, cudaStream_t);
NCL_INST(float)
NCL_INST(double)
#undef NCL_INST

}  // namespace ncl
