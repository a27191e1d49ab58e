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
#include "diag32.cuh"

#include <cmath>
#include <cstdio>

namespace ncl {

// ---------------------------------------------------------------------------
// FP64 values of the lower KKT entries:
//   K2r (Eq. K2r): H_ij, Sigma_i + delta on the primal diagonal, J_ri in the
//                  (2,1) block, -1/rho on the dual diagonal;
//   K   (Eq. K1):  H_ij + (Sigma_i + delta) [i=j] + rho * sum_r J_ri J_rj,
//                  the product summed over the constraint rows shared by i, j
//                  in a fixed order (no atomics).
// ---------------------------------------------------------------------------
__global__ void k_kkt_values(DevPlan P, const double* const* __restrict__ vals, const double* __restrict__ delta,
                             const double* __restrict__ rho, double* __restrict__ Klow) {
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
      for (int64_t p = p0; p < p1; p++) s = fma(Jv[P.pair_p[p]], Jv[P.pair_q[p]], s);
      v = fma(rho[inst], s, v);
    }
    Klow[e] = v;
  }
}

void launch_kkt_values(const DevPlan& P, const double* const* vals, const double* delta, const double* rho,
                       double* Klow, cudaStream_t st) {
  if (P.nnzA == 0) return;
  int64_t blocks = (P.nnzA + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_kkt_values<<<(unsigned)blocks, 256, 0, st>>>(P, vals, delta, rho, Klow);
}

// ||K||_inf per instance (max absolute row sum), as the bit pattern of a
// non-negative double so that atomicMax on the integer orders it.
__global__ void k_knorm(DevPlan P, const double* __restrict__ Klow, unsigned long long* knorm) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < P.dim;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t q = P.F_rowptr[r]; q < P.F_rowptr[r + 1]; q++) s += fabs(Klow[P.F_src[q]]);
    atomicMax(&knorm[P.row_inst[r]], (unsigned long long)__double_as_longlong(s));
  }
}

void launch_knorm(const DevPlan& P, const double* Klow, unsigned long long* knorm, cudaStream_t st) {
  if (P.dim == 0) return;
  int64_t blocks = (P.dim + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_knorm<<<(unsigned)blocks, 256, 0, st>>>(P, Klow, knorm);
}

// ---------------------------------------------------------------------------
// Front assembly.  One CTA per (supernode, run of ASM_ROWS front rows):
// zero the rows, store the original entries, then add the children's update
// blocks child by child (a child's rows map to distinct parent rows, so the
// threads of one child never collide; children are added in a fixed order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_assemble(DevPlan P, DevNum<T> N, const int2* __restrict__ items, double eps,
                                                  int policy) {
  static_assert(ASM_ROWS == PANEL_NB, "the first assembly CTA owns the first diagonal block");
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
  // children
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++) {
    __syncthreads();
    const int c = P.child_list[k];
    const int nbc = P.sn_nrow[c] - P.sn_ncol[c];
    const int32_t* rel = P.relmap + P.relmap_off[c];
    const T* Uc = N.U + P.sn_Uoff[c];
    const int alo = lower_bound_i32(rel, nbc, r0);
    const int ahi = lower_bound_i32(rel, nbc, r1);
    for (int a = alo + warp; a < ahi; a += nw) {
      const int ra = rel[a];
      const T* urow = Uc + (int64_t)a * nbc;
      for (int b = lane; b <= a; b += 32) {
        const int rb = rel[b];
        const T v = urow[b];
        if (rb < ncol) Lb[(int64_t)ra * ncp + rb] += v;
        else Ub[(int64_t)(ra - ncol) * nb + (rb - ncol)] += v;
      }
    }
  }
  // a front factored by panels: this CTA holds the complete first diagonal
  // block (rows [0, 32)), so it factors it now
  if (r0 == 0 && (P.sn_flags[s] & 1)) {
    __syncthreads();
    if (warp == 0) factor_diag32<T>(P, N, s, 0, eps, policy, lane);
  }
}

template <typename T>
void launch_assemble(const DevPlan& P, const DevNum<T>& N, const int2* items, int count, double eps, int policy,
                     cudaStream_t st) {
  if (count <= 0) return;
  k_assemble<T><<<count, 256, 0, st>>>(P, N, items, eps, policy);
}

// ---------------------------------------------------------------------------
// Small fronts: one CTA factors the whole front in shared memory.
// Right-looking over the ncol pivots (only the L part is updated), then the
// update block F22 -= L21 D1 L21^T straight from shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_factor_small(DevPlan P, DevNum<T> N, const int32_t* __restrict__ list,
                                                      double eps, int policy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = list[blockIdx.x];
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
  const int col0 = P.sn_col0[s];
  __shared__ int8_t sgn[64];
  T* F = reinterpret_cast<T*>(smem_raw);
  T* w = F + (int64_t)nrow * ncp;
  T* Lg = N.L + P.sn_Loff[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < nrow * ncp; idx += blockDim.x) F[idx] = Lg[idx];
  for (int k = threadIdx.x; k < ncol; k += blockDim.x) sgn[k] = P.col_sign[col0 + k];
  __syncthreads();
  // pivot columns: right-looking, rows over warps, pivot columns over lanes
  for (int k = 0; k < ncol; k++) {
    int8_t stt;
    const T dk = static_pivot<T>(F[k * ncp + k], sgn[k], eps, policy, stt);
    for (int i = k + 1 + threadIdx.x; i < nrow; i += blockDim.x) w[i] = F[i * ncp + k];
    __syncthreads();
    const T invd = T(1) / dk;
    for (int i = k + 1 + warp; i < nrow; i += 8) {
      const T li = w[i] * invd;
      for (int j = k + 1 + lane; j < ncol && j <= i; j += 32) F[i * ncp + j] -= li * w[j];
      if (lane == 0) F[i * ncp + k] = li;
    }
    if (threadIdx.x == 0) {
      F[k * ncp + k] = dk;
      N.D[col0 + k] = dk;
      N.piv[col0 + k] = stt;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nrow * ncp; idx += blockDim.x) Lg[idx] = F[idx];
  // update block F22 -= L21 D1 L21^T, 4 x 4 register tiles of the lower triangle
  const int nb = nrow - ncol;
  if (nb == 0) return;
  for (int k = threadIdx.x; k < ncol; k += blockDim.x) w[k] = F[k * ncp + k];
  __syncthreads();
  T* Ug = N.U + P.sn_Uoff[s];
  const int nbt = (nb + 3) >> 2;
  const int ntile = nbt * (nbt + 1) / 2;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
    int ta = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (ta * (ta + 1) / 2 > t) ta--;
    while ((ta + 1) * (ta + 2) / 2 <= t) ta++;
    const int tb = t - ta * (ta + 1) / 2;
    const int a0 = ta * 4, b0 = tb * 4;
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
      for (int y = 0; y < 4; y++) acc[x][y] = T(0);
    const T* ra[4];
    const T* rb[4];
#pragma unroll
    for (int x = 0; x < 4; x++) {
      ra[x] = F + (int64_t)(ncol + min(a0 + x, nb - 1)) * ncp;
      rb[x] = F + (int64_t)(ncol + min(b0 + x, nb - 1)) * ncp;
    }
    for (int k = 0; k < ncol; k++) {
      const T dk = w[k];
      T av[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; x++) {
        av[x] = ra[x][k];
        bv[x] = rb[x][k] * dk;
      }
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int a = a0 + x;
      if (a >= nb) continue;
#pragma unroll
      for (int y = 0; y < 4; y++) {
        const int b = b0 + y;
        if (b <= a) Ug[(int64_t)a * nb + b] -= acc[x][y];
      }
    }
  }
}

template <typename T>
void launch_factor_small(const DevPlan& P, const DevNum<T>& N, const int32_t* list, int count, double eps,
                         int policy, cudaStream_t st) {
  if (count <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_factor_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMALL_SMEM + 4096);
    attr = true;
  }
  k_factor_small<T><<<count, 256, SMALL_SMEM + 4096, st>>>(P, N, list, eps, policy);
}

// ---------------------------------------------------------------------------
// Panel of a large front: pivot columns [p0, pe), pe - p0 <= PANEL_NB.
// k_panel_diag (one CTA per front) factors the diagonal block in shared
// memory and writes L11 and D1 back; then k_panel_rows solves the rows
// below it, PANEL_ROWS rows per CTA, one row per thread:
//   q = L11^-1 f_i (forward substitution), l_i = D1^-1 q.
// (Two launches: the row CTAs must read the factored block, which no CTA
// of the same launch may be rewriting.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename T>
__global__ void __launch_bounds__(PANEL_ROWS) k_panel_rows(DevPlan P, DevNum<T> N, const int4* __restrict__ items) {
  __shared__ T Db[PANEL_NB][PANEL_NB + 1];
  const int4 it = items[blockIdx.x];
  const int s = it.x, p0 = it.y, r0 = it.z;
  const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
  const int pe = min(p0 + PANEL_NB, ncol);
  const int nbk = pe - p0;
  const T* Lc = N.L + P.sn_Loff[s];
  for (int idx = threadIdx.x; idx < PANEL_NB * PANEL_NB; idx += blockDim.x) {
    const int i = idx / PANEL_NB, j = idx % PANEL_NB;
    Db[i][j] = (i < nbk && j <= i) ? Lc[(int64_t)(p0 + i) * ncp + p0 + j] : T(1);
  }
  __syncthreads();
  const int i = r0 + threadIdx.x;
  if (i < nrow && i >= pe && i < r0 + PANEL_ROWS) {
    T q[PANEL_NB];
    T* row = N.L + P.sn_Loff[s] + (int64_t)i * ncp + p0;
    // the 32 values of the row are 16-byte aligned (ncp % 4 == 0, p0 % 32 == 0)
    if (nbk == PANEL_NB) {
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int t = 0; t < PANEL_NB; t += 4) {
          const float4 v = *reinterpret_cast<const float4*>(row + t);
          q[t] = v.x, q[t + 1] = v.y, q[t + 2] = v.z, q[t + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < PANEL_NB; t += 2) {
          const double2 v = *reinterpret_cast<const double2*>(row + t);
          q[t] = v.x, q[t + 1] = v.y;
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < PANEL_NB; t++) q[t] = (t < nbk) ? row[t] : T(0);
    }
    // forward substitution q = L11^-1 f, column by column (short dependency chains)
#pragma unroll
    for (int u = 0; u < PANEL_NB - 1; u++) {
      const T qu = q[u];
#pragma unroll
      for (int t = u + 1; t < PANEL_NB; t++) q[t] -= Db[t][u] * qu;
    }
#pragma unroll
    for (int t = 0; t < PANEL_NB; t++) {
      q[t] = (t < nbk) ? q[t] / Db[t][t] : T(0);
      if (t < nbk) row[t] = q[t];
    }
    if constexpr (sizeof(T) == 4) {
      // split TF32 operands of the tensor-core updates: L = hi + lo and
      // W = L D = hi + lo, zero on the padding columns
      const int64_t so = P.sn_Soff ? P.sn_Soff[s] : -1;
      if (N.S && so >= 0) {
        const int64_t plane = (int64_t)nrow * ncp;
        float* sp = N.S + so + (int64_t)i * ncp + p0;
#pragma unroll
        for (int t = 0; t < PANEL_NB; t++) {
          if (p0 + t < ncp) {
            const float l = (float)q[t];
            const float w = (t < nbk) ? l * (float)Db[t][t] : 0.f;
            const float lh = round_tf32(l), wh = round_tf32(w);
            sp[t] = lh;
            sp[plane + t] = round_tf32(l - lh);
            sp[2 * plane + t] = wh;
            sp[3 * plane + t] = round_tf32(w - wh);
          }
        }
      }
    }
  }
}

template <typename T>
void launch_panel_rows(const DevPlan& P, const DevNum<T>& N, const int4* items, int count, cudaStream_t st) {
  if (count <= 0) return;
  k_panel_rows<T><<<count, PANEL_ROWS, 0, st>>>(P, N, items);
}

// ---------------------------------------------------------------------------
// SIMT update C -= A diag(d) B^T (lower part), 64 x 64 tiles, 256 threads,
// 4 x 4 outputs per thread.  FP64 uses DFMA, FP32 FFMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decode_tile(int64_t t, int Nt, int& ti, int& tj) {
  const int64_t tri = (int64_t)Nt * (Nt + 1) / 2;
  if (t < tri) {
    int a = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
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
                                                   int nprob, double eps, int policy) {
  constexpr int TB = GEMM_TILE, KC = 16;
  __shared__ T As[KC][TB + 1];
  __shared__ T Bs[KC][TB + 1];
  // find the problem of this tile
  const int64_t gt = blockIdx.x;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile0 <= gt) lo = mid;
    else hi = mid - 1;
  }
  const GemmProb pb = probs[lo];
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
  for (int k0 = 0; k0 < pb.K; k0 += KC) {
    for (int idx = threadIdx.x; idx < TB * KC; idx += 256) {
      const int r = idx / KC, kk = idx % KC;
      const int k = k0 + kk;
      const int ia = i0 + r, jb = j0 + r;
      As[kk][r] = (ia < pb.M && k < pb.K) ? A[(int64_t)ia * pb.lda + k] : T(0);
      Bs[kk][r] = (jb < pb.N && k < pb.K) ? B[(int64_t)jb * pb.lda + k] * d[k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; kk++) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; b++) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + ty + 16 * a;
    if (i >= pb.M) continue;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      if (j >= pb.N || j > i) continue;
      C[(int64_t)i * pb.ldc + j] -= acc[a][b];
    }
  }
  // tile (0,0) of a trailing update holds the next panel's diagonal block,
  // now fully updated: factor it here
  if (gt == pb.tile0 && pb.next_p0 >= 0) {
    __syncthreads();
    if (threadIdx.x < 32) factor_diag32<T>(P, N, pb.front, pb.next_p0, eps, policy, threadIdx.x);
  }
}

template <typename T>
void launch_gemm_simt(const DevPlan& P, const DevNum<T>& N, const GemmProb* probs, int nprob, int64_t ntiles,
                      double eps, int policy, cudaStream_t st) {
  if (ntiles <= 0) return;
  k_gemm_simt<T><<<(unsigned)ntiles, 256, 0, st>>>(P, N, probs, nprob, eps, policy);
}

// ---------------------------------------------------------------------------
// Inertia and perturbed-pivot counts per instance:
// counts[4*inst + {0,1,2,3}] = (n_pos, n_neg, n_zero, n_perturbed), plus
// counts[4*ninst] = number of non-finite pivots.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_inertia(DevPlan P, DevNum<T> N, long long* counts) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.dim;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int inst = P.col_inst[k];
    const int8_t st = N.piv[k];
    const T d = N.D[k];
    long long* c = counts + 4 * inst;
    if (st == 3) {
      atomicAdd((unsigned long long*)&counts[4 * P.ninst], 1ull);
      continue;
    }
    if (st == 2) atomicAdd((unsigned long long*)&c[2], 1ull);
    else if (d > T(0)) atomicAdd((unsigned long long*)&c[0], 1ull);
    else if (d < T(0)) atomicAdd((unsigned long long*)&c[1], 1ull);
    else atomicAdd((unsigned long long*)&c[2], 1ull);
    if (st == 1) atomicAdd((unsigned long long*)&c[3], 1ull);
  }
}

template <typename T>
void launch_inertia(const DevPlan& P, const DevNum<T>& N, long long* counts, cudaStream_t st) {
  if (P.dim == 0) return;
  int64_t blocks = (P.dim + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_inertia<T><<<(unsigned)blocks, 256, 0, st>>>(P, N, counts);
}

#define NCL_INST(T)                                                                                     \
  template void launch_assemble<T>(const DevPlan&, const DevNum<T>&, const int2*, int, double, int,     \
                                   cudaStream_t);                                                       \
  template void launch_factor_small<T>(const DevPlan&, const DevNum<T>&, const int32_t*, int, double,   \
                                       int, cudaStream_t);                                              \
  template void launch_panel_rows<T>(const DevPlan&, const DevNum<T>&, const int4*, int, cudaStream_t); \
  template void launch_gemm_simt<T>(const DevPlan&, const DevNum<T>&, const GemmProb*, int, int64_t,    \
                                    double, int, cudaStream_t);                                         \
  template void launch_inertia<T>(const DevPlan&, const DevNum<T>&, long long*, cudaStream_t);
NCL_INST(float)
NCL_INST(double)
#undef NCL_INST

}  // namespace ncl
