// Persistent factorisation of the large fronts of one level (sm_103a).
//
// The pivot columns of a large front are factored 128 at a time (the
// right-looking blocked LDL^T with D diagonal and static pivoting of Section
// 3.1).  Instead of one launch per panel step followed by one launch for the
// step's trailing update, one persistent launch per level walks a task list
// built on the host, in which every task depends only on tasks listed before
// it:
//   DIAG(f, p)       factor the diagonal block of panel p of front f (the
//                    diagonal role of panel_roles.cuh, publishing each
//                    32-column sub-block by a release flag);
//   ROWS(f, p, r)    the 64 rows qe + 64 r.. below the panel: L21 and, for a
//                    tensor-core front, its split TF32 operands (the row role);
//   UPD(f, p, i, j)  the 128 x 128 tile (i, j) of the trailing update of
//                    panel p, C -= L_i D_p L_j^T over the panel's 128
//                    columns, on tcgen05 split-TF32 (tensor-core fronts) or
//                    on FMA units.
// The list is ordered with a look-ahead of one panel: the tiles of the next
// panel's columns first, then that panel's DIAG and ROWS, then the rest of
// the current trailing update, so that the critical path DIAG -> ROWS of the
// next rows -> one tile update -> DIAG no longer waits for whole launches.
// CTAs take tasks in list order from a counter; a task waits (bounded) for
// per-front counters: tile (i, j) has had cnt[i][j] trailing updates
// applied, panel p has finished rows[p][t] row tasks in row tile t.  Every
// task a CTA waits for was taken earlier by a CTA that is running, so the
// waits cannot deadlock whatever the scheduling order; past the limit the
// CTA sets the error flag, and every later task is skipped.
#include "panel_roles.cuh"
#include "tc_ops.cuh"

namespace ncl {

namespace {

constexpr int DAG_THREADS = 256;
constexpr int DAG_STAGES = 3;
constexpr int DAG_TILE = 128;

__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// thread 0: wait (bounded) until *p >= v; false on a timeout (err is set) or
// when err was already set by someone else
__device__ __forceinline__ bool dag_wait_geq(const int* p, int v, int* err, long long limit) {
  if (ld_acquire_i32(p) >= v) return true;
  const long long t0 = clock64();
  while (ld_acquire_i32(p) < v) {
    if (ld_acquire_i32(err)) return false;
    if (clock64() - t0 > limit) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// C[i][j] -= sum_k A[i][k] d[k] B[j][k] on a 64 x 64 block (rows i0.., columns
// j0.. of the tile), FMA units, 256 threads with 4 x 4 outputs each; an entry
// is updated only if i < M, j < Nn and row_abs + i >= col_abs + j (the lower
// part of the front).  As / Bs: shared, 2 x 16 x 65 values.
template <typename T>
__device__ __forceinline__ void simt_block64(T* C, int64_t ldc, const T* A, const T* B, int64_t lda, const T* d,
                                             int K, int M, int Nn, int i0, int j0, int row_abs, int col_abs,
                                             T* As, T* Bs) {
  constexpr int TB = 64, KC = 16, LD = TB + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = T(0);
  const int kk = threadIdx.x & 15, rr = threadIdx.x >> 4;
  T fa[4], fb[4];
  auto fetch = [&](int k0) {
    const int k = k0 + kk;
    const bool kin = k < K;
    const T dk = kin ? d[k] : T(0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int ia = i0 + rr + 16 * q, jb = j0 + rr + 16 * q;
      fa[q] = (ia < M && kin) ? A[(int64_t)ia * lda + k] : T(0);
      fb[q] = (jb < Nn && kin) ? B[(int64_t)jb * lda + k] * dk : T(0);
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      As[kk * LD + rr + 16 * q] = fa[q];
      Bs[kk * LD + rr + 16 * q] = fb[q];
    }
    __syncthreads();
    if (k0 + KC < K) fetch(k0 + KC);
#pragma unroll
    for (int k2 = 0; k2 < KC; k2++) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) av[a] = As[k2 * LD + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; b++) bv[b] = Bs[k2 * LD + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  T cv[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      cv[a][b] = (i < M && j < Nn && row_abs + i >= col_abs + j) ? C[(int64_t)i * ldc + j] : T(0);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = j0 + tx + 16 * b;
      if (i < M && j < Nn && row_abs + i >= col_abs + j) C[(int64_t)i * ldc + j] = cv[a][b] - acc[a][b];
    }
  }
}

}  // namespace

int front_dag_smem(int esz) {
  const int roles = macro_panel_smem(esz, DAG_TILE);
  const int simt = 2 * 16 * 65 * esz;
  const int tc = esz == 4 ? DAG_STAGES * TC_STAGE_BYTES : 0;
  return std::max(std::max(roles, simt), tc) + 1024;   // + alignment of the swizzled stages
}

template <typename T>
__global__ void __launch_bounds__(DAG_THREADS, 1)
    k_front_dag(DevPlan P, DevNum<T> N, const DagTask* __restrict__ tasks, int ntasks, int* head, int* cnt,
                int* sync, const CUtensorMap* __restrict__ maps, int* err, double eps, int policy,
                long long wait) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task, s_ok, s_fail;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t bars[2 * DAG_STAGES + 1];
  constexpr bool TC = sizeof(T) == 4;
  // 1024-byte aligned base (the 128-byte swizzle atom of the TMA stages)
  unsigned char* sb = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = bars;
  uint64_t* empty = bars + DAG_STAGES;
  uint64_t* done = bars + 2 * DAG_STAGES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if constexpr (TC) {
    if (tid == 0) {
      for (int s = 0; s < DAG_STAGES; s++) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], 1);
      }
      mbar_init(done, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&s_tmem, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  uint32_t g = 0;       // k-stages this CTA has pushed through its TMA pipeline
  uint32_t ntile = 0;   // tensor-core tiles this CTA has completed (done-barrier phases)
  for (;;) {
    if (tid == 0) s_task = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const DagTask tk = tasks[t];
    const int s = tk.s, p = tk.p;
    const int ncol = P.sn_ncol[s], nrow = P.sn_nrow[s], ncp = P.sn_ncolp[s];
    const int q0 = DAG_TILE * p, qe = min(q0 + DAG_TILE, ncol);
    int* tcnt = cnt + tk.cbase;          // tile counters, Rt x Ct
    int* rdone = cnt + tk.rbase;         // row-task counters, P x Rt
    if (tid == 0) {
      bool ok = !ld_acquire_i32(err);
      if (ok) {
        if (tk.kind == DAG_DIAG) {
          ok = dag_wait_geq(tcnt + p * tk.Ct + p, p, err, wait);
        } else if (tk.kind == DAG_ROWS) {
          const int r0 = qe + MACRO_ROWS * tk.x, r1 = min(r0 + MACRO_ROWS, nrow);
          for (int rt = r0 / DAG_TILE; ok && rt <= (r1 - 1) / DAG_TILE; rt++)
            ok = dag_wait_geq(tcnt + rt * tk.Ct + p, p, err, wait);
        } else {
          const int ti = tk.x, tj = tk.y;
          const int ei = (DAG_TILE * ti + MACRO_ROWS < nrow) ? 2 : 1;
          const int ej = (DAG_TILE * tj + MACRO_ROWS < nrow) ? 2 : 1;
          ok = dag_wait_geq(rdone + p * tk.Rt + ti, ei, err, wait) &&
               dag_wait_geq(rdone + p * tk.Rt + tj, ej, err, wait) &&
               dag_wait_geq(tcnt + ti * tk.Ct + tj, p, err, wait);
        }
      }
      s_ok = ok;
      s_fail = 0;
    }
    __syncthreads();
    if (!s_ok) continue;   // after an error every later task is skipped
    if (tk.kind == DAG_DIAG) {
      panel_diag_role<T, DAG_TILE>(P, N, s, q0, sync + tk.slot + 1, eps, policy, sb);
    } else if (tk.kind == DAG_ROWS) {
      panel_rows_role<T, DAG_TILE>(P, N, s, q0, qe + MACRO_ROWS * tk.x, sync + tk.slot + 1, err, wait, sb);
      // the split operands just stored are read by other CTAs' TMA
      asm volatile("fence.proxy.async.global;" ::: "memory");
    } else {
      const int ti = tk.x, tj = tk.y;
      const int row_a = DAG_TILE * ti, row_b = DAG_TILE * tj;
      const int M = min(DAG_TILE, nrow - row_a), Nn = min(DAG_TILE, ncol - row_b);
      T* C = N.L + P.sn_Loff[s] + (int64_t)row_a * ncp + row_b;
      bool on_tc = false;
      if constexpr (TC) on_tc = tk.map >= 0;
      if (!on_tc) {
        const T* Lb = N.L + P.sn_Loff[s];
        T* As = reinterpret_cast<T*>(sb);
        T* Bs = As + 16 * 65;
        for (int bi = 0; bi < 2; bi++)
          for (int bj = 0; bj < 2; bj++) {
            if (64 * bi >= M || 64 * bj >= Nn || row_a + 64 * bi + 63 < row_b + 64 * bj) continue;
            simt_block64<T>(C, ncp, Lb + (int64_t)row_a * ncp + q0, Lb + (int64_t)row_b * ncp + q0, ncp,
                            N.D + P.sn_col0[s] + q0, qe - q0, M, Nn, 64 * bi, 64 * bj, row_a, row_b, As, Bs);
          }
      } else if constexpr (TC) {
        // split-TF32 tile product on the tensor cores: thread 0 loads the
        // k-chunks by TMA, thread 32 issues the MMAs, all eight warps read
        // the accumulator back (warp w: TMEM lanes 32 (w % 4).., columns
        // 64 (w / 4)..) and update C through shared memory
        const CUtensorMap* mLhi = maps + 4 * tk.map;
        const int nk = (qe - q0) / TC_BK;
        const uint32_t tmem = s_tmem;
        int issued = 0;
        if (tid == 0) {
          // the operands were written by other CTAs' generic stores (acquired
          // above): order them before this thread's asynchronous TMA reads
          asm volatile("fence.proxy.async.global;" ::: "memory");
          for (int kt = 0; kt < nk; kt++) {
            const uint32_t gg = g + kt, st = gg % DAG_STAGES;
            if (gg >= DAG_STAGES && !mbar_wait_bounded(&empty[st], ((gg / DAG_STAGES) - 1) & 1, wait)) {
              s_fail = 1;
              break;
            }
            issued = kt + 1;
            unsigned char* sp = sb + st * TC_STAGE_BYTES;
            mbar_expect_tx(&full[st], TC_STAGE_BYTES);
            const int x = q0 + kt * TC_BK;
            tma_load_2d(sp, mLhi, x, row_a, &full[st]);
            tma_load_2d(sp + TC_TILE_BYTES, mLhi + 1, x, row_a, &full[st]);
            tma_load_2d(sp + 2 * TC_TILE_BYTES, mLhi + 2, x, row_b, &full[st]);
            tma_load_2d(sp + 3 * TC_TILE_BYTES, mLhi + 3, x, row_b, &full[st]);
          }
        } else if (tid == 32) {
          for (int kt = 0; kt < nk; kt++) {
            const uint32_t gg = g + kt, st = gg % DAG_STAGES;
            if (!mbar_wait_bounded(&full[st], (gg / DAG_STAGES) & 1, wait)) {
              s_fail = 1;
              break;
            }
            tc_fence_after();
            const uint32_t a_hi = smem_u32(sb + st * TC_STAGE_BYTES);
            const uint32_t a_lo = a_hi + TC_TILE_BYTES;
            const uint32_t b_hi = a_hi + 2 * TC_TILE_BYTES;
            const uint32_t b_lo = a_hi + 3 * TC_TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 8; kk++) {
              const uint32_t off = kk * 32;
              umma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), (kt | kk) != 0);
              umma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), 1);
              umma_tf32(tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), 1);
            }
            umma_commit(&empty[st]);
          }
          umma_commit(done);
        }
        __syncwarp();
        if (!mbar_wait_bounded(done, ntile & 1, wait)) s_fail = 1;
        tc_fence_after();
        __syncthreads();
        if (s_fail) {
          if (tid == 0) {
            atomicExch(err, 1);
            // the copies already issued may still be landing: wait (bounded)
            // for the last phase of every stage that has one in flight
            for (int kt = issued > DAG_STAGES ? issued - DAG_STAGES : 0; kt < issued; kt++) {
              const uint32_t gg = g + kt;
              mbar_wait_bounded(&full[gg % DAG_STAGES], (gg / DAG_STAGES) & 1, wait);
            }
          }
        } else {
          float* stg = reinterpret_cast<float*>(sb) + warp * (32 * 33);
          const int quad = warp & 3, half = warp >> 2;
          const int ib = 32 * quad;
#pragma unroll 1
          for (int c = 0; c < 2; c++) {
            const int jb = 64 * half + 32 * c;
            float v[32];
            tmem_ld_32x32(tmem + ((uint32_t)ib << 16) + (uint32_t)jb, v);
#pragma unroll
            for (int u = 0; u < 32; u++) stg[lane * 33 + u] = v[u];
            __syncwarp();
            const int j = jb + lane;
            if (jb < Nn && ib < M && row_a + ib + 31 >= row_b + jb) {
              float cv[32];
#pragma unroll
              for (int rr = 0; rr < 32; rr++) {
                const int i = ib + rr;
                cv[rr] = (i < M && j < Nn && row_a + i >= row_b + j) ? C[(int64_t)i * ncp + j] : 0.f;
              }
#pragma unroll
              for (int rr = 0; rr < 32; rr++) {
                const int i = ib + rr;
                if (i < M && j < Nn && row_a + i >= row_b + j) C[(int64_t)i * ncp + j] = cv[rr] - stg[rr * 33 + lane];
              }
            }
            __syncwarp();
          }
        }
        g += nk;
        ntile++;
        tc_fence_before();
      }
    }
    // the next task may refill this shared memory by TMA: order this task's
    // generic accesses before those asynchronous writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !s_fail) {
      if (tk.kind == DAG_ROWS) {
        const int r0 = qe + MACRO_ROWS * tk.x;
        if (qe < ncol) {
          __threadfence();
          red_release_add(rdone + p * tk.Rt + r0 / DAG_TILE, 1);
        }
      } else if (tk.kind == DAG_UPD) {
        __threadfence();
        st_release_i32(tcnt + tk.x * tk.Ct + tk.y, p + 1);
      }
    }
  }
  if constexpr (TC) {
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(s_tmem, 128);
  }
}

template <typename T>
void launch_front_dag(const DevPlan& P, const DevNum<T>& N, const DagTask* tasks, int ntasks, int grid, int* head,
                      int* cnt, int* sync, const CUtensorMap* maps, int* err, double eps, int policy, long long wait,
                      cudaStream_t st) {
  if (ntasks <= 0) return;
  static bool attr = false;
  const int smem = front_dag_smem((int)sizeof(T));
  if (!attr) {
    cudaFuncSetAttribute(k_front_dag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  k_front_dag<T><<<grid, DAG_THREADS, smem, st>>>(P, N, tasks, ntasks, head, cnt, sync, maps, err, eps, policy, wait);
}

template void launch_front_dag<float>(const DevPlan&, const DevNum<float>&, const DagTask*, int, int, int*, int*,
                                      int*, const CUtensorMap*, int*, double, int, long long, cudaStream_t);
template void launch_front_dag<double>(const DevPlan&, const DevNum<double>&, const DagTask*, int, int, int*, int*,
                                       int*, const CUtensorMap*, int*, double, int, long long, cudaStream_t);

}  // namespace ncl
