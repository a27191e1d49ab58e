// Split-TF32 dense updates on the 5th-generation tensor cores (sm_103a).
//
//   C[i][j] -= sum_k L[ra+i][k] * d[k] * L[rb+j][k]     (j <= i, lower part)
//
// which is the trailing update of a front's pivot columns and the update
// block F22 -= L21 D1 L21^T of the multifrontal LDL^T.  Each FP32 operand is
// split into two TF32 terms, x = x_hi + x_lo (x_hi = x rounded to TF32,
// x_lo = the remainder rounded to TF32), and the product is accumulated in
// FP32 as A_hi B_hi + A_hi B_lo + A_lo B_hi, which keeps FP32-level accuracy
// (the dropped A_lo B_lo term is about 2^-22 relative).  The split operands
// L_hi, L_lo, W_hi, W_lo (W = L D) are written by the macro-panel row kernel
// next to L, so this kernel is a plain TMA -> tcgen05.mma -> TMEM -> epilogue.
//
// One CTA computes one 128 x 128 tile of C: thread 0 issues TMA loads
// (128-byte swizzle, 3-stage mbarrier pipeline), thread 32 issues the MMAs
// (M=128, N=128, K=8 per instruction, FP32 accumulator in 128 TMEM
// columns) and commits them to the stage barriers, then all four warps read
// their 32 accumulator lanes back with tcgen05.ld and update C.  Every wait
// is bounded: on a timeout the kernel sets an error flag, skips the update,
// waits (bounded) for the TMA copies it has issued, frees its TMEM and
// returns.
#include "runtime.h"
#include "tc_ops.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <vector>

namespace ncl {

namespace {

__global__ void __launch_bounds__(128) k_update_tc(DevNum<float> Nm, const TcProb* __restrict__ probs,
                                                   const int32_t* __restrict__ tile_prob,
                                                   const CUtensorMap* __restrict__ maps, int* err, int stages,
                                                   long long wait) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment of the shared-window address (the swizzle atom)
  unsigned char* sb = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sb + stages * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // problem and tile of this CTA
  const int64_t gt = blockIdx.x;
  const TcProb pb = probs[tile_prob[gt]];
  int ti, tj;
  decode_lower_tile(gt - pb.tile0, pb.Nt, ti, tj);
  const int i0 = ti * TC_M, j0 = tj * TC_N;
  const CUtensorMap* mLhi = maps + 4 * pb.map;
  const CUtensorMap* mLlo = mLhi + 1;
  const CUtensorMap* mWhi = mLhi + 2;
  const CUtensorMap* mWlo = mLhi + 3;

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < stages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mLhi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mWhi)) : "memory");
  }
  if (warp == 0) tmem_alloc(tslot, TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nk = pb.nk;

  int issued = 0;   // TMA stages issued by the producer (thread 0)
  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kt = 0; kt < nk; kt++) {
      const int s = kt % stages;
      if (kt >= stages && !mbar_wait_bounded(&empty[s], ((kt / stages) - 1) & 1, wait)) {
        s_fail = 1;
        break;
      }
      issued = kt + 1;
      unsigned char* st = sb + s * TC_STAGE_BYTES;
      mbar_expect_tx(&full[s], TC_STAGE_BYTES);
      const int x = pb.k0 + kt * TC_BK;
      tma_load_2d(st, mLhi, x, pb.row_a + i0, &full[s]);
      tma_load_2d(st + TC_TILE_BYTES, mLlo, x, pb.row_a + i0, &full[s]);
      tma_load_2d(st + 2 * TC_TILE_BYTES, mWhi, x, pb.row_b + j0, &full[s]);
      tma_load_2d(st + 3 * TC_TILE_BYTES, mWlo, x, pb.row_b + j0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int kt = 0;
    for (; kt < nk; kt++) {
      const int s = kt % stages;
      if (!mbar_wait_bounded(&full[s], (kt / stages) & 1, wait)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = smem_u32(sb + s * TC_STAGE_BYTES);
      const uint32_t a_lo = a_hi + TC_TILE_BYTES;
      const uint32_t b_hi = a_hi + 2 * TC_TILE_BYTES;
      const uint32_t b_lo = a_hi + 3 * TC_TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; kk++) {
        const uint32_t off = kk * 32;   // 8 TF32 values = 32 bytes along K
        umma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), (kt | kk) != 0);
        umma_tf32(tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), 1);
        umma_tf32(tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), 1);
      }
      umma_commit(&empty[s]);
    }
    umma_commit(done);
  }
  __syncwarp();

  // epilogue: lane (row) 32*warp + lane of the accumulator
  if (!mbar_wait_bounded(done, 0, wait)) s_fail = 1;
  tc_fence_after();
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      atomicExch(err, 1);
      // a wait ran out: the TMA copies already issued may still be landing
      // in this CTA's shared memory, so wait (bounded) for the last phase of
      // every stage that has one in flight before the CTA exits (the phases
      // of a stage complete in order)
      for (int kt = issued > stages ? issued - stages : 0; kt < issued; kt++)
        mbar_wait_bounded(&full[kt % stages], (kt / stages) & 1, wait);
    }
  } else {
    // accumulator rows 32*warp .. 32*warp+31 are this warp's TMEM lanes;
    // each 32 x 32 chunk goes through shared memory (the operand stages are
    // free now) so that every global access of the update is one coalesced
    // 128-byte row segment
    float* C = (pb.c_in_u ? Nm.U : Nm.L) + pb.c_off;
    float* stg = reinterpret_cast<float*>(sb) + warp * (32 * 33);
    const int ib = i0 + warp * 32;
#pragma unroll 1
    for (int c = 0; c < TC_N / 32; c++) {
      float v[32];
      tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      const int jb = j0 + c * 32;
#pragma unroll
      for (int t = 0; t < 32; t++) stg[lane * 33 + t] = v[t];
      __syncwarp();
      const int j = jb + lane;
      if (jb < pb.N && jb <= ib + 31 && ib < pb.M) {
        // all 32 row loads first, then the updates: one memory latency per chunk
        float cv[32];
#pragma unroll
        for (int rr = 0; rr < 32; rr++) {
          const int i = ib + rr;
          cv[rr] = (i < pb.M && j < pb.N && j <= i) ? C[(int64_t)i * pb.ldc + j] : 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < 32; rr++) {
          const int i = ib + rr;
          if (i < pb.M && j < pb.N && j <= i) C[(int64_t)i * pb.ldc + j] = cv[rr] - stg[rr * 33 + lane];
        }
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// split x = hi + lo, both TF32 (round to nearest)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void k_split_rows(const float* __restrict__ L, const float* __restrict__ d, int rows, int ld, int K,
                             float* __restrict__ S) {
  const int64_t plane = (int64_t)rows * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % ld);
    const float l = k < K ? L[e] : 0.f;
    const float w = k < K ? l * d[k] : 0.f;
    const float lh = to_tf32(l), wh = to_tf32(w);
    S[e] = lh;
    S[plane + e] = to_tf32(l - lh);
    S[2 * plane + e] = wh;
    S[3 * plane + e] = to_tf32(w - wh);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

bool tc_encode_maps(const float* split, int64_t rows, int64_t ld, CUtensorMap* out4, std::string* why) {
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !fn) {
      if (why) *why = "cuTensorMapEncodeTiled unavailable";
      return false;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int64_t plane = rows * ld;
  for (int a = 0; a < 4; a++) {
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_M};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(&out4[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)(split + a * plane), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      if (why) *why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      return false;
    }
  }
  return true;
}

int tc_smem_bytes() { return TC_SMEM; }

int64_t tc_tiles(int M, int N, int* Nt_out) {
  const int Mt = (M + TC_M - 1) / TC_M, Nt = (N + TC_N - 1) / TC_N;
  *Nt_out = Nt;
  return (int64_t)Nt * (Nt + 1) / 2 + (int64_t)(Mt - Nt) * Nt;
}

void launch_update_tc(const DevPlan& P, const DevNum<float>& N, const TcProb* probs, const int32_t* tile_prob,
                      int64_t ntiles, int stages, const CUtensorMap* maps, int* err, long long wait, cudaStream_t st) {
  (void)P;
  if (ntiles <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    attr = true;
  }
  stages = stages < 1 ? 1 : (stages > TC_STAGES ? TC_STAGES : stages);
  k_update_tc<<<(unsigned)ntiles, 128, tc_smem_for(stages), st>>>(N, probs, tile_prob, maps, err, stages, wait);
}

void launch_split_rows(const float* L, const float* d, int rows, int ld, int K, float* S, cudaStream_t st) {
  const int64_t n = (int64_t)rows * ld;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  k_split_rows<<<(unsigned)b, 256, 0, st>>>(L, d, rows, ld, K, S);
}

}  // namespace ncl
