// Tall-skinny contraction C = A^T B (A: N x k1, B: N x k2, FP32, column-major) on the
// 5th-generation tensor cores: the dense part of the reduced-precision projection
// H = Phi^T (K(rho) Phi) (Section 3.1, Eq. hatkbm; the cost term 2 N_u^e k^2 N_e of Section 3.3
// is this contraction in the paper's element-wise form).
//
// Precision. Each FP32 operand x is split exactly into hi + lo: hi is x with its low 13
// mantissa bits cleared (a TF32 number) and lo = x - hi (exact in FP32). Stacking [A_hi; A_lo]
// (128 rows) against [B_hi; B_lo] (128 columns) makes one 128 x 128 x 8 kind::tf32 MMA form all
// four products hi*hi, hi*lo, lo*hi, lo*lo, whose sum carries about 20 significant bits per
// product. Products accumulate in FP32 in TMEM over one segment (SEG chunks of 32 rows), then
// in compensated FP32 pairs in registers (about 2^-48 relative), then in FP64: once per CTA and
// in the fixed-order sum over CTAs of the caller.
//
// Pipeline (one CTA per SM; each CTA owns a contiguous row range and one 64 x 64 output tile):
//   warp 0     TMA producer: 32-row chunks of A and B (64 columns each) in a STAGES-deep ring,
//              128-byte swizzle, completion counted on full[s];
//   warps 2-5  split each landed chunk in place (hi over the raw tile, lo 8 KB above it), fence
//              the writes to the async proxy, arrive on conv[s];
//   warp 1     owns TMEM (two 128 x 128 FP32 accumulators); one lane issues 4 MMAs per chunk
//              and commits empty[s] per chunk and tfull[b] per segment;
//   warps 6-13 drain a finished accumulator with tcgen05.ld into compensated FP32 sums (two
//              warps per 32-lane quarter, each thread one accumulator row and 32 of the 64
//              output columns), release it on tempty[b]; at the end rows i and 64 + i are
//              combined into the CTA's FP64 partial tile.
// Every wait is bounded by wait_cycles. On expiry the CTA records TOPO_ERR_TIMEOUT, lets its
// copies and MMAs in flight finish (bounded again), frees its TMEM and returns.
// One CTA holds > 190 KB of shared memory, so no second CTA of this kernel (the only TMEM user
// of the library) shares its SM, and the TMEM allocation cannot wait on another CTA.
#include <cuda.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace topo {
namespace {

constexpr int KCH = 32;               // reduction rows per chunk: 128 B of FP32 = one swizzle row
constexpr int STAGES = 6;             // chunks in flight
constexpr int HALF = 8192;            // one 64-row x 128-B operand tile
constexpr int STAGE_BYTES = 4 * HALF; // A_hi | A_lo | B_hi | B_lo
constexpr int SEG = 8;                // chunks accumulated in FP32 before an FP64 drain
constexpr int NTHREADS = 448;       // warps 0-1 issue, 2-5 split, 6-13 drain
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 512;

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28; M = N = 128.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// s + c += v, compensated (Knuth's TwoSum): s carries the rounded sum, c the accumulated
// rounding errors, so the pair holds the running sum to about 2^-48 relative. FP32 only:
// FP64 runs at 1/64 of the FP32 rate on GB300.
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v) {
  const float t = __fadd_rn(s, v);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
  s = t;
  c = __fadd_rn(c, err);
}

__global__ void __launch_bounds__(NTHREADS, 1)
    atb_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int k1, int k2,
                  long long N, long long rows_per_cta, double* __restrict__ partial, int* status,
                  long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment in the shared window (the swizzle atoms repeat every 1024 B)
  unsigned char* base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = (uint64_t*)(base + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = full + STAGES;
  uint64_t* conv = empty + STAGES;
  uint64_t* tfull = conv + STAGES;  // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* done = tempty + 2;      // [1]
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_j = (k2 + 63) / 64;
  const int i0 = (blockIdx.y / tiles_j) * 64, j0 = (blockIdx.y % tiles_j) * 64;
  const long long r_begin = (long long)blockIdx.x * rows_per_cta;
  const long long r_end = min(N, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + KCH - 1) / KCH);
  const int nseg = (nchunks + SEG - 1) / SEG;
  const Ctl ctl{abort_flag, status, wait_cycles};

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
      mbar_init(su32(&conv[s]), 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&tfull[b]), 1);
      mbar_init(su32(&tempty[b]), 8);
    }
    mbar_init(su32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t stage0 = su32(base);

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int issued = 0;
      for (int ci = 0; ci < nchunks; ++ci) {
        const int s = ci % STAGES, u = ci / STAGES;
        if (u >= 1 && !wait_bar(su32(&empty[s]), (u - 1) & 1, ctl, true)) break;
        const uint32_t fb = su32(&full[s]);
        mbar_expect_tx(fb, 2 * HALF);
        const int x = (int)(r_begin + (long long)ci * KCH);
        const uint32_t dst = stage0 + s * STAGE_BYTES;
        tma_load_2d(dst, &tmA, x, i0, fb);
        tma_load_2d(dst + 2 * HALF, &tmB, x, j0, fb);
        ++issued;
      }
      // copies in flight land before the CTA may leave
      const Ctl td{abort_flag, status, kTeardownCycles};
      for (int ci = max(0, issued - STAGES); ci < issued; ++ci)
        wait_bar(su32(&full[ci % STAGES]), (ci / STAGES) & 1, td, false);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      bool ok = true;
      for (int q = 0; q < nseg && ok; ++q) {
        const int b = q & 1;
        if (q >= 2 && !wait_bar(su32(&tempty[b]), ((q >> 1) - 1) & 1, ctl, true)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * 128);
        const int cend = min(nchunks, (q + 1) * SEG);
        for (int ci = q * SEG; ci < cend; ++ci) {
          const int s = ci % STAGES;
          if (!wait_bar(su32(&conv[s]), (ci / STAGES) & 1, ctl, true)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = stage0 + s * STAGE_BYTES;
          const uint64_t da = smem_desc_sw128(st), db = smem_desc_sw128(st + 2 * HALF);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // K = 8 TF32 = 32 B per MMA: advance the start address by 32 B
            tc_mma(dt, da + 2 * kk, db + 2 * kk, (ci > q * SEG || kk > 0) ? 1u : 0u);
          tc_commit(su32(&empty[s]));
        }
        if (ok) tc_commit(su32(&tfull[b]));
      }
      // every MMA issued by this thread completes before TMEM is released
      tc_commit(su32(done));
      const Ctl td{abort_flag, status, kTeardownCycles};
      wait_bar(su32(done), 0, td, false);
    }
  } else if (warp < 6) {
    // ---- split: x -> hi (in place) + lo (8 KB above) ----
    const int t = threadIdx.x - 64;
    for (int ci = 0; ci < nchunks; ++ci) {
      const int s = ci % STAGES;
      const bool ok = wait_bar(su32(&full[s]), (ci / STAGES) & 1, ctl, true);
      if (!__all_sync(0xffffffffu, ok)) break;
      unsigned char* st = base + s * STAGE_BYTES;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4* hi = (float4*)(st + h * 2 * HALF);
        float4* lo = (float4*)(st + h * 2 * HALF + HALF);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int f = t + 128 * q;
          const float4 v = hi[f];
          float4 a, d;
          a.x = tf32_hi(v.x);
          a.y = tf32_hi(v.y);
          a.z = tf32_hi(v.z);
          a.w = tf32_hi(v.w);
          d.x = v.x - a.x;
          d.y = v.y - a.y;
          d.z = v.z - a.z;
          d.w = v.w - a.w;
          hi[f] = a;
          lo[f] = d;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(&conv[s]));
    }
  } else {
    // ---- drain: TMEM (FP32) -> compensated FP32 pairs in registers; thread = accumulator row ----
    const int quarter = warp & 3;  // this warp may read TMEM lanes 32 * quarter ... + 31
    const int row = 32 * quarter + lane;
    const int c0 = 32 * ((warp - 6) >> 2);  // output columns c0 ... c0 + 31 of the tile
    float accs[32], accc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) accs[j] = accc[j] = 0.0f;
    int drained = 0;
    for (int q = 0; q < nseg; ++q) {
      const int b = q & 1;
      const bool ok = wait_bar(su32(&tfull[b]), (q >> 1) & 1, ctl, true);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * 128);
#pragma unroll
      for (int cb = 0; cb < 32; cb += 8) {
        uint32_t r0[8], r1[8];
        tc_ld8(ta + c0 + cb, r0);       // [A_hi or A_lo row] x B_hi columns
        tc_ld8(ta + 64 + c0 + cb, r1);  // [A_hi or A_lo row] x B_lo columns
        tc_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          two_sum_add(accs[cb + i], accc[cb + i], __uint_as_float(r0[i]));
          two_sum_add(accs[cb + i], accc[cb + i], __uint_as_float(r1[i]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(&tempty[b]));
      ++drained;
    }
    // combine row i (A_hi) with row 64 + i (A_lo) through shared memory; every stage is idle
    // once the last accumulator has been drained
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const bool complete = (drained == nseg) && !*abort_flag;
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (complete) {
      double* X = (double*)base;  // 64 x 65
      if (row >= 64) {
#pragma unroll
        for (int j = 0; j < 32; ++j) X[(row - 64) * 65 + c0 + j] = (double)accs[j] + (double)accc[j];
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (row < 64 && i0 + row < k1) {
        double* out = partial + (size_t)blockIdx.x * k1 * k2 + (size_t)(i0 + row) * k2;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j0 + c0 + j < k2) out[j0 + c0 + j] = ((double)accs[j] + (double)accc[j]) + X[row * 65 + c0 + j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

bool encode_map_f32_2d(CUtensorMap* m, const float* A, long long ld, long long rows, long long cols, unsigned box_x,
                       unsigned box_y, bool swizzle128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {box_x, box_y};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D map of an FP32 column-major N x k block: x = row (contiguous), y = column; box 32 x 64
// with the 128-byte swizzle; rows >= N and columns >= k read as zero.
static bool make_map(CUtensorMap* m, const float* A, long long lda, int k, long long N) {
  return encode_map_f32_2d(m, A, lda, N, k, KCH, 64, true);
}

topo_status launch_atb_tc_partial(topo_ctx* c, const float* A, long long lda, int k1, const float* B, long long ldb,
                                  int k2, long long N, double* partial, size_t partial_cap, int* G_out) {
  if (k1 < 1 || k2 < 1 || k1 > 128 || k2 > 128 || N < 1 || N > 0x7fffffffLL)
    return fail(c, TOPO_ERR_INVALID, "internal: tensor-core contraction shape out of range");
  if ((lda % 4) || (ldb % 4) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return fail(c, TOPO_ERR_INVALID, "internal: tensor-core contraction needs 16-byte aligned columns");
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, lda, k1, N) || !make_map(&mb, B, ldb, k2, N))
    return fail(c, TOPO_ERR_CUDA, "cuTensorMapEncodeTiled failed for the projection operands");
  const int tiles = ((k1 + 63) / 64) * ((k2 + 63) / 64);
  long long G = std::max(1, (c->num_sms + tiles - 1) / tiles);
  long long rows = (N + G - 1) / G;
  rows = ((rows + KCH - 1) / KCH) * KCH;
  G = (N + rows - 1) / rows;
  if ((size_t)G * k1 * k2 > partial_cap) return fail(c, TOPO_ERR_INVALID, "internal: atb partial buffer too small");
  TOPO_CUDA_TRY(c, cudaFuncSetAttribute(atb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  atb_tc_kernel<<<dim3((unsigned)G, tiles), NTHREADS, SMEM_BYTES, c->stream>>>(
      ma, mb, k1, k2, N, rows, partial, &c->d_sync->status, c->wait_cycles);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  *G_out = (int)G;
  return TOPO_OK;
}

}  // namespace topo
