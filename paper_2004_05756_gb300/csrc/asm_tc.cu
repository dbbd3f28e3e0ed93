// Reduced matrices of many candidate designs on the 5th-generation tensor cores, to FP64
// accuracy: H_r = sum_e E(rho_r,e) Hel_e (Section 3.4 and Remark rom_assemble: the part of the
// reduced operator that changes with the density), computed as the contraction
// C[r][p] = sum_e E[r][e] Hel[e][p] over the element rows e of one basis.
//
// Exact operand splitting: the Ozaki scheme (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), in the form that runs it on low-precision
// tensor cores with FP32 accumulation (Mukunoki, Ozaki, Ogita and Imamura, "DGEMM using Tensor
// Cores, and Its Accurate and Reproducible Versions", ISC High Performance 2020):
//   - balancing: element e's term E[r][e] Hel[e][p] is written as (E[r][e] s_e)(Hel[e][p] / s_e)
//     with s_e the power of two of the largest |Hel[e][.]| of the CTA's columns. SIMP moduli span
//     1e-9 .. 1 and element matrices of a snapshot basis the inverse range (soft elements move
//     most), so without it a scale common to all elements would cost the soft elements' terms
//     up to 30 bits; with it both operands are balanced along the sum (a diagonal scaling of the
//     inner dimension by powers of two, exact). s_e depends on the basis only, so a candidate's
//     result does not depend on the other candidates;
//   - over one CTA's element rows, row r of E s and column p of Hel / s each get a power-of-two
//     scale tau above their largest magnitude; |x| / tau * 2^55 is truncated to an integer
//     q < 2^55;
//   - q is written as 8 balanced base-128 digits, q = sum_i d_i 128^(7 - i), |d_i| <= 64, each
//     exact in BF16;
//   - a product of two digits is an integer of magnitude <= 4096, exact in FP32. Level
//     l = i + j gathers the at most 8 digit pairs of one order, so one element row adds at most
//     2^15 to a level and 512 rows at most 2^24: the FP32 sums of the MMAs are exact integers
//     over 512 element rows;
//   - levels 0..7 are kept. The dropped levels and the truncation of q change a product by
//     about 2^-55 of the scales' product per operand (2^-55 tau_E |Hel / s| + 2^-55 tau_H |E s|
//     plus 2^-53 |E Hel| for the dropped levels), the size of an FP64 rounding of the sum;
//   - every 512 rows the levels are combined as sum_l V_l 2^(-7 l) in FP64 registers, and the
//     sum is scaled back by tau_r tau_p 2^-12 at the end of the range.
// Each candidate's result depends only on its own row of E (exact integer sums, fixed-order FP64
// combination), so it is the same alone and inside a batch.
//
// One CTA per SM (194 KB of shared memory), 256 threads; CTA (g, t) owns element rows
// [g * rows_per_cta, ...) and output columns [64 t, 64 t + 64). Per block of 64 element rows:
//   all threads  read the FP64 block of E (128 candidate rows) and of Hel (64 columns), split
//                each value into its 8 digits and write one BF16 tile per digit in the K-major,
//                128-byte-swizzled layout of the MMA descriptors, then fence the tiles to the
//                async proxy;
//   thread 0     issues 36 digit pairs x 4 MMAs (kind::f16, BF16 inputs, M = 128, N = 64,
//                K = 16) into 8 FP32 accumulators of 64 TMEM columns, one per level, and commits
//                them to an mbarrier;
//   all threads  wait for the commit before the tiles are written again; every 8 blocks and at
//                the end of the range they drain the 8 levels with tcgen05.ld into FP64 sums.
// The balancing exponents s_e are formed per block (warp maxima over 32 columns, two per element
// combined in shared memory); a pre-pass over the CTA's rows forms the scales tau from the
// balanced exponents the same way.
// Every wait is bounded by wait_cycles. On expiry the CTA records TOPO_ERR_TIMEOUT, waits
// (bounded again) for the MMAs it issued, frees its TMEM and returns without writing.
// One CTA holds more than half of the SM's shared memory, so no second CTA of this kernel or of
// the projection contraction (the library's other TMEM user) shares its SM, and the allocation
// of all 512 TMEM columns cannot wait on another CTA.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace topo {
namespace {

constexpr int OZ_M = 128;          // candidate rows of one MMA (TMEM lanes)
constexpr int OZ_N = 64;           // output columns of one CTA (packed pairs)
constexpr int OZ_KB = 64;          // element rows per block: 128 B of BF16, one swizzle row
constexpr int OZ_D = 8;            // digits per operand
constexpr int OZ_DRAIN = 8;        // blocks (512 element rows) of exact FP32 accumulation
constexpr int OZ_THREADS = 256;
constexpr int A_TILE = OZ_M * 128;  // one digit of the E block (16 KB)
constexpr int B_TILE = OZ_N * 128;  // one digit of the Hel block (8 KB)
constexpr int OZ_TAIL = 2048;       // barriers, TMEM slot, abort flag, exponents and flags
constexpr int OZ_SMEM = 1024 + OZ_D * (A_TILE + B_TILE) + OZ_TAIL;

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28; M = 128, N = 64.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_N >> 3) << 17) |
                              ((uint32_t)(OZ_M >> 4) << 24);

__device__ __forceinline__ void tc_mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(OZ_IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ int biased_exponent(const double* p) {
  return (int)((((const unsigned*)p)[1] >> 20) & 0x7ffu);  // the high word of the little-endian double
}

// The 8 balanced base-128 digits of q = trunc(|x 2^off| / 2^(mx - 1022) * 2^55) with the sign
// of x, most significant first. mx >= the biased exponent of x 2^off, so q < 2^55:
// q = (53-bit significand << 2) >> (mx - exponent - off). Zero and subnormal x give 0.
__device__ __forceinline__ void oz_digits(double x, int mx, int off, int (&d)[OZ_D]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ffu);
  const int sh = mx - ex - off;
  unsigned long long q = 0;
  if (ex != 0 && sh >= 0 && sh < 55) q = (((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2) >> sh;
  int carry = 0;
#pragma unroll
  for (int i = OZ_D - 1; i >= 1; --i) {
    const int u = (int)((q >> (7 * (OZ_D - 1 - i))) & 127u) + carry;  // 0 .. 128
    carry = u >= 64 ? 1 : 0;
    d[i] = u - 128 * carry;  // -64 .. 63
  }
  d[0] = (int)(q >> 49) + carry;  // 0 .. 64
  if (b >> 63) {
#pragma unroll
    for (int i = 0; i < OZ_D; ++i) d[i] = -d[i];
  }
}

// An integer |d| <= 2^22 as FP32 without a conversion instruction: 1.5 * 2^23 + d is exact.
__device__ __forceinline__ float small_int_to_float(int d) { return __int_as_float(0x4B400000 + d) - 12582912.0f; }

// Split 8 consecutive K values of one operand row, value j balanced by 2^(sgn * (sexp[j] - 1023)),
// into the 8 digit tiles (16 bytes each).
__device__ __forceinline__ void oz_store_unit(unsigned char* tiles, int tile_bytes, int row, int chunk,
                                              const double (&v)[8], int mx, const int* sexp, int sgn) {
  int d[8][OZ_D];
#pragma unroll
  for (int j = 0; j < 8; ++j) oz_digits(v[j], mx, sgn * (sexp[j] - 1023), d[j]);
  const uint32_t off = sw128_offset(row, chunk);
#pragma unroll
  for (int i = 0; i < OZ_D; ++i) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __nv_bfloat162 b2 =
          __floats2bfloat162_rn(small_int_to_float(d[2 * h][i]), small_int_to_float(d[2 * h + 1][i]));
      w[h] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(tiles + i * tile_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// sexp[j] = the largest biased exponent of Hel[e0 + j][p0 .. p0 + 63] (Inf and NaN left out, 0
// where all are zero), for the block's 64 element rows. Thread t takes column t % 64 and rows
// t / 64 + 4 i (eh[i], all loads issued first): a warp maximum over its 32 columns, then one
// atomic per warp and row. Ends with a block barrier.
constexpr int OZ_HROWS = OZ_KB / (OZ_THREADS / OZ_N);  // 16 block rows of Hel per thread
__device__ __forceinline__ void oz_block_balance(const double* __restrict__ Hel, int npair, int p0, long long e0,
                                                 long long e_end, int* sexp, int (&eh)[OZ_HROWS]) {
  const int t = threadIdx.x, n = t & (OZ_N - 1), j0 = t / OZ_N;
#pragma unroll
  for (int i = 0; i < OZ_HROWS; ++i) {
    const int j = j0 + 4 * i;
    eh[i] = (p0 + n < npair && e0 + j < e_end) ? biased_exponent(Hel + (e0 + j) * npair + p0 + n) : 0;
  }
#pragma unroll
  for (int i = 0; i < OZ_HROWS; ++i) {
    const int m = __reduce_max_sync(0xffffffffu, eh[i] == 0x7ff ? 0 : eh[i]);
    if ((t & 31) == 0) atomicMax(&sexp[j0 + 4 * i], m);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    asm_oz_kernel(const double* __restrict__ Hel, const double* __restrict__ E, long long rows, long long ldE,
                  int npair, int nr, long long rows_per_cta, double* __restrict__ partial, int* status,
                  long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment in the shared window (the swizzle atoms repeat every 1024 B)
  unsigned char* base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  unsigned char* tilesA = base;
  unsigned char* tilesB = base + OZ_D * A_TILE;
  unsigned char* tail = tilesB + OZ_D * B_TILE;
  uint64_t* mma_bar = (uint64_t*)tail;
  uint64_t* done_bar = mma_bar + 1;
  uint32_t* tmem_slot = (uint32_t*)(done_bar + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* rexp = (int*)(tail + 64);  // [OZ_M] scale exponents of E's balanced rows
  int* cexp = rexp + OZ_M;        // [OZ_N] scale exponents of Hel's balanced columns
  int* rbad = cexp + OZ_N;        // [OZ_M] rows holding Inf or NaN
  int* cbad = rbad + OZ_M;        // [OZ_N] columns holding Inf or NaN
  int* sexp = cbad + OZ_N;        // [OZ_KB] balancing exponents of the current block

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p0 = blockIdx.y * OZ_N;
  const long long e_begin = (long long)blockIdx.x * rows_per_cta;
  const long long e_end = min(rows, e_begin + rows_per_cta);
  const int nkb = (int)((e_end - e_begin + OZ_KB - 1) / OZ_KB);
  const Ctl ctl{abort_flag, status, wait_cycles};

  if (tid == 0) {
    mbar_init(su32(mma_bar), 1);
    mbar_init(su32(done_bar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < OZ_M) rexp[tid] = rbad[tid] = 0;
  if (tid < OZ_N) cexp[tid] = cbad[tid] = 0;
  if (tid < OZ_KB) sexp[tid] = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // ---- scale exponents of the balanced operands over this CTA's element rows ----
  for (int kb = 0; kb < nkb; ++kb) {
    const long long e0 = e_begin + (long long)kb * OZ_KB;
    int eh[OZ_HROWS];
    oz_block_balance(Hel, npair, p0, e0, e_end, sexp, eh);
    // columns of Hel / s: this thread's column tid % 64 at rows tid / 64 + 4 i
    {
      const int n = tid & (OZ_N - 1), j0 = tid / OZ_N;
      int m = 0, bad = 0;
#pragma unroll
      for (int i = 0; i < OZ_HROWS; ++i) {
        if (eh[i] == 0x7ff) bad = 1;
        else if (eh[i] != 0) m = max(m, eh[i] - sexp[j0 + 4 * i] + 1023);
      }
      atomicMax(&cexp[n], m);
      if (bad) cbad[n] = 1;
    }
    // rows of E s: thread = element tid % 64, rows tid / 64 + 4 i (loads first); warp maxima
    // over 32 elements, one atomic per warp and row
    {
      const int e = tid & (OZ_KB - 1), se = sexp[e];
      int ex[OZ_M / 4];
#pragma unroll
      for (int i = 0; i < OZ_M / 4; ++i) {
        const int r = (tid >> 6) + 4 * i;
        ex[i] = (r < nr && e0 + e < e_end) ? biased_exponent(E + r * ldE + e0 + e) : 0;
      }
#pragma unroll
      for (int i = 0; i < OZ_M / 4; ++i) {
        const int r = (tid >> 6) + 4 * i;
        const int bad = ex[i] == 0x7ff;
        const int v = (ex[i] != 0 && !bad && se != 0) ? ex[i] + se - 1023 : 0;
        const int mv = __reduce_max_sync(0xffffffffu, v);
        const int mb = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0 && r < nr) {
          atomicMax(&rexp[r], mv);
          if (mb) rbad[r] = 1;
        }
      }
    }
    __syncthreads();
    if (tid < OZ_KB) sexp[tid] = 0;
    __syncthreads();
  }

  // drain role: TMEM lanes 32 (warp % 4) ... (candidate rows), output columns c0 .. c0 + 31
  const int quarter = warp & 3, c0 = 32 * (warp >> 2);
  double acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.0;
  bool ok = true;
  for (int kb = 0; kb < nkb; ++kb) {
    if (kb > 0) {  // the MMAs of the previous block have read the tiles
      ok = wait_bar(su32(mma_bar), (kb - 1) & 1, ctl, true);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
    }
    const long long e0 = e_begin + (long long)kb * OZ_KB;
    {
      int eh[OZ_HROWS];
      oz_block_balance(Hel, npair, p0, e0, e_end, sexp, eh);
    }
    // E block: unit = (candidate row, 8-row chunk), 4 per thread
#pragma unroll 1
    for (int s = 0; s < (OZ_M * 8) / OZ_THREADS; ++s) {
      const int u = tid + OZ_THREADS * s, row = u >> 3, ch = u & 7;
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long e = e0 + 8 * ch + j;
        v[j] = (row < nr && e < e_end) ? __ldg(E + row * ldE + e) : 0.0;
      }
      oz_store_unit(tilesA, A_TILE, row, ch, v, rexp[row], sexp + 8 * ch, 1);
    }
    // Hel block: unit = (pair column, 8-row chunk), 2 per thread; lanes run along the columns
#pragma unroll 1
    for (int s = 0; s < (OZ_N * 8) / OZ_THREADS; ++s) {
      const int u = tid + OZ_THREADS * s, col = u & (OZ_N - 1), ch = u / OZ_N;
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long e = e0 + 8 * ch + j;
        v[j] = (p0 + col < npair && e < e_end) ? __ldg(Hel + e * npair + p0 + col) : 0.0;
      }
      oz_store_unit(tilesB, B_TILE, col, ch, v, cexp[col], sexp + 8 * ch, -1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid < OZ_KB) sexp[tid] = 0;  // read again only after the next block's barrier
    const bool first = (kb % OZ_DRAIN) == 0;
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int i = 0; i < OZ_D; ++i) {
        const uint64_t da = smem_desc_sw128(su32(tilesA + i * A_TILE));
#pragma unroll 1
        for (int j = 0; i + j < OZ_D; ++j) {
          const uint64_t db = smem_desc_sw128(su32(tilesB + j * B_TILE));
          const uint32_t dt = tmem + (uint32_t)((i + j) * OZ_N);  // level i + j
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // K = 16 BF16 = 32 B per MMA
            tc_mma_bf16(dt, da + 2 * kk, db + 2 * kk, (first && i == 0 && kk == 0) ? 0u : 1u);
        }
      }
      tc_commit(su32(mma_bar));
    }
    if ((kb % OZ_DRAIN) == OZ_DRAIN - 1 || kb == nkb - 1) {
      ok = wait_bar(su32(mma_bar), kb & 1, ctl, true);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
#pragma unroll
      for (int cb = 0; cb < 32; cb += 8) {
        uint32_t v[OZ_D][8];
#pragma unroll
        for (int l = 0; l < OZ_D; ++l) tc_ld8(ta + (uint32_t)(l * OZ_N + cb), v[l]);
        tc_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          double t = (double)__uint_as_float(v[OZ_D - 1][i]);
#pragma unroll
          for (int l = OZ_D - 2; l >= 0; --l) t = fma(t, 0x1p-7, (double)__uint_as_float(v[l][i]));
          acc[cb + i] += t;
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  // every MMA this CTA issued completes before its TMEM is released
  if (tid == 0) {
    tc_commit(su32(done_bar));
    const Ctl td{abort_flag, status, kTeardownCycles};
    wait_bar(su32(done_bar), 0, td, false);
  }
  tc_fence_before();
  __syncthreads();
  const bool complete = ok && !*abort_flag;
  if (complete) {
    const int row = 32 * quarter + lane;
    if (row < nr) {
      const int er = rexp[row], rb = rbad[row];
      double* out = partial + ((size_t)blockIdx.x * nr + row) * npair;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = c0 + j;
        if (p0 + col < npair) {
          // Inf or NaN in the row or column: the digits are meaningless, the sum is NaN
          out[p0 + col] = (rb || cbad[col]) ? __longlong_as_double(0x7ff8000000000000LL)
                                            : ldexp(acc[j], (er - 1022) + (cexp[col] - 1022) - 12);
        }
      }
    }
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

// Partial sums partial[g][r][p] = sum over the element rows of chunk g of E[r][e] Hel[e][p] for
// r < nr <= 128, p < npair; *G_out receives the number of chunks (the caller's fixed-order
// final sum runs over them).
topo_status launch_asm_tc_partial(topo_ctx* c, const double* Hel, const double* E, long long rows, long long ldE,
                                  int npair, int nr, double* partial, size_t partial_cap, int* G_out) {
  if (nr < 1 || nr > OZ_M || npair < 1 || rows < 1 || ldE < rows)
    return fail(c, TOPO_ERR_INVALID, "internal: tensor-core assembly shape out of range");
  const int tiles = (npair + OZ_N - 1) / OZ_N;
  if (tiles > 65535) return fail(c, TOPO_ERR_INVALID, "internal: tensor-core assembly has too many columns");
  long long G = std::max(1, c->num_sms / tiles);
  long long per = (rows + G - 1) / G;
  per = ((per + OZ_KB - 1) / OZ_KB) * OZ_KB;
  G = (rows + per - 1) / per;
  if ((size_t)G * nr * npair > partial_cap) return fail(c, TOPO_ERR_INVALID, "internal: assembly partials too small");
  TOPO_CUDA_TRY(c, cudaFuncSetAttribute(asm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  asm_oz_kernel<<<dim3((unsigned)G, (unsigned)tiles), OZ_THREADS, OZ_SMEM, c->stream>>>(
      Hel, E, rows, ldE, npair, nr, per, partial, &c->d_sync->status, c->wait_cycles);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  *G_out = (int)G;
  return TOPO_OK;
}

long long asm_tc_chunks(topo_ctx* c, long long rows, int npair) {
  const int tiles = (npair + OZ_N - 1) / OZ_N;
  long long G = std::max(1, c->num_sms / tiles);
  long long per = (rows + G - 1) / G;
  per = ((per + OZ_KB - 1) / OZ_KB) * OZ_KB;
  return (rows + per - 1) / per;
}

}  // namespace topo
