// Reduced basis of a snapshot block by classical Gram-Schmidt applied twice (CGS2), with the
// rank rule of topo_rom_build, in one cooperative launch (Section 3.1: Phi spans the snapshot
// states; Section 3.4: the basis update of every trust-region step).
//
// Per snapshot column j, in order: copy it into the next free basis slot, twice subtract its
// projection on the basis so far (k dot products, one grid reduction, one update), then one
// norm reduction; the column is kept (scaled to unit norm) when that norm is at least
// drop_rel times the largest snapshot norm, else its slot is reused. Then b = Phi^T f and k
// go to device memory. Each thread owns fixed rows of every vector for the whole launch, so
// inside a CTA only the reductions synchronise; across CTAs only the per-CTA partial sums are
// shared, in two alternating buffers: a CTA can only write buffer r % 2 again after every CTA
// has passed the barrier that follows its reads of reduction r - 1. All sums run in a fixed
// order (rows by thread, warps by shuffle tree, CTAs by reduce_slots).
// Every grid barrier is bounded by wait_cycles (TOPO_ERR_TIMEOUT in the device status).
#include <algorithm>

#include "common.cuh"

namespace topo {
namespace {

constexpr int CG_THREADS = 256;
constexpr int CG_SLOTS = 129;  // up to 128 dot products or one norm per reduction
constexpr int CG_CHUNK = 16;   // dot products accumulated per pass over a CTA's rows

struct Cgs2Args {
  const double* U;  // snapshots, m columns at stride ldu
  long long ldu;
  int m;
  double* Phi;  // basis, at stride ldp (may be U)
  long long ldp;
  const double* f;
  double* b;  // b[q] = Phi_q^T f, q < k
  long long N, rows;
  double drop_rel;
  double* partial;  // [2][CG_SLOTS][G]
  int* k_out;
  GridBar* gb;
  int* status;
  long long wait_cycles;
};

// slots[q * G + cta] = this CTA's sum of acc[q] over its threads, q < nq (fixed order).
__device__ __forceinline__ void block_sums_to_slots(const double (&acc)[CG_CHUNK], int nq, double* slots,
                                                    unsigned G, double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < CG_CHUNK; ++q) {
    if (q >= nq) break;
    const double t = warp_sum(acc[q]);
    if (l == 0) red[w * CG_CHUNK + q] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < nq) {
    double t = 0.0;
    for (int ww = 0; ww < CG_THREADS / 32; ++ww) t += red[ww * CG_CHUNK + threadIdx.x];
    slots[(size_t)threadIdx.x * G + blockIdx.x] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(CG_THREADS) cgs2_kernel(const __grid_constant__ Cgs2Args a) {
  __shared__ double red[(CG_THREADS / 32) * CG_CHUNK];
  __shared__ double coef[CG_SLOTS];
  const unsigned G = gridDim.x;
  const long long r0 = (long long)blockIdx.x * a.rows, r1 = min(a.N, r0 + a.rows);
  unsigned long long bar = 0;
  int buf = 0;
  auto slots = [&](int slot) { return a.partial + ((size_t)buf * CG_SLOTS + slot) * G; };
  // per-CTA partial sums of A_q^T x over this CTA's rows, q < nq, into slots 0 .. nq - 1
  auto dots = [&](const double* A, long long lda, int nq, const double* x) {
    for (int q0 = 0; q0 < nq; q0 += CG_CHUNK) {
      const int nc = min(CG_CHUNK, nq - q0);
      double acc[CG_CHUNK];
#pragma unroll
      for (int q = 0; q < CG_CHUNK; ++q) acc[q] = 0.0;
      for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) {
        const double xi = x[i];
#pragma unroll
        for (int q = 0; q < CG_CHUNK; ++q)
          if (q < nc) acc[q] = fma(A[(long long)(q0 + q) * lda + i], xi, acc[q]);
      }
      block_sums_to_slots(acc, nc, slots(q0), G, red);
    }
  };
  auto grid_sync = [&]() { return grid_barrier(a.gb, a.status, bar, a.wait_cycles, G); };

  // the largest snapshot norm
  for (int j0 = 0; j0 < a.m; j0 += CG_CHUNK) {
    const int nc = min(CG_CHUNK, a.m - j0);
    double acc[CG_CHUNK];
#pragma unroll
    for (int q = 0; q < CG_CHUNK; ++q) acc[q] = 0.0;
    for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) {
#pragma unroll
      for (int q = 0; q < CG_CHUNK; ++q)
        if (q < nc) {
          const double u = a.U[(long long)(j0 + q) * a.ldu + i];
          acc[q] = fma(u, u, acc[q]);
        }
    }
    block_sums_to_slots(acc, nc, slots(j0), G, red);
  }
  if (!grid_sync()) return;
  reduce_slots(slots(0), G, a.m, coef);
  buf ^= 1;
  double scale = 0.0;
  for (int j = 0; j < a.m; ++j) scale = fmax(scale, sqrt(coef[j]));

  int k = 0;
  if (scale > 0.0) {
    for (int j = 0; j < a.m; ++j) {
      double* v = a.Phi + (long long)k * a.ldp;
      const double* u = a.U + (long long)j * a.ldu;
      if (v != u)
        for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) v[i] = u[i];
      for (int pass = 0; pass < 2 && k > 0; ++pass) {
        dots(a.Phi, a.ldp, k, v);
        if (!grid_sync()) return;
        reduce_slots(slots(0), G, k, coef);
        buf ^= 1;
        for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) {
          double acc = 0.0;
          for (int q = 0; q < k; ++q) acc = fma(a.Phi[(long long)q * a.ldp + i], coef[q], acc);
          v[i] = v[i] - acc;
        }
      }
      {
        double acc[CG_CHUNK];
        acc[0] = 0.0;
        for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) acc[0] = fma(v[i], v[i], acc[0]);
        block_sums_to_slots(acc, 1, slots(0), G, red);
      }
      if (!grid_sync()) return;
      reduce_slots(slots(0), G, 1, coef);
      buf ^= 1;
      const double hn = sqrt(coef[0]);
      if (hn >= a.drop_rel * scale) {
        const double s = 1.0 / hn;
        for (long long i = r0 + threadIdx.x; i < r1; i += CG_THREADS) v[i] *= s;
        ++k;
      }
      __syncthreads();  // coef is read above before the next reduction writes it
    }
  }
  if (k > 0) {
    dots(a.Phi, a.ldp, k, a.f);
    if (!grid_sync()) return;
    reduce_slots(slots(0), G, k, coef);
    if (blockIdx.x == 0)
      for (int q = threadIdx.x; q < k; q += CG_THREADS) a.b[q] = coef[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.k_out = k;
}

}  // namespace

size_t cgs2_scratch_doubles(topo_ctx* c) { return (size_t)2 * CG_SLOTS * (size_t)std::max(1, c->num_sms) + 64; }

// CGS2 of the m snapshot columns of U (stride ld) into Phi (stride ld; may be U), b = Phi^T f,
// and the rank k into k_dev (device int; 0 until the launch completes). scratch holds
// cgs2_scratch_doubles(c) doubles.
topo_status launch_cgs2(topo_ctx* c, const double* U, int m, long long ld, double* Phi, const double* f, double* b,
                        double drop_rel, double* scratch, int* k_dev) {
  const long long N = c->g.ndof;
  int occ = 0;
  TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cgs2_kernel, CG_THREADS, 0));
  if (occ < 1) return fail(c, TOPO_ERR_CUDA, "cgs2 kernel cannot be resident");
  long long G = std::max(1, c->num_sms);
  if (c->pcg_max_ctas > 0 && G > c->pcg_max_ctas) G = c->pcg_max_ctas;  // the context's share of the GPU
  long long rows = (N + G - 1) / G;
  rows = std::max(32LL, ((rows + 31) / 32) * 32);
  G = (N + rows - 1) / rows;
  Cgs2Args a;
  a.U = U;
  a.ldu = ld;
  a.m = m;
  a.Phi = Phi;
  a.ldp = ld;
  a.f = f;
  a.b = b;
  a.N = N;
  a.rows = rows;
  a.drop_rel = drop_rel;
  a.partial = scratch;
  a.k_out = k_dev;
  a.gb = c->d_bar;
  a.status = &c->d_sync->status;
  a.wait_cycles = c->wait_cycles;
  TOPO_CUDA_TRY(c, cudaMemsetAsync(c->d_bar, 0, sizeof(GridBar), c->stream));
  TOPO_CUDA_TRY(c, cudaMemsetAsync(k_dev, 0, sizeof(int), c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(CG_THREADS);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TOPO_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, cgs2_kernel, a));
  note_launch();
  return TOPO_OK;
}

}  // namespace topo
