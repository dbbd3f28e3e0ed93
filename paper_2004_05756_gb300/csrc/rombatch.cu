// topo_rom_eval_batch: ROM design evaluations of many candidate designs on one resident basis
// (Section 3.1 Eq. rom_soln, Section 3.3, Section 3.4), in one call.
//
// A trust-region step (Algorithm 2) evaluates many candidates on the same basis. Evaluated one
// by one, every candidate streams the element reduced matrices Hel again and pays a dozen
// small launches whose latency exceeds their work. Here the candidates share every launch:
//   rho_r = filter(psi_r)                          one launch (grid.y = candidate)
//   H_r = sum_e E(rho_r,e) Hel_e                    tensor cores (csrc/asm_tc.cu, the default):
//                                                   Hel read once per 128 candidates, Ozaki
//                                                   digits in BF16, exact FP32 sums, FP64 result;
//                                                   or FP64 SIMT: Hel read once per group of RC
//                                                   candidates, RC accumulators per thread and pair
//   y_r = H_r^-1 b, J_k,r = b^T y_r                 one warp per candidate
//   u_r = Phi y_r                                   Phi read once per group
//   ||f - K(rho_r) u_r||, its ratio to ||f||,      one launch (grid.y = candidate) on staged
//   dc_r = -E'(rho_r) u_r,e^T K_e u_r,e             tiles of u_r; the adjoint filter of dc_r
//                                                   one more
// Every sum runs in a fixed order, so each candidate's results are bitwise independent of the
// others in the batch.
#include <algorithm>

#include "common.cuh"

namespace topo {

constexpr int RC = 32;   // candidates per group (FP64 accumulators per thread)
constexpr int SG = 128;  // candidates per tensor-core assembly (the MMA's M)

topo_status launch_reduced_solve_batch(topo_ctx* c, int k, int R, const double* b, double* H, double* y, double* J,
                                       int* ok);
topo_status launch_asm_tc_partial(topo_ctx* c, const double* Hel, const double* E, long long rows, long long ldE,
                                  int npair, int nr, double* partial, size_t partial_cap, int* G_out);
long long asm_tc_chunks(topo_ctx* c, long long rows, int npair);

// E(rho_r,e) for R designs (N_e + 1 rows each: the last row, weight 1, carries Phi_D^T Phi_D).
__global__ void moduli_batch_kernel(Grid g, const double* rho, long long ldr, double* E, int R) {
  const long long rows = g.nel + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows * R;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / rows, e = t % rows;
    E[t] = e < g.nel ? young<double>(rho[r * ldr + e], g.E0, g.Emin, g.ipenal) : 1.0;
  }
}

// partial[g][r][p] = sum over the CTA's rows e of E[r][e] Hel[e][p] for the nr <= RC candidates
// of the group (rows of E at stride ldE). Thread = pair p (grid.y covers the pairs); the group's
// moduli for a chunk of rows are staged in shared memory and read as broadcasts.
constexpr int ASM_ROWS = 32;
__global__ void __launch_bounds__(256) assemble_multi_partial_kernel(const double* __restrict__ Hel,
                                                                     const double* __restrict__ E, long long rows,
                                                                     long long ldE, int npair, int nr,
                                                                     long long rows_per_cta, double* partial) {
  __shared__ double Es[RC][ASM_ROWS];
  const int p = blockIdx.y * blockDim.x + threadIdx.x;
  const long long r0 = blockIdx.x * rows_per_cta, r1 = min(rows, r0 + rows_per_cta);
  double acc[RC];
#pragma unroll
  for (int q = 0; q < RC; ++q) acc[q] = 0.0;
  for (long long c0 = r0; c0 < r1; c0 += ASM_ROWS) {
    const int nrow = (int)min((long long)ASM_ROWS, r1 - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < RC * ASM_ROWS; t += blockDim.x) {
      const int q = t / ASM_ROWS, e = t % ASM_ROWS;
      Es[q][e] = (q < nr && e < nrow) ? __ldg(E + (size_t)q * ldE + c0 + e) : 0.0;
    }
    __syncthreads();
    if (p < npair) {
      for (int e = 0; e < nrow; ++e) {
        const double h = __ldcs(Hel + (c0 + e) * npair + p);
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = fma(Es[q][e], h, acc[q]);
      }
    }
  }
  if (p < npair)
    for (int q = 0; q < nr; ++q) partial[((size_t)blockIdx.x * nr + q) * npair + p] = acc[q];
}

// H_r (k x k row-major, symmetric) = sum over the G partials, for the nr candidates: a warp
// per entry, lanes summing g = lane, lane + 32, ... in order, then a shuffle tree (fixed order).
__global__ void assemble_multi_final_kernel(const double* __restrict__ partial, int G, int k, int nr, double* H) {
  const int npair = k * (k + 1) / 2;
  const int l = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < (long long)nr * npair; t += nw) {
    const int q = (int)(t / npair), p = (int)(t % npair);
    double s = 0.0;
    for (int g = l; g < G; g += 32) s += __ldcg(partial + ((size_t)g * nr + q) * npair + p);
    s = warp_sum(s);
    if (l != 0) continue;
    int i = 0, rem = p;
    while (rem >= k - i) {
      rem -= k - i;
      ++i;
    }
    const int j = i + rem;
    double* Hq = H + (size_t)q * k * k;
    Hq[i * k + j] = s;
    Hq[j * k + i] = s;
  }
}

// U[r][i] = sum_q Phi[q][i] y[r][q] for the nr <= RC candidates of a group (column stride ldu).
__global__ void __launch_bounds__(256) basis_combine_kernel(const double* __restrict__ Phi, long long ld, int k,
                                                            const double* __restrict__ Y, int nr, long long N,
                                                            double* U, long long ldu) {
  extern __shared__ double Ys[];  // [RC][k]
  for (int t = threadIdx.x; t < RC * k; t += blockDim.x) Ys[t] = (t / k) < nr ? Y[t] : 0.0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = 0.0;
    for (int j = 0; j < k; ++j) {
      const double ph = __ldg(Phi + (long long)j * ld + i);
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = fma(ph, Ys[q * k + j], acc[q]);
    }
    for (int q = 0; q < nr; ++q) U[(long long)q * ldu + i] = acc[q];
  }
}

// H[r] (k x k, row-major) = sum_e E[r][e] Hel[e] for nr candidates whose moduli rows (rows =
// N_e + 1 each) sit at stride ldE: tensor cores in one pass when the context selects them and
// nr <= SG, else FP64 SIMT in groups of RC. part holds part_cap doubles.
static topo_status assemble_reduced(topo_ctx* c, const double* Hel, const double* E, long long rows, long long ldE,
                                    int k, int nr, double* part, size_t part_cap, double* H) {
  const int npair = k * (k + 1) / 2;
  const int fin_blocks = (int)std::min<long long>(8LL * c->num_sms, ((long long)nr * npair + 7) / 8);
  if (c->rom_asm_tensor && nr <= SG) {
    int G = 0;
    topo_status s = launch_asm_tc_partial(c, Hel, E, rows, ldE, npair, nr, part, part_cap, &G);
    if (s) return s;
    assemble_multi_final_kernel<<<fin_blocks, 256, 0, c->stream>>>(part, G, k, nr, H);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    return TOPO_OK;
  }
  long long G = 2LL * c->num_sms;
  long long per = (rows + G - 1) / G;
  per = ((per + ASM_ROWS - 1) / ASM_ROWS) * ASM_ROWS;
  G = (rows + per - 1) / per;
  if ((size_t)G * std::min(nr, RC) * npair > part_cap)
    return fail(c, TOPO_ERR_INVALID, "internal: assembly partials too small");
  for (int r0 = 0; r0 < nr; r0 += RC) {
    const int ng = std::min(RC, nr - r0);
    assemble_multi_partial_kernel<<<dim3((unsigned)G, (npair + 255) / 256), std::min(256, ((npair + 31) / 32) * 32),
                                    0, c->stream>>>(Hel, E + (size_t)r0 * ldE, rows, ldE, npair, ng, per, part);
    note_launch();
    assemble_multi_final_kernel<<<(int)std::min<long long>(8LL * c->num_sms, ((long long)ng * npair + 7) / 8), 256, 0,
                                  c->stream>>>(part, (int)G, k, ng, H + (size_t)r0 * k * k);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
  }
  return TOPO_OK;
}

// Doubles of partial sums assemble_reduced needs for nr candidates.
static size_t assemble_part_doubles(topo_ctx* c, long long rows, int k, int nr) {
  const int npair = k * (k + 1) / 2;
  long long G = 2LL * c->num_sms;
  long long per = (rows + G - 1) / G;
  per = ((per + ASM_ROWS - 1) / ASM_ROWS) * ASM_ROWS;
  G = (rows + per - 1) / per;
  size_t n = (size_t)G * std::min(nr, RC) * npair;
  if (c->rom_asm_tensor && nr <= SG) n = std::max(n, (size_t)asm_tc_chunks(c, rows, npair) * nr * npair);
  return n;
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_rom_eval_batch(topo_ctx* c, int R, const double* psi, int ldp, int filtered,
                                           const double* Hel, const double* Phi, int k, int ld, const double* b,
                                           const double* f, double* Jk, double* resnorm, double* yhat,
                                           double* dpsi) {
  if (!c) return TOPO_ERR_INVALID;
  const Grid& g = c->g;
  const long long N = g.ndof, Ne = g.nel;
  if (R < 0) return fail(c, TOPO_ERR_INVALID, "topo_rom_eval_batch: R < 0");
  if (R == 0) return TOPO_OK;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_eval_batch: 1 <= k <= 128");
  if ((long long)ldp < Ne || (long long)ld < N)
    return fail(c, TOPO_ERR_INVALID, "topo_rom_eval_batch: ldp >= N_e and ld >= N required");
  if (!dev_ptr_ok(psi) || !dev_ptr_ok(Hel) || !dev_ptr_ok(Phi) || !dev_ptr_ok(b) || !dev_ptr_ok(f) ||
      !dev_ptr_ok(Jk) || !dev_ptr_ok(resnorm) || (yhat && !dev_ptr_ok(yhat)) || (dpsi && !dev_ptr_ok(dpsi)))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_eval_batch: null or misaligned pointer");
  if (dpsi && dpsi == psi) return fail(c, TOPO_ERR_INVALID, "topo_rom_eval_batch: dpsi aliases psi");
  const long long rows = Ne + 1;
  const long long tiles = residual_tiles(c);
  // candidates per assembly: 128 on the tensor cores (Hel streamed once per 128), else RC
  const int sg = std::min(R, c->rom_asm_tensor ? SG : RC);
  const size_t part_n = assemble_part_doubles(c, rows, k, sg);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_rho = take((size_t)sg * Ne * 8), o_E = take((size_t)sg * rows * 8), o_part = take(part_n * 8),
               o_H = take((size_t)sg * k * k * 8), o_y = take((size_t)sg * k * 8), o_U = take((size_t)RC * N * 8),
               o_dc = take((size_t)RC * Ne * 8), o_rp = take((size_t)RC * 2 * tiles * 8), o_ok = take((size_t)sg * 4);
  topo_status s = ensure_scratch(c, off);
  if (s) return s;
  char* base = (char*)c->d_scratch;
  double* rho = (double*)(base + o_rho);
  double* E = (double*)(base + o_E);
  double* part = (double*)(base + o_part);
  double* H = (double*)(base + o_H);
  double* ybuf = (double*)(base + o_y);
  double* U = (double*)(base + o_U);
  double* dc = (double*)(base + o_dc);
  double* rpart = (double*)(base + o_rp);
  int* ok = (int*)(base + o_ok);
  for (int s0 = 0; s0 < R; s0 += sg) {
    const int ns = std::min(sg, R - s0);
    const double* psi_s = psi + (size_t)s0 * ldp;
    // densities
    const double* rho_s = psi_s;
    long long ldr = ldp;
    if (filtered) {
      s = launch_filter_batch(c, psi_s, ldp, rho, Ne, ns, 0);
      if (s) return s;
      rho_s = rho;
      ldr = Ne;
    }
    moduli_batch_kernel<<<(int)std::min<long long>(8LL * c->num_sms, (rows * ns + 255) / 256), 256, 0, c->stream>>>(
        g, rho_s, ldr, E, ns);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    // reduced matrices and reduced solves of the super-group
    s = assemble_reduced(c, Hel, E, rows, rows, k, ns, part, part_n, H);
    if (s) return s;
    double* y_s = yhat ? yhat + (size_t)s0 * k : ybuf;
    s = launch_reduced_solve_batch(c, k, ns, b, H, y_s, Jk + s0, ok);
    if (s) return s;
    // reduced states, residual norms, gradients, in groups of RC
    for (int r0 = 0; r0 < ns; r0 += RC) {
      const int nr = std::min(RC, ns - r0);
      const double* rho_g = rho_s + (size_t)r0 * ldr;
      const double* y_g = y_s + (size_t)r0 * k;
      const size_t smem = (size_t)RC * k * sizeof(double);  // <= 32 KB for k <= 128
      basis_combine_kernel<<<(int)std::min<long long>(4LL * c->num_sms, (N + 255) / 256), 256, smem, c->stream>>>(
          Phi, ld, k, y_g, nr, N, U, N);
      note_launch();
      TOPO_CUDA_TRY(c, cudaGetLastError());
      const int rg = s0 + r0;
      // residual norms, and with dpsi the element gradients from the same staged tiles
      s = launch_residual64_batch(c, rho_g, ldr, U, N, f, resnorm + 2 * (size_t)rg, nr, rpart, dpsi ? dc : nullptr,
                                  Ne);
      if (s) return s;
      if (dpsi) {
        s = filtered ? launch_filter_batch(c, dc, Ne, dpsi + (size_t)rg * ldp, ldp, nr, 1)
                     : (cudaMemcpy2DAsync(dpsi + (size_t)rg * ldp, (size_t)ldp * 8, dc, (size_t)Ne * 8, (size_t)Ne * 8,
                                          nr, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                            ? TOPO_OK
                            : fail(c, TOPO_ERR_CUDA, "topo_rom_eval_batch: copy of the gradients"));
        if (s) return s;
      }
    }
  }
  return TOPO_OK;
}

extern "C" topo_status topo_rom_assemble_batch(topo_ctx* c, int R, const double* E, long long ldE, const double* Hel,
                                               int k, double* H) {
  if (!c) return TOPO_ERR_INVALID;
  const long long rows = c->g.nel + 1;
  if (R < 0) return fail(c, TOPO_ERR_INVALID, "topo_rom_assemble_batch: R < 0");
  if (R == 0) return TOPO_OK;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_assemble_batch: 1 <= k <= 128");
  if (ldE < rows) return fail(c, TOPO_ERR_INVALID, "topo_rom_assemble_batch: ldE >= N_e + 1 required");
  if (!dev_ptr_ok(E) || !dev_ptr_ok(Hel) || !dev_ptr_ok(H))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_assemble_batch: null or misaligned pointer");
  const int sg = std::min(R, c->rom_asm_tensor ? SG : RC);
  const size_t part_n = assemble_part_doubles(c, rows, k, sg);
  topo_status s = ensure_scratch(c, part_n * 8);
  if (s) return s;
  double* part = (double*)c->d_scratch;
  for (int s0 = 0; s0 < R; s0 += sg) {
    const int ns = std::min(sg, R - s0);
    s = assemble_reduced(c, Hel, E + (size_t)s0 * ldE, rows, ldE, k, ns, part, part_n, H + (size_t)s0 * k * k);
    if (s) return s;
  }
  return TOPO_OK;
}
