// topo_rom_eval_batch: ROM design evaluations of many candidate designs on one resident basis
// (Section 3.1 Eq. rom_soln, Section 3.3, Section 3.4), in one call.
//
// A trust-region step (Algorithm 2) evaluates many candidates on the same basis. Evaluated one
// by one, every candidate streams the element reduced matrices Hel again and pays a dozen
// small launches whose latency exceeds their work. Here the candidates share every launch:
//   rho_r = filter(psi_r)                          one launch (grid.y = candidate)
//   H_r = sum_e E(rho_r,e) Hel_e                    Hel read once per group of RC candidates,
//                                                   RC FP64 accumulators per thread and pair
//   y_r = H_r^-1 b, J_k,r = b^T y_r                 one warp per candidate
//   u_r = Phi y_r                                   Phi read once per group
//   ||f - K(rho_r) u_r||, its ratio to ||f||        one launch (grid.y = candidate)
//   dc_r = -E'(rho_r) u_r,e^T K_e u_r,e, dpsi_r      one launch each
// Every sum runs in a fixed order, so each candidate's results are bitwise independent of the
// others in the batch.
#include <algorithm>

#include "common.cuh"

namespace topo {

constexpr int RC = 32;  // candidates per group (FP64 accumulators per thread)

topo_status launch_reduced_solve_batch(topo_ctx* c, int k, int R, const double* b, double* H, double* y, double* J,
                                       int* ok);

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
// of the group. Thread = pair p (grid.y covers the pairs); the group's moduli for a chunk of
// rows are staged in shared memory and read as broadcasts.
constexpr int ASM_ROWS = 32;
__global__ void __launch_bounds__(256) assemble_multi_partial_kernel(const double* __restrict__ Hel,
                                                                     const double* __restrict__ E, long long rows,
                                                                     int npair, int nr, long long rows_per_cta,
                                                                     double* partial) {
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
      Es[q][e] = (q < nr && e < nrow) ? __ldg(E + (size_t)q * rows + c0 + e) : 0.0;
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

// J_k of the group's candidates: written by the reduced solves into Jk (already in place).

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
  const int npair = k * (k + 1) / 2;
  const long long rows = Ne + 1;
  long long G = 2LL * c->num_sms;
  long long per = (rows + G - 1) / G;
  per = ((per + ASM_ROWS - 1) / ASM_ROWS) * ASM_ROWS;
  G = (rows + per - 1) / per;
  const long long tiles = residual_tiles(c);
  // scratch for one group of RC candidates
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_rho = take((size_t)RC * Ne * 8), o_E = take((size_t)RC * rows * 8),
               o_part = take((size_t)G * RC * npair * 8), o_H = take((size_t)RC * k * k * 8),
               o_y = take((size_t)RC * k * 8), o_U = take((size_t)RC * N * 8), o_dc = take((size_t)RC * Ne * 8),
               o_rp = take((size_t)RC * 2 * tiles * 8), o_ok = take((size_t)RC * 4);
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
  for (int r0 = 0; r0 < R; r0 += RC) {
    const int nr = std::min(RC, R - r0);
    const double* psi_g = psi + (size_t)r0 * ldp;
    // densities
    const double* rho_g = psi_g;
    long long ldr = ldp;
    if (filtered) {
      s = launch_filter_batch(c, psi_g, ldp, rho, Ne, nr, 0);
      if (s) return s;
      rho_g = rho;
      ldr = Ne;
    }
    moduli_batch_kernel<<<(int)std::min<long long>(8LL * c->num_sms, (rows * nr + 255) / 256), 256, 0, c->stream>>>(
        g, rho_g, ldr, E, nr);
    note_launch();
    // reduced matrices of the group
    assemble_multi_partial_kernel<<<dim3((unsigned)G, (npair + 255) / 256), std::min(256, ((npair + 31) / 32) * 32), 0,
                                    c->stream>>>(Hel, E, rows, npair, nr, per, part);
    note_launch();
    assemble_multi_final_kernel<<<(int)std::min<long long>(8LL * c->num_sms, ((long long)nr * npair + 7) / 8), 256, 0,
                                  c->stream>>>(part, (int)G, k, nr, H);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    double* y_g = yhat ? yhat + (size_t)r0 * k : ybuf;
    s = launch_reduced_solve_batch(c, k, nr, b, H, y_g, Jk + r0, ok);
    if (s) return s;
    // reduced states, residual norms, gradients
    const size_t smem = (size_t)RC * k * sizeof(double);
    if (smem > 48 * 1024)
      TOPO_CUDA_TRY(c, cudaFuncSetAttribute(basis_combine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    basis_combine_kernel<<<(int)std::min<long long>(4LL * c->num_sms, (N + 255) / 256), 256, smem, c->stream>>>(
        Phi, ld, k, y_g, nr, N, U, N);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    s = launch_residual64_batch(c, rho_g, ldr, U, N, f, resnorm + 2 * (size_t)r0, nr, rpart);
    if (s) return s;
    if (dpsi) {
      s = launch_grad_batch(c, rho_g, ldr, U, N, dc, Ne, nr);
      if (s) return s;
      s = filtered ? launch_filter_batch(c, dc, Ne, dpsi + (size_t)r0 * ldp, ldp, nr, 1)
                   : (cudaMemcpy2DAsync(dpsi + (size_t)r0 * ldp, (size_t)ldp * 8, dc, (size_t)Ne * 8, (size_t)Ne * 8,
                                        nr, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                          ? TOPO_OK
                          : fail(c, TOPO_ERR_CUDA, "topo_rom_eval_batch: copy of the gradients"));
      if (s) return s;
    }
  }
  return TOPO_OK;
}
