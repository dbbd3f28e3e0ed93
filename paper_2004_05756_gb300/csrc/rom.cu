// Galerkin reduced-order model on the GPU (Section 3.1, Eq. rom_soln and hatkbm; Section 3.3;
// the basis of Eq. rob-optim).
//
//   basis       classical Gram-Schmidt applied twice per snapshot (FP64), rank rule on the
//               orthogonalised norm;
//   projection  H = Phi^T (K(rho) Phi), b = Phi^T f: matrix-free applies of K to the k basis
//               columns, then a tall-skinny contraction over the N rows with fixed-order
//               partial sums (deterministic); FP64, or FP32 applies/contraction for the
//               refined precision forms;
//   reduced     one-CTA FP64 Cholesky of the k x k matrix and triangular solves; the FP32
//               forms refine yhat with FP64 reduced residuals b - Phi^T K(rho) Phi yhat;
//   residual    u_k = Phi yhat, r = f - K(rho) u_k, ||r||_2 and ||r||_2 / ||f||_2 in FP64.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace topo {

// dynamic shared memory of the k x k Cholesky kernels at the largest k (128): k^2 + k doubles
constexpr int kCholSmemMax = (128 * 128 + 128) * (int)sizeof(double);


// ---------------------------------------------------------------------------------------
// C = A^T B over N rows (A: N x k1, B: N x k2, column-major, leading dims lda, ldb), written as
// per-CTA partial sums partial[blockIdx.x][i * k2 + j] (FP64). A CTA owns a contiguous row
// range and one TILE x TILE output tile (blockIdx.y); its 256 threads each accumulate a
// (TILE/16) x (TILE/16) block. TILE follows k (16, 32 or 64) so small bases waste no FMAs.
// ---------------------------------------------------------------------------------------
template <typename T, int TILE>
__global__ void __launch_bounds__(256) atb_partial_kernel(const T* __restrict__ A, long long lda, int k1,
                                                          const T* __restrict__ B, long long ldb, int k2,
                                                          long long N, long long rows_per_cta, double* partial,
                                                          const int* gate) {
  constexpr int RB = 32;          // rows staged per pass
  constexpr int PT = TILE / 16;   // outputs per thread per direction
  __shared__ T As[RB][TILE + 1];
  __shared__ T Bs[RB][TILE + 1];
  if (gate && *gate == 0) return;
  const int tiles_j = (k2 + TILE - 1) / TILE;
  const int ti = blockIdx.y / tiles_j, tj = blockIdx.y % tiles_j;
  const int i0 = ti * TILE, j0 = tj * TILE;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[PT][PT];
#pragma unroll
  for (int u = 0; u < PT; ++u)
#pragma unroll
    for (int v = 0; v < PT; ++v) acc[u][v] = (T)0;
  const long long r_begin = blockIdx.x * rows_per_cta;
  const long long r_end = min(N, r_begin + rows_per_cta);
  for (long long r0 = r_begin; r0 < r_end; r0 += RB) {
    for (int idx = threadIdx.x; idx < RB * TILE; idx += 256) {
      const int col = idx / RB, row = idx % RB;
      const long long r = r0 + row;
      const bool rin = r < r_end;
      As[row][col] = (rin && i0 + col < k1) ? A[(long long)(i0 + col) * lda + r] : (T)0;
      Bs[row][col] = (rin && j0 + col < k2) ? B[(long long)(j0 + col) * ldb + r] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int row = 0; row < RB; ++row) {
      T av[PT], bv[PT];
#pragma unroll
      for (int u = 0; u < PT; ++u) av[u] = As[row][ty * PT + u];
#pragma unroll
      for (int v = 0; v < PT; ++v) bv[v] = Bs[row][tx * PT + v];
#pragma unroll
      for (int u = 0; u < PT; ++u)
#pragma unroll
        for (int v = 0; v < PT; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* out = partial + (size_t)blockIdx.x * k1 * k2;
#pragma unroll
  for (int u = 0; u < PT; ++u)
#pragma unroll
    for (int v = 0; v < PT; ++v) {
      const int i = i0 + ty * PT + u, j = j0 + tx * PT + v;
      if (i < k1 && j < k2) out[i * k2 + j] = (double)acc[u][v];
    }
}

// C[e] = sum over g < G of partial[g * KK + e] (KK = k1 k2) in a fixed order: a CTA takes 32
// consecutive entries (lane = entry); warp w sums the partials g in [G w / 8, G (w + 1) / 8) in
// order, then the 8 warp sums are added in warp order. Spreading the G-long sums over many SMs
// keeps this FP64 reduction short.
__global__ void __launch_bounds__(256) atb_final_kernel(const double* __restrict__ partial, int G, int KK, double* C,
                                                        const int* gate) {
  __shared__ double red[8][33];
  if (gate && *gate == 0) return;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int e = blockIdx.x * 32 + l;
  const int g0 = (int)((long long)G * w / 8), g1 = (int)((long long)G * (w + 1) / 8);
  double s = 0.0;
  if (e < KK)
    for (int g = g0; g < g1; ++g) s += __ldcg(partial + (size_t)g * KK + e);
  red[w][l] = s;
  __syncthreads();
  if (w == 0 && e < KK) {
    double t = red[0][l];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][l];
    C[e] = t;
  }
}

// C = (C + C^T) / 2 for a k x k row-major matrix (one thread per pair i < j).
__global__ void symmetrize_kernel(double* C, int k, const int* gate) {
  if (gate && *gate == 0) return;
  const long long npair = (long long)k * (k - 1) / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npair; t += (long long)gridDim.x * blockDim.x) {
    // pair t -> (i, j), i < j, row-major over the strict upper triangle
    int i = 0;
    long long rem = t;
    while (rem >= k - 1 - i) {
      rem -= k - 1 - i;
      ++i;
    }
    const int j = i + 1 + (int)rem;
    const double v = 0.5 * (C[i * k + j] + C[j * k + i]);
    C[i * k + j] = v;
    C[j * k + i] = v;
  }
}

// c = A^T v (A: N x k, v: N), per-CTA partials partial[blockIdx.x * k + j]; warp w handles
// columns w, w+8, ...; lanes stride the CTA's row range.
__global__ void atv_partial_kernel(const double* __restrict__ A, long long lda, int k, const double* __restrict__ v,
                                   long long N, long long rows_per_cta, double* partial, const int* gate) {
  if (gate && *gate == 0) return;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long r_begin = blockIdx.x * rows_per_cta;
  const long long r_end = min(N, r_begin + rows_per_cta);
  for (int j = w; j < k; j += nw) {
    const double* a = A + (long long)j * lda;
    double acc = 0.0;
    for (long long r = r_begin + l; r < r_end; r += 32) acc = fma(a[r], v[r], acc);
    acc = warp_sum(acc);
    if (l == 0) partial[(size_t)blockIdx.x * k + j] = acc;
  }
}

// out[j] = (subtract ? base[j] - s : s), s = sum_g partial[g * k + j]: one warp per j, lanes
// summing g = lane, lane + 32, ... in order, then a shuffle tree (an order fixed by G alone).
__global__ void atv_final_kernel(const double* partial, int G, int k, double* out, const double* base,
                                 const int* gate) {
  if (gate && *gate == 0) return;
  const int l = threadIdx.x & 31, nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < k; j += nw) {
    double s0 = 0.0, s1 = 0.0;
    int g = l;
    for (; g + 32 < G; g += 64) {
      s0 += __ldcg(partial + (size_t)g * k + j);
      s1 += __ldcg(partial + (size_t)(g + 32) * k + j);
    }
    if (g < G) s0 += __ldcg(partial + (size_t)g * k + j);
    const double s = warp_sum(s0 + s1);
    if (l == 0) out[j] = base ? base[j] - s : s;
  }
}

// y = A c (mode 0), or y -= A c (mode 1); A: N x k, c FP64[k] (device).
__global__ void gemv_kernel(const double* __restrict__ A, long long lda, int k, const double* __restrict__ cvec,
                            double* y, long long N, int mode, const int* gate) {
  extern __shared__ double sc[];
  if (gate && *gate == 0) return;
  for (int j = threadIdx.x; j < k; j += blockDim.x) sc[j] = cvec[j];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(A[(long long)j * lda + r], sc[j], acc);
    y[r] = mode ? y[r] - acc : acc;
  }
}

// ||x||^2 partials (per CTA) and the final sqrt into *out.
__global__ void nrm2_partial_kernel(const double* x, long long N, double* partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
    acc = fma(x[r], x[r], acc);
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}
__global__ void nrm2_final_kernel(const double* partial, int G, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) acc += partial[i];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) *out = sqrt(t);
}

__global__ void scale_kernel(double* x, long long N, const double* nrm) {
  const double s = 1.0 / *nrm;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
    x[r] *= s;
}

__global__ void to_float_kernel(const double* __restrict__ A, long long lda, int k, float* B, long long ldb,
                                long long N) {
  const long long total = N * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long j = t / N, r = t % N;
    B[j * ldb + r] = (float)A[j * lda + r];
  }
}

// ---------------------------------------------------------------------------------------
// One-CTA FP64 Cholesky H = L L^T (row-major k x k in global memory, overwritten with L in
// the lower triangle), then y = H^{-1} b and J = b^T y. A pivot <= 0 (or NaN) sets
// TOPO_ERR_NOT_SPD and writes NaN to y and J.
// ---------------------------------------------------------------------------------------
__global__ void cholesky_kernel(double* H, int k, int* status, int* ok_flag, const int* gate) {
  extern __shared__ double A[];  // k * k
  __shared__ int bad;
  if (gate && *gate == 0) return;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) A[e] = H[e];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[j * k + j];
      if (!(d > 0.0)) {
        bad = 1;
      } else {
        A[j * k + j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double ljj = A[j * k + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) A[i * k + j] /= ljj;
    __syncthreads();
    const int n = k - j - 1;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int i = j + 1 + t / n, l = j + 1 + t % n;
      if (l <= i) A[i * k + l] -= A[i * k + j] * A[l * k + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, l = e % k;
    H[e] = (l <= i) ? A[e] : 0.0;
  }
  if (threadIdx.x == 0) {
    *ok_flag = !bad;
    if (bad && status) atomicCAS(status, 0, (int)TOPO_ERR_NOT_SPD);
  }
}

// The whole k x k reduced solve in one warp for k <= KMAX <= 32: FP64 Cholesky H = L L^T with
// lane i holding row i in registers, then y = H^{-1} b by forward and backward substitution
// and J = b^T y. L is written back into H (lower triangle, zeros above) as cholesky_kernel
// does; the substitutions multiply by the reciprocal pivots computed during the factorisation,
// so the solve takes k square roots and k divisions (each a long FP64 dependency chain here).
// A pivot <= 0 (or NaN) sets TOPO_ERR_NOT_SPD and writes NaN to y and J.
template <int KMAX>
__device__ __forceinline__ void chol_small_body(double* H, int k, const double* b, double* y, double* J, int* status,
                                                int* ok_flag) {
  __shared__ double Ls[KMAX][KMAX + 1];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  double a[KMAX];
#pragma unroll
  for (int c = 0; c < KMAX; ++c) a[c] = (lane < k && c < k) ? H[lane * k + c] : 0.0;
  double myinv = 0.0;  // 1 / L[lane][lane]
  bool bad = false;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k && !bad) {
      const double d = __shfl_sync(FULL, a[j], j);
      if (!(d > 0.0)) {
        bad = true;  // the same value in every lane: uniform
      } else {
        const double ljj = sqrt(d), inv = 1.0 / ljj;
        if (lane == j) {
          a[j] = ljj;
          myinv = inv;
        } else if (lane > j) {
          a[j] *= inv;
        }
#pragma unroll
        for (int c = j + 1; c < KMAX; ++c) {
          const double lcj = __shfl_sync(FULL, a[j], c);  // L[c][j], held by lane c
          if (c < k && lane >= c) a[c] = fma(-a[j], lcj, a[c]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < KMAX; ++c)
    if (lane < k && c < k) {
      const double v = c <= lane ? a[c] : 0.0;
      H[lane * k + c] = v;
      Ls[lane][c] = v;
    }
  __syncwarp();
  if (bad) {
    if (lane < k) y[lane] = __longlong_as_double(0x7ff8000000000000LL);
    if (lane == 0) {
      *J = __longlong_as_double(0x7ff8000000000000LL);
      *ok_flag = 0;
      if (status) atomicCAS(status, 0, (int)TOPO_ERR_NOT_SPD);
    }
    return;
  }
  // L z = b (column-oriented: lane c finishes z_c, the lanes below subtract its share)
  const double bl = lane < k ? b[lane] : 0.0;
  double r = bl, z = 0.0;
#pragma unroll
  for (int c = 0; c < KMAX; ++c)
    if (c < k) {
      const double zc = __shfl_sync(FULL, r * myinv, c);
      if (lane == c) z = zc;
      if (lane > c) r = fma(-a[c], zc, r);
    }
  // L^T y = z (from the last row up; L[c][lane] from shared memory)
  double r2 = z, yv = 0.0;
#pragma unroll
  for (int c = KMAX - 1; c >= 0; --c)
    if (c < k) {
      const double yc = __shfl_sync(FULL, r2 * myinv, c);
      if (lane == c) yv = yc;
      if (lane < c) r2 = fma(-Ls[c][lane], yc, r2);
    }
  if (lane < k) y[lane] = yv;
  double t = lane < k ? bl * yv : 0.0;
  t = warp_sum(t);
  if (lane == 0) {
    *J = t;
    *ok_flag = 1;
  }
}

template <int KMAX>
__global__ void __launch_bounds__(32) chol_small_kernel(double* H, int k, const double* b, double* y, double* J,
                                                        int* status, int* ok_flag) {
  chol_small_body<KMAX>(H, k, b, y, J, status, ok_flag);
}

// R reduced solves, one warp each: H + r k^2, y + r k, J + r, ok + r (one right-hand side b).
template <int KMAX>
__global__ void __launch_bounds__(32) chol_small_batch_kernel(double* H, int k, const double* b, double* y, double* J,
                                                              int* status, int* ok) {
  const int r = blockIdx.x;
  chol_small_body<KMAX>(H + (size_t)r * k * k, k, b, y + (size_t)r * k, J + r, status, ok + r);
}

// Reduced solves of different problems (each its own H, b, k <= 32), one warp each.
__global__ void __launch_bounds__(32) chol_small_multi_kernel(const RedSolve* __restrict__ tab) {
  const RedSolve t = tab[blockIdx.x];
  chol_small_body<32>(t.H, t.k, t.b, t.y, t.J, t.status, t.ok);
}

cudaError_t launch_chol_small_multi(const RedSolve* tab, int n, cudaStream_t stream) {
  chol_small_multi_kernel<<<n, 32, 0, stream>>>(tab);
  note_launch();
  return cudaGetLastError();
}

// Solve L L^T x = rhs (L lower, row-major). mode 0: y = x; mode 1: y += x. Skipped (y left
// unchanged) when *skip is non-zero; NaN output when the factorisation failed.
__global__ void chol_solve_kernel(const double* L, int k, const double* rhs, double* y, int mode, const int* ok_flag,
                                  const int* gate) {
  extern __shared__ double sm[];
  double* Ls = sm;          // k*k
  double* z = sm + k * k;   // k
  if (gate && *gate == 0) return;
  if (!*ok_flag) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = nan("");
    return;
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ls[e] = L[e];
  for (int i = threadIdx.x; i < k; i += blockDim.x) z[i] = rhs[i];
  __syncthreads();
  // forward: L z = rhs (column sweep)
  for (int i = 0; i < k; ++i) {
    if (threadIdx.x == 0) z[i] /= Ls[i * k + i];
    __syncthreads();
    const double zi = z[i];
    for (int t = i + 1 + threadIdx.x; t < k; t += blockDim.x) z[t] -= Ls[t * k + i] * zi;
    __syncthreads();
  }
  // backward: L^T x = z
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) z[i] /= Ls[i * k + i];
    __syncthreads();
    const double xi = z[i];
    for (int t = threadIdx.x; t < i; t += blockDim.x) z[t] -= Ls[i * k + t] * xi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = mode ? y[i] + z[i] : z[i];
}

// J = b^T y (fixed order, one CTA).
__global__ void dot_small_kernel(const double* b, const double* y, int k, double* J) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) acc = fma(b[i], y[i], acc);
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) *J = t;
}

// Convergence test of the reduced refinement (runs while flags[2] "active" is set):
// ||g|| <= tol ||b|| sets flags[1] "converged" and clears "active".
__global__ void refine_flag_kernel(const double* g, const double* b, int k, double tol, int* flags) {
  __shared__ double red[32];
  if (flags[2] == 0) return;
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    a = fma(g[i], g[i], a);
    c = fma(b[i], b[i], c);
  }
  const double ta = block_sum(a, red);
  const double tc = block_sum(c, red);
  if (threadIdx.x == 0 && sqrt(ta) <= tol * sqrt(tc)) {
    flags[1] = 1;
    flags[2] = 0;
  }
}

// flags[2] = active = Cholesky of the FP32 matrix succeeded (flags[0]).
__global__ void refine_start_kernel(int* flags) { flags[2] = flags[0]; }
// flags[3] = fallback to FP64: the FP32 matrix was not SPD, or refinement did not converge.
__global__ void refine_end_kernel(int* flags, int require_conv) {
  flags[3] = (!flags[0] || (require_conv && !flags[1])) ? 1 : 0;
}

// ---------------------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------------------
struct RowSplit {
  int G;
  long long rows;
};
static RowSplit row_split(topo_ctx* c, long long N, int per_sm) {
  long long G = (long long)per_sm * c->num_sms;
  long long rows = (N + G - 1) / G;
  rows = ((rows + 31) / 32) * 32;
  if (rows < 32) rows = 32;
  G = (N + rows - 1) / rows;
  if (G < 1) G = 1;
  return {(int)G, rows};
}

// Fixed-order sum of the G partial k1 x k2 tiles into C; sym (k1 == k2): C = (C + C^T) / 2.
static topo_status launch_atb_final(topo_ctx* c, const double* partial, int G, int k1, int k2, double* C, int sym,
                                    const int* gate) {
  const int KK = k1 * k2;
  atb_final_kernel<<<(KK + 31) / 32, 256, 0, c->stream>>>(partial, G, KK, C, gate);
  note_launch();
  if (sym && k1 == k2 && k1 > 1) {
    const long long npair = (long long)k1 * (k1 - 1) / 2;
    symmetrize_kernel<<<(int)std::min<long long>((npair + 255) / 256, 64), 256, 0, c->stream>>>(C, k1, gate);
    note_launch();
  }
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

template <typename T>
static topo_status launch_atb(topo_ctx* c, const T* A, long long lda, int k1, const T* B, long long ldb, int k2,
                              long long N, double* partial_buf, size_t partial_cap, double* C, int sym,
                              const int* gate = nullptr) {
  RowSplit rs = row_split(c, N, 2);
  size_t need = (size_t)rs.G * k1 * k2;
  if (need > partial_cap) return fail(c, TOPO_ERR_INVALID, "internal: atb partial buffer too small");
  const int kmax = std::max(k1, k2);
  if (kmax <= 16) {
    atb_partial_kernel<T, 16><<<dim3(rs.G, 1), 256, 0, c->stream>>>(A, lda, k1, B, ldb, k2, N, rs.rows, partial_buf, gate);
  } else if (kmax <= 32) {
    atb_partial_kernel<T, 32><<<dim3(rs.G, 1), 256, 0, c->stream>>>(A, lda, k1, B, ldb, k2, N, rs.rows, partial_buf, gate);
  } else {
    const int tiles = ((k1 + 63) / 64) * ((k2 + 63) / 64);
    atb_partial_kernel<T, 64><<<dim3(rs.G, tiles), 256, 0, c->stream>>>(A, lda, k1, B, ldb, k2, N, rs.rows, partial_buf,
                                                                        gate);
  }
  note_launch();
  return launch_atb_final(c, partial_buf, rs.G, k1, k2, C, sym, gate);
}

static topo_status launch_atv(topo_ctx* c, const double* A, long long lda, int k, const double* v, long long N,
                              double* partial_buf, size_t partial_cap, double* out, const double* base,
                              const int* gate = nullptr) {
  RowSplit rs = row_split(c, N, 4);
  if ((size_t)rs.G * k > partial_cap) return fail(c, TOPO_ERR_INVALID, "internal: atv partial buffer too small");
  atv_partial_kernel<<<rs.G, 256, 0, c->stream>>>(A, lda, k, v, N, rs.rows, partial_buf, gate);
  note_launch();
  atv_final_kernel<<<(k + 7) / 8, 256, 0, c->stream>>>(partial_buf, rs.G, k, out, base, gate);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

static int stream_blocks(topo_ctx* c, long long N) {
  long long b = (N + 255) / 256;
  long long cap = 8LL * c->num_sms;
  return (int)std::max(1LL, std::min(b, cap));
}

static size_t partial_capacity(topo_ctx* c, long long N, int k) {
  RowSplit a = row_split(c, N, 2), b = row_split(c, N, 4);
  return std::max((size_t)a.G * k * k, (size_t)b.G * k) + 64;
}

// Projection H = Phi^T K Phi (and optionally b = Phi^T f) into H (k x k, row-major).
static topo_status project(topo_ctx* c, const double* rho, const double* Phi, int k, long long ld, topo_prec prec,
                           double* H, double* b, const double* f, char* scratch, const int* gate = nullptr) {
  const long long N = c->g.ndof;
  size_t pcap = partial_capacity(c, N, k);
  double* partial = (double*)scratch;
  char* p = scratch + ((pcap * sizeof(double) + 255) & ~(size_t)255);
  if (prec == TOPO_FP64) {
    double* W = (double*)p;
    topo_status s = launch_apply(c, rho, Phi, W, k, (int)ld, TOPO_FP64, gate);
    if (s) return s;
    // W has leading dimension ld (same as Phi)
    s = launch_atb<double>(c, Phi, ld, k, W, ld, k, N, partial, pcap, H, 1, gate);
    if (s) return s;
  } else {
    // FP32 copies with a leading dimension padded to 32 rows (16-byte aligned TMA strides)
    const long long ld32 = (N + 31) & ~31LL;
    float* P32 = (float*)p;
    float* W32 = P32 + (size_t)ld32 * k;
    to_float_kernel<<<stream_blocks(c, N * k), 256, 0, c->stream>>>(Phi, ld, k, P32, ld32, N);
    note_launch();
    topo_status s = launch_apply(c, rho, P32, W32, k, (int)ld32, prec);
    if (s) return s;
    if (c->rom_tensor) {
      int G = 0;
      s = launch_atb_tc_partial(c, P32, ld32, k, W32, ld32, k, N, partial, pcap, &G);
      if (s) return s;
      s = launch_atb_final(c, partial, G, k, k, H, 1, nullptr);
      if (s) return s;
    } else {
      s = launch_atb<float>(c, P32, ld32, k, W32, ld32, k, N, partial, pcap, H, 1);
      if (s) return s;
    }
  }
  if (b) return launch_atv(c, Phi, ld, k, f, N, partial, pcap, b, nullptr);
  return TOPO_OK;
}

static size_t project_scratch(topo_ctx* c, int k, long long ld, topo_prec prec) {
  const long long N = c->g.ndof;
  size_t pcap = partial_capacity(c, N, k);
  size_t s = ((pcap * sizeof(double) + 255) & ~(size_t)255);
  if (prec == TOPO_FP64)
    s += (size_t)ld * k * sizeof(double);
  else
    s += 2 * (size_t)((N + 31) & ~31LL) * k * sizeof(float);
  return s + 256;
}

// FP64 Cholesky of H_work (overwritten with L), yhat = H^{-1} b, Jk = b^T yhat. A non-positive
// pivot sets TOPO_ERR_NOT_SPD in the device status and writes NaN.
topo_status launch_reduced_solve(topo_ctx* c, int k, const double* b, double* H_work, double* yhat, double* Jk,
                                 int* ok) {
  if (k <= 16) {
    chol_small_kernel<16><<<1, 32, 0, c->stream>>>(H_work, k, b, yhat, Jk, &c->d_sync->status, ok);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    return TOPO_OK;
  }
  if (k <= 32) {
    chol_small_kernel<32><<<1, 32, 0, c->stream>>>(H_work, k, b, yhat, Jk, &c->d_sync->status, ok);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    return TOPO_OK;
  }
  const size_t sm_chol = (size_t)k * k * sizeof(double);
  const size_t sm_solve = sm_chol + k * sizeof(double);
  if (sm_solve > 48 * 1024) {  // one value for every k, so concurrent host threads never lower it
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemMax));
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemMax));
  }
  cholesky_kernel<<<1, 256, sm_chol, c->stream>>>(H_work, k, &c->d_sync->status, ok, nullptr);
  note_launch();
  chol_solve_kernel<<<1, 128, sm_solve, c->stream>>>(H_work, k, b, yhat, 0, ok, nullptr);
  note_launch();
  dot_small_kernel<<<1, 128, 0, c->stream>>>(b, yhat, k, Jk);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

// R reduced solves with one right-hand side b: H, y, J and ok hold R consecutive instances.
topo_status launch_reduced_solve_batch(topo_ctx* c, int k, int R, const double* b, double* H, double* y, double* J,
                                       int* ok) {
  if (k <= 16) {
    chol_small_batch_kernel<16><<<R, 32, 0, c->stream>>>(H, k, b, y, J, &c->d_sync->status, ok);
    note_launch();
  } else if (k <= 32) {
    chol_small_batch_kernel<32><<<R, 32, 0, c->stream>>>(H, k, b, y, J, &c->d_sync->status, ok);
    note_launch();
  } else {
    for (int r = 0; r < R; ++r) {
      topo_status s = launch_reduced_solve(c, k, b, H + (size_t)r * k * k, y + (size_t)r * k, J + r, ok + r);
      if (s) return s;
    }
  }
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

topo_status reduced_solve(topo_ctx* c, int k, const double* b, double* H_work, double* yhat, double* Jk) {
  topo_status s = ensure_red(c, 256);
  if (s) return s;
  return launch_reduced_solve(c, k, b, H_work, yhat, Jk, (int*)c->d_red);
}


// ---------------------------------------------------------------------------------------
// POD of a snapshot block (Section 4.2, Eq. rob-optim): the leading left singular vectors of U
// from the eigen-decomposition of its Gram matrix U^T U (FP64) by the cyclic Jacobi method on one
// CTA: each step rotates M/2 disjoint index pairs of the round-robin schedule at once (columns,
// then rows, then the accumulated eigenvectors), sweeps until the off-diagonal mass is below
// 1e-30 of the diagonal's (at most 40 sweeps).
// ---------------------------------------------------------------------------------------
constexpr int POD_MAX = 64;

// Gram (m x m, row-major) with column `skip` left out -> coefficients coef (m x n, row-major:
// Pod_i = sum_j coef[j][i] U_j) and the singular values sigma[0 .. m' - 1], m' = m - (skip >= 0).
__global__ void __launch_bounds__(256) pod_jacobi_kernel(const double* __restrict__ gram, int m, int skip, int n,
                                                        double* coef, double* sigma) {
  extern __shared__ double sm[];
  const int mp = m - (skip >= 0 ? 1 : 0);
  const int M = mp + (mp & 1);  // even (a dummy index when mp is odd)
  const int ldm = POD_MAX + 1;
  double* G = sm;               // M x ldm
  double* V = G + POD_MAX * ldm;  // M x ldm
  __shared__ int idx[POD_MAX];    // local index -> column of U
  __shared__ int pp[POD_MAX / 2], qq[POD_MAX / 2];
  __shared__ double cs[POD_MAX / 2], sn[POD_MAX / 2];
  __shared__ int order[POD_MAX];
  __shared__ int done;
  __shared__ double red[2][8];
  if (threadIdx.x == 0) {
    int t = 0;
    for (int j = 0; j < m; ++j)
      if (j != skip) idx[t++] = j;
    done = 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
    const int r = t / M, c = t % M;
    G[r * ldm + c] = (r < mp && c < mp) ? gram[idx[r] * m + idx[c]] : 0.0;
    V[r * ldm + c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40 && M > 1; ++sweep) {
    for (int round = 0; round < M - 1; ++round) {
      if (threadIdx.x < M / 2) {
        const int i = threadIdx.x;
        auto pos = [&](int k) { return k == 0 ? 0 : ((k - 1 + round) % (M - 1)) + 1; };
        int p = pos(i), q = pos(M - 1 - i);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        pp[i] = p;
        qq[i] = q;
        const double apq = G[p * ldm + q], app = G[p * ldm + p], aqq = G[q * ldm + q];
        double c = 1.0, s = 0.0;
        if (q < mp && apq != 0.0) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // columns of G and V: (x_p, x_q) <- (c x_p - s x_q, s x_p + c x_q)
      for (int t = threadIdx.x; t < M * (M / 2); t += blockDim.x) {
        const int r = t / (M / 2), k = t % (M / 2);
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double gp = G[r * ldm + p], gq = G[r * ldm + q];
        G[r * ldm + p] = c * gp - s * gq;
        G[r * ldm + q] = s * gp + c * gq;
        const double vp = V[r * ldm + p], vq = V[r * ldm + q];
        V[r * ldm + p] = c * vp - s * vq;
        V[r * ldm + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows of G
      for (int t = threadIdx.x; t < M * (M / 2); t += blockDim.x) {
        const int col = t / (M / 2), k = t % (M / 2);
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double gp = G[p * ldm + col], gq = G[q * ldm + col];
        G[p * ldm + col] = c * gp - s * gq;
        G[q * ldm + col] = s * gp + c * gq;
      }
      __syncthreads();
    }
    // off-diagonal and diagonal mass (fixed order)
    double off = 0.0, dia = 0.0;
    for (int t = threadIdx.x; t < mp * mp; t += blockDim.x) {
      const int r = t / mp, c = t % mp;
      const double g = G[r * ldm + c];
      if (r == c)
        dia += g * g;
      else
        off += g * g;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = off;
      red[1][threadIdx.x >> 5] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double o = 0.0, d = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        o += red[0][w];
        d += red[1][w];
      }
      done = !(o > 1e-30 * d);
    }
    __syncthreads();
    if (done) break;
  }
  // eigenvalues in descending order (ties by index); small ones are rounding noise of the Gram
  // matrix (absolute error ~ eps lambda_max): their vectors are left out
  if (threadIdx.x == 0) {
    for (int i = 0; i < mp; ++i) order[i] = i;
    for (int i = 1; i < mp; ++i) {
      const int v = order[i];
      const double lv = G[v * ldm + v];
      int j = i - 1;
      while (j >= 0 && G[order[j] * ldm + order[j]] < lv) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
  }
  __syncthreads();
  const double lmax = mp > 0 ? fmax(G[order[0] * ldm + order[0]], 0.0) : 0.0;
  for (int i = threadIdx.x; i < mp; i += blockDim.x) sigma[i] = sqrt(fmax(G[order[i] * ldm + order[i]], 0.0));
  for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
    const int j = t / n, i = t % n;
    double v = 0.0;
    if (i < mp && j != skip) {
      const int jl = j - (skip >= 0 && j > skip ? 1 : 0);
      const int e = order[i];
      const double lam = G[e * ldm + e];
      if (lam > 64.0 * 2.220446049250313e-16 * lmax) v = V[jl * ldm + e] / sqrt(lam);
    }
    coef[t] = v;
  }
}

// Pod_i = sum_j coef[j][i] U_j (i < n), then Pod_n = append (when given).
__global__ void __launch_bounds__(256) pod_combine_kernel(const double* __restrict__ U, long long ld, int m,
                                                         const double* __restrict__ coef, int n,
                                                         const double* __restrict__ append, double* Pod,
                                                         long long ldp, long long N) {
  extern __shared__ double cf[];  // m x n
  for (int t = threadIdx.x; t < m * n; t += blockDim.x) cf[t] = coef[t];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    double u[POD_MAX];
#pragma unroll 8
    for (int j = 0; j < m; ++j) u[j] = U[(long long)j * ld + r];
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc = fma(cf[j * n + i], u[j], acc);
      Pod[(long long)i * ldp + r] = acc;
    }
    if (append) Pod[(long long)n * ldp + r] = append[r];
  }
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_rom_build(topo_ctx* c, const double* rho, const double* Usnap, int m, int ld, double* Phi,
                                      int* k_out, double* H, double* b, const double* f) {
  if (!c) return TOPO_ERR_INVALID;
  const long long N = c->g.ndof;
  if (!k_out) return fail(c, TOPO_ERR_INVALID, "topo_rom_build: k_out is NULL");
  *k_out = 0;
  if (m < 1 || m > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_build: 1 <= m <= 128");
  if ((long long)ld < N) return fail(c, TOPO_ERR_INVALID, "topo_rom_build: ld < N");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(Usnap) || !dev_ptr_ok(Phi) || (H && !dev_ptr_ok(H)) || !dev_ptr_ok(b) ||
      !dev_ptr_ok(f))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_build: null or misaligned pointer");
  // CGS2 with the rank rule (drop a column whose orthogonalised norm is below 1e-10 of the
  // largest snapshot norm), b = Phi^T f and k in one cooperative launch, then one read of k
  const size_t ncg = cgs2_scratch_doubles(c);
  size_t need = std::max(project_scratch(c, m, ld, TOPO_FP64), (ncg + 64) * sizeof(double));
  topo_status s = ensure_scratch(c, need);
  if (s) return s;
  char* scratch = (char*)c->d_scratch;
  int* k_dev = (int*)((double*)scratch + ncg);
  s = launch_cgs2(c, Usnap, m, ld, Phi, f, b, 1e-10, (double*)scratch, k_dev);
  if (s) return s;
  int k = 0;
  TOPO_CUDA_TRY(c, cudaMemcpyAsync(&k, k_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  TOPO_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  TOPO_CUDA_TRY(c, cudaGetLastError());
  *k_out = k;
  if (k == 0 || !H) return TOPO_OK;  // b = Phi^T f is in place
  return project(c, rho, Phi, k, ld, TOPO_FP64, H, nullptr, nullptr, scratch);  // H only: b stays the launch's
}

extern "C" topo_status topo_rom_solve(topo_ctx* c, const double* rho, const double* Phi, int k, int ld,
                                      const double* b, double* H_work, double* yhat, double* Jk, topo_prec prec) {
  if (!c) return TOPO_ERR_INVALID;
  const long long N = c->g.ndof;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_solve: 1 <= k <= 128");
  if ((long long)ld < N) return fail(c, TOPO_ERR_INVALID, "topo_rom_solve: ld < N");
  if (prec != TOPO_FP64 && prec != TOPO_FP32_REFINED && prec != TOPO_FP32_BF16KE_REFINED)
    return fail(c, TOPO_ERR_INVALID, "topo_rom_solve: unknown precision");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(Phi) || !dev_ptr_ok(b) || !dev_ptr_ok(H_work) || !dev_ptr_ok(yhat) ||
      !dev_ptr_ok(Jk))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_solve: null or misaligned pointer");
  size_t pcap = partial_capacity(c, N, k);
  // the mixed forms may fall back to the FP64 projection, which needs its own (larger) W
  const size_t proj = std::max(project_scratch(c, k, ld, prec), project_scratch(c, k, ld, TOPO_FP64));
  const size_t extra = (2 * (size_t)N + 4 * 128 + 64) * sizeof(double);
  size_t need = proj + 256 + extra + 1024;
  topo_status s = ensure_scratch(c, need);
  if (s) return s;
  char* scratch = (char*)c->d_scratch;
  s = project(c, rho, Phi, k, ld, prec, H_work, nullptr, nullptr, scratch);
  if (s) return s;
  // flags live after the projection scratch
  char* tail = scratch + proj;
  int* flags = (int*)tail;  // [0] ok32 [1] converged [2] active [3] fallback [4] ok64
  double* tailD = (double*)(tail + 256);
  TOPO_CUDA_TRY(c, cudaMemsetAsync(flags, 0, 8 * sizeof(int), c->stream));
  const size_t sm_chol = (size_t)k * k * sizeof(double);
  const size_t sm_solve = sm_chol + k * sizeof(double);
  if (sm_solve > 48 * 1024) {  // one value for every k, so concurrent host threads never lower it
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemMax));
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemMax));
  }
  if (prec == TOPO_FP64) {
    cholesky_kernel<<<1, 256, sm_chol, c->stream>>>(H_work, k, &c->d_sync->status, flags + 4, nullptr);
    note_launch();
    chol_solve_kernel<<<1, 128, sm_solve, c->stream>>>(H_work, k, b, yhat, 0, flags + 4, nullptr);
    note_launch();
  } else {
    // FP32 reduced matrix: factor it (a failure is not an error here), solve, then refine
    // yhat with FP64 reduced residuals g = b - Phi^T K(rho) (Phi yhat).
    cholesky_kernel<<<1, 256, sm_chol, c->stream>>>(H_work, k, nullptr, flags + 0, nullptr);
    note_launch();
    chol_solve_kernel<<<1, 128, sm_solve, c->stream>>>(H_work, k, b, yhat, 0, flags + 0, flags + 0);
    note_launch();
    refine_start_kernel<<<1, 1, 0, c->stream>>>(flags);
    note_launch();
    double* u = tailD;
    double* w = u + N;
    double* g = w + N;  // [k]
    double* partial = (double*)scratch;  // projection partials are dead now
    const int nb = stream_blocks(c, N);
    const int* active = flags + 2;
    for (int it = 0; it < c->rom_refine; ++it) {
      gemv_kernel<<<nb, 256, k * sizeof(double), c->stream>>>(Phi, ld, k, yhat, u, N, 0, active);
      note_launch();
      s = launch_apply(c, rho, u, w, 1, (int)N, TOPO_FP64, active);
      if (s) return s;
      s = launch_atv(c, Phi, ld, k, w, N, partial, pcap, g, b, active);
      if (s) return s;
      refine_flag_kernel<<<1, 128, 0, c->stream>>>(g, b, k, 1e-11, flags);
      note_launch();
      chol_solve_kernel<<<1, 128, sm_solve, c->stream>>>(H_work, k, g, yhat, 1, flags + 0, active);
      note_launch();
    }
    refine_end_kernel<<<1, 1, 0, c->stream>>>(flags, c->rom_refine > 0 ? 1 : 0);
    note_launch();
    // FP64 fallback, executed on the device only when flags[3] is set
    const int* fb = flags + 3;
    s = project(c, rho, Phi, k, ld, TOPO_FP64, H_work, nullptr, nullptr, scratch, fb);
    if (s) return s;
    cholesky_kernel<<<1, 256, sm_chol, c->stream>>>(H_work, k, &c->d_sync->status, flags + 4, fb);
    note_launch();
    chol_solve_kernel<<<1, 128, sm_solve, c->stream>>>(H_work, k, b, yhat, 0, flags + 4, fb);
    note_launch();
  }
  dot_small_kernel<<<1, 128, 0, c->stream>>>(b, yhat, k, Jk);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_rom_error(topo_ctx* c, const double* rho, const double* Phi, int k, int ld,
                                      const double* yhat, const double* f, double* resnorm, double* uk_opt) {
  if (!c) return TOPO_ERR_INVALID;
  const long long N = c->g.ndof;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_error: 1 <= k <= 128");
  if ((long long)ld < N) return fail(c, TOPO_ERR_INVALID, "topo_rom_error: ld < N");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(Phi) || !dev_ptr_ok(yhat) || !dev_ptr_ok(f) || !dev_ptr_ok(resnorm) ||
      (uk_opt && !dev_ptr_ok(uk_opt)))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_error: null or misaligned pointer");
  double* uk = uk_opt;
  if (!uk) {
    topo_status s = ensure_scratch(c, (size_t)N * sizeof(double) + 256);
    if (s) return s;
    uk = (double*)c->d_scratch;
  }
  gemv_kernel<<<stream_blocks(c, N), 256, k * sizeof(double), c->stream>>>(Phi, ld, k, yhat, uk, N, 0, nullptr);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return launch_residual64(c, rho, uk, f, nullptr, resnorm);
}

extern "C" topo_status topo_rom_pod(topo_ctx* c, const double* U, int m, int ld, int skip, int n,
                                    const double* append, double* Pod, int ldp, double* sigma) {
  if (!c) return TOPO_ERR_INVALID;
  const long long N = c->g.ndof;
  const int mp = m - (skip >= 0 ? 1 : 0);
  if (m < 1 || m > POD_MAX) return fail(c, TOPO_ERR_INVALID, "topo_rom_pod: 1 <= m <= 64");
  if (skip < -1 || skip >= m) return fail(c, TOPO_ERR_INVALID, "topo_rom_pod: skip must be -1 or a column index");
  if (n < 0 || n > mp) return fail(c, TOPO_ERR_INVALID, "topo_rom_pod: 0 <= n <= the columns kept");
  if ((long long)ld < N || (long long)ldp < N) return fail(c, TOPO_ERR_INVALID, "topo_rom_pod: ld and ldp >= N");
  if (!dev_ptr_ok(U) || !dev_ptr_ok(Pod) || !dev_ptr_ok(sigma) || (append && !dev_ptr_ok(append)))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_pod: null or misaligned pointer");
  if (n == 0 && !append) return TOPO_OK;
  RowSplit rs = row_split(c, N, 2);
  const size_t pcap = (size_t)rs.G * m * m;
  const size_t gbytes = ((size_t)m * m * sizeof(double) + 255) & ~(size_t)255;
  const size_t cbytes = ((size_t)m * std::max(n, 1) * sizeof(double) + 255) & ~(size_t)255;
  topo_status s = ensure_scratch(c, pcap * sizeof(double) + gbytes + cbytes + 256);
  if (s) return s;
  double* partial = (double*)c->d_scratch;
  double* gram = (double*)((char*)c->d_scratch + pcap * sizeof(double));
  double* coef = (double*)((char*)gram + gbytes);
  if (n > 0) {
    s = launch_atb<double>(c, U, ld, m, U, ld, m, N, partial, pcap, gram, 1);
    if (s) return s;
    const int smem = 2 * POD_MAX * (POD_MAX + 1) * (int)sizeof(double);
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(pod_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pod_jacobi_kernel<<<1, 256, smem, c->stream>>>(gram, m, skip, n, coef, sigma);
    note_launch();
  }
  const long long blocks = std::min<long long>(4LL * c->num_sms, (N + 255) / 256);
  pod_combine_kernel<<<(int)blocks, 256, (size_t)m * std::max(n, 1) * sizeof(double), c->stream>>>(
      U, ld, m, coef, n, append, Pod, ldp, N);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_rom_rhs(topo_ctx* c, const double* Phi, int k, int ld, const double* v, double* out) {
  if (!c) return TOPO_ERR_INVALID;
  const long long N = c->g.ndof;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_rhs: 1 <= k <= 128");
  if ((long long)ld < N) return fail(c, TOPO_ERR_INVALID, "topo_rom_rhs: ld < N");
  if (!dev_ptr_ok(Phi) || !dev_ptr_ok(v) || !dev_ptr_ok(out))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_rhs: null or misaligned pointer");
  const size_t pcap = partial_capacity(c, N, k);
  topo_status s = ensure_scratch(c, pcap * sizeof(double) + 256);
  if (s) return s;
  return launch_atv(c, Phi, ld, k, v, N, (double*)c->d_scratch, pcap, out, nullptr);
}

// ---------------------------------------------------------------------------------------
// sigma_min(K(rho)) by shift-invert Lanczos (Lanczos on K^-1, each step a topo_solve_hdm),
// for the a posteriori bounds of Section 3.3 (Theorem rom_primal_error, rom_output_error).
// ---------------------------------------------------------------------------------------
namespace topo {

// A start vector with no component on Dirichlet DOFs (the Krylov space then stays on the free
// DOFs, where K is the paper's eliminated K_ff) and a deterministic spread elsewhere.
__global__ void lanczos_start_kernel(Grid g, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.ndof; i += (long long)gridDim.x * blockDim.x)
    v[i] = is_fixed(g, i) ? 0.0 : 1.0 + (double)(((unsigned long long)i * 2654435761ull) % 1024ull) / 1024.0;
}

__global__ void lanczos_alpha_kernel(const double* h1, const double* h2, int j, double* alpha) {
  if (threadIdx.x == 0 && blockIdx.x == 0) alpha[j] = h1[j] + h2[j];
}

__global__ void lanczos_tri_kernel(const double* alpha, const double* beta, int m, double* T) {
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int r = t / m, c = t % m;
    T[t] = r == c ? alpha[r] : (c == r + 1 ? beta[r] : (r == c + 1 ? beta[c] : 0.0));
  }
}

// out = [1 / theta, 1 / (theta + beta_m |s_m|), theta, beta_m |s_m|] from the top Ritz pair of T
// (sigma[0]^2 = theta, coef[m - 1] sigma[0] = the last component of its unit eigenvector).
__global__ void lanczos_final_kernel(const double* sigma, const double* coef, const double* beta, int m, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double theta = sigma[0] * sigma[0];
  const double res = beta[m - 1] * fabs(coef[m - 1] * sigma[0]);
  out[0] = 1.0 / theta;
  out[1] = 1.0 / (theta + res);
  out[2] = theta;
  out[3] = res;
}

}  // namespace topo

extern "C" topo_status topo_sigma_min(topo_ctx* c, const double* rho, int steps, double rtol, double* out) {
  if (!c) return TOPO_ERR_INVALID;
  if (steps < 2 || steps > POD_MAX) return fail(c, TOPO_ERR_INVALID, "topo_sigma_min: 2 <= steps <= 64");
  if (!(rtol > 0.0 && rtol <= 1e-2)) return fail(c, TOPO_ERR_INVALID, "topo_sigma_min: 0 < rtol <= 1e-2");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(out)) return fail(c, TOPO_ERR_INVALID, "topo_sigma_min: null or misaligned pointer");
  const long long N = c->g.ndof;
  const size_t pcap = partial_capacity(c, N, steps + 1);
  // one buffer of its own: the solves use the context's scratch
  const size_t nV = (size_t)(steps + 1) * N, nsmall = 4 * (size_t)(steps + 1) + (size_t)steps * steps + 2 * steps + 8;
  double* buf = nullptr;
  TOPO_CUDA_TRY(c, cudaMalloc(&buf, sizeof(double) * (nV + pcap + nsmall)));
  double* V = buf;
  double* partial = V + nV;
  double* h1 = partial + pcap;
  double* h2 = h1 + (steps + 1);
  double* alpha = h2 + (steps + 1);
  double* beta = alpha + (steps + 1);
  double* T = beta + (steps + 1);
  double* coef = T + (size_t)steps * steps;
  double* sigma = coef + steps;
  double* nrm = sigma + steps;
  topo_status st = TOPO_OK;
  const int nb = stream_blocks(c, N);
  const RowSplit rs = row_split(c, N, 4);
  auto normalize = [&](double* x, double* into) -> topo_status {
    nrm2_partial_kernel<<<rs.G, 256, 0, c->stream>>>(x, N, partial);
    note_launch();
    nrm2_final_kernel<<<1, 256, 0, c->stream>>>(partial, rs.G, into);
    note_launch();
    scale_kernel<<<nb, 256, 0, c->stream>>>(x, N, into);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    return TOPO_OK;
  };
  lanczos_start_kernel<<<nb, 256, 0, c->stream>>>(c->g, V);
  note_launch();
  st = normalize(V, nrm);
  for (int j = 0; j < steps && !st; ++j) {
    double* vj = V + (size_t)j * N;
    double* w = V + (size_t)(j + 1) * N;
    if (cudaMemsetAsync(w, 0, sizeof(double) * N, c->stream) != cudaSuccess) {
      st = fail(c, TOPO_ERR_CUDA, "topo_sigma_min: memset");
      break;
    }
    topo_solve_info info;
    st = topo_solve_hdm(c, rho, vj, w, 1, (int)N, rtol, 200000, TOPO_FP64, &info);
    if (st) break;
    // w -= V_j (V_j^T w), twice (CGS2); alpha_j is the sum of both passes' j-th coefficient
    const int k = j + 1;
    st = launch_atv(c, V, N, k, w, N, partial, pcap, h1, nullptr);
    if (st) break;
    gemv_kernel<<<nb, 256, k * sizeof(double), c->stream>>>(V, N, k, h1, w, N, 1, nullptr);
    note_launch();
    st = launch_atv(c, V, N, k, w, N, partial, pcap, h2, nullptr);
    if (st) break;
    gemv_kernel<<<nb, 256, k * sizeof(double), c->stream>>>(V, N, k, h2, w, N, 1, nullptr);
    note_launch();
    lanczos_alpha_kernel<<<1, 32, 0, c->stream>>>(h1, h2, j, alpha);
    note_launch();
    st = normalize(w, beta + j);
  }
  if (!st) {
    lanczos_tri_kernel<<<1, 256, 0, c->stream>>>(alpha, beta, steps, T);
    note_launch();
    const int smem = 2 * POD_MAX * (POD_MAX + 1) * (int)sizeof(double);
    if (cudaFuncSetAttribute(pod_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      st = fail(c, TOPO_ERR_CUDA, "topo_sigma_min: shared memory attribute");
  }
  if (!st) {
    pod_jacobi_kernel<<<1, 256, 2 * POD_MAX * (POD_MAX + 1) * sizeof(double), c->stream>>>(T, steps, -1, 1, coef, sigma);
    note_launch();
    lanczos_final_kernel<<<1, 32, 0, c->stream>>>(sigma, coef, beta, steps, out);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) st = fail(c, TOPO_ERR_CUDA, "topo_sigma_min: launch");
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  return st;
}
