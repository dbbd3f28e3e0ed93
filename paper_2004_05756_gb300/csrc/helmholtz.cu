// Helmholtz density filter (Section 2.2, Eq. helm-soln .. cdens-star) on the structured grid:
//   b_n = (1 / 2^d) sum of psi_e over the elements around node n        (Eq. helm-res1)
//   phi = H^-1 b, H = r^2 (stiffness) + mass of the Q1 Helmholtz operator (Neumann ends)
//   rho_e = (1 / 2^d) sum of phi over the element's nodes                 (Eq. phitorho)
//
// The solve is exact, by diagonalisation. On a uniform grid of unit Q1 elements H is a Kronecker
// sum of the 1D Q1 matrices, e.g. in 2D H = r^2 (M_y (x) K_x + K_y (x) M_x) + M_y (x) M_x, and the
// 1D Neumann pair (K, M) (n elements, n + 1 nodes) has the generalised eigenvectors
// v_q[j] = cos(pi q j / n), q = 0 .. n:
//   K v_q = lambda_q M v_q,   lambda_q = 6 (1 - cos t) / (2 + cos t),  t = pi q / n,
//   v_p^T M v_q = mu_q delta_pq,   mu_q = (2 + cos t) / 3 * (n / 2)  (n for q = 0 and q = n),
// (the boundary rows are half the interior rows and the cosines are even about both ends, so
// the interior relation holds there too). With V the symmetric cosine matrix of each direction,
//   H^-1 = (V_z (x) V_y (x) V_x) D (V_z (x) V_y (x) V_x),
//   D = 1 / (mu_x mu_y mu_z (r^2 (lambda_x + lambda_y + lambda_z) + 1)),
// so phi takes two transforms (one mode product per direction, each a plain FP64 matrix product)
// and a diagonal scaling. With unit elements the load map is 2^d times the transpose of the
// averaging map and H is symmetric, so the filter is its own adjoint.
//
// The R fields of a batched call share every matrix product (stacked along a free dimension).
// The cosines are formed from the exact integer residue (q j) mod 2n.
#include <cmath>

#include "common.cuh"

namespace topo {

constexpr int GB_M = 64, GB_N = 64, GB_K = 16;
constexpr double kPi = 3.141592653589793238462643383279502884;

// C[b] = A[b] B[b] (row-major, leading dimensions lda, ldb, ldc; batch strides sA, sB, sC;
// a stride of 0 shares the operand). Tile TM x TN (64 x 64, or 32 x 32 when the big tiles would
// leave SMs idle: FP64 FMA issue is the bound, so every SM should hold a tile), 256 threads as a
// 16 x 16 grid, each with (TM / 16) x (TN / 16) outputs at rows ty + 16i and columns tx + 16j
// (conflict-free shared-memory reads, coalesced stores).
template <int TM, int TN>
__global__ void __launch_bounds__(256) helm_gemm_kernel(int M, int N, int K, const double* __restrict__ A,
                                                        long long lda, long long sA, const double* __restrict__ B,
                                                        long long ldb, long long sB, double* __restrict__ C,
                                                        long long ldc, long long sC) {
  constexpr int RI = TM / 16, RJ = TN / 16;
  __shared__ double As[GB_K][TM + 1];
  __shared__ double Bs[GB_K][TN + 1];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[RI][RJ];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < RJ; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += GB_K) {
#pragma unroll
    for (int q = 0; q < (TM * GB_K) / 256; ++q) {
      const int t = threadIdx.x + 256 * q;
      const int r = t / GB_K, kk = t % GB_K;
      const int gr = m0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[(long long)gr * lda + gk] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < (TN * GB_K) / 256; ++q) {
      const int t = threadIdx.x + 256 * q;
      const int kb = t / TN, cb = t % TN;
      const int gkb = k0 + kb, gc = n0 + cb;
      Bs[kb][cb] = (gkb < K && gc < N) ? B[(long long)gkb * ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      double a[RI], b[RJ];
#pragma unroll
      for (int i = 0; i < RI; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int gr = m0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < RJ; ++j) {
      const int gc = n0 + tx + 16 * j;
      if (gc < N) C[(long long)gr * ldc + gc] = acc[i][j];
    }
  }
}

// The cosine matrix of one direction (n elements): V[q][j] = cos(pi ((q j) mod 2n) / n).
__global__ void helm_cos_kernel(int n, double* V) {
  const int n1 = n + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n1 * n1;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q = t / n1, j = t - q * n1;
    const long long m = (q * j) % (2LL * n);
    V[t] = cos(kPi * (double)m / (double)n);
  }
}

// 1D eigen data of one direction: lambda_q and mu_q (lm[0..n], lm[n+1..2n+1]).
__device__ inline void helm_eig1(int n, int q, double* lambda, double* mu) {
  const double c = cos(kPi * (double)q / (double)n);
  *lambda = 6.0 * (1.0 - c) / (2.0 + c);
  *mu = (2.0 + c) / 3.0 * ((q == 0 || q == n) ? (double)n : 0.5 * (double)n);
}

// D[(qz, qy, qx)] = 1 / (mu_x mu_y mu_z (r^2 (lambda_x + lambda_y + lambda_z) + 1)).
__global__ void helm_diag_kernel(Grid g, double r2, double* D) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nnodes;
       t += (long long)gridDim.x * blockDim.x) {
    const int qx = (int)(t % g.nnx);
    const long long rest = t / g.nnx;
    const int qy = (int)(rest % g.nny), qz = (int)(rest / g.nny);
    double lx, mx, ly, my, lz = 0.0, mz = 1.0;
    helm_eig1(g.nx, qx, &lx, &mx);
    helm_eig1(g.ny, qy, &ly, &my);
    if (g.dim == 3) helm_eig1(g.nz, qz, &lz, &mz);
    D[t] = 1.0 / (mx * my * mz * (r2 * (lx + ly + lz) + 1.0));
  }
}

// b_n = 2^-d sum of the field over the elements around node n, for R fields (field r at
// in + r ldin; output contiguous, field-major).
__global__ void helm_load_kernel(Grid g, const double* __restrict__ in, long long ldin, int R, double* out) {
  const double s = g.dim == 2 ? 0.25 : 0.125;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nnodes * R;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / g.nnodes);
    const long long n = t - (long long)r * g.nnodes;
    const int i = (int)(n % g.nnx);
    const long long rest = n / g.nnx;
    const int j = (int)(rest % g.nny), k = (int)(rest / g.nny);
    const double* f = in + (long long)r * ldin;
    double acc = 0.0;
    for (int dz = (g.dim == 3 ? -1 : 0); dz <= 0; ++dz) {
      const int ez = k + dz;
      if (g.dim == 3 && (ez < 0 || ez >= g.nz)) continue;
      for (int dy = -1; dy <= 0; ++dy) {
        const int ey = j + dy;
        if (ey < 0 || ey >= g.ny) continue;
        for (int dx = -1; dx <= 0; ++dx) {
          const int ex = i + dx;
          if (ex < 0 || ex >= g.nx) continue;
          acc += f[ex + (long long)g.nx * (ey + (long long)g.ny * (g.dim == 3 ? ez : 0))];
        }
      }
    }
    out[t] = s * acc;
  }
}

__global__ void helm_scale_kernel(long long nnodes, int R, const double* __restrict__ D, double* X) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nnodes * R;
       t += (long long)gridDim.x * blockDim.x)
    X[t] *= D[t % nnodes];
}

// rho_e = 2^-d sum of phi over the element's nodes, for R fields (out + r ldout).
__global__ void helm_avg_kernel(Grid g, const double* __restrict__ phi, int R, double* out, long long ldout) {
  const double s = g.dim == 2 ? 0.25 : 0.125;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.nel * R;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / g.nel);
    const long long e = t - (long long)r * g.nel;
    const int i = (int)(e % g.nx);
    const long long rest = e / g.nx;
    const int j = (int)(rest % g.ny), k = (int)(rest / g.ny);
    const double* f = phi + (long long)r * g.nnodes;
    double acc = 0.0;
    for (int dz = 0; dz <= (g.dim == 3 ? 1 : 0); ++dz)
      for (int dy = 0; dy <= 1; ++dy)
        for (int dx = 0; dx <= 1; ++dx) acc += f[(i + dx) + (long long)g.nnx * ((j + dy) + (long long)g.nny * (k + dz))];
    out[(long long)r * ldout + e] = s * acc;
  }
}

static long long grid_cap(topo_ctx* c, long long n) {
  long long b = (n + 255) / 256;
  return std::max(1LL, std::min(b, 16LL * c->num_sms));
}

static topo_status gemm(topo_ctx* c, int M, int N, int K, const double* A, long long lda, long long sA, const double* B,
                        long long ldb, long long sB, double* C, long long ldc, long long sC, int batch) {
  const long long big = (long long)((N + GB_N - 1) / GB_N) * ((M + GB_M - 1) / GB_M) * batch;
  if (big >= c->num_sms) {
    const dim3 grid((unsigned)((N + GB_N - 1) / GB_N), (unsigned)((M + GB_M - 1) / GB_M), (unsigned)batch);
    helm_gemm_kernel<GB_M, GB_N><<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  } else {
    const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32), (unsigned)batch);
    helm_gemm_kernel<32, 32><<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  }
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

// X (R fields of nnz x nny x nnx, x fastest) -> (Vz (x) Vy (x) Vx) X, through Y; the result ends
// in X or Y: returns the buffer that holds it.
static double* helm_transform(topo_ctx* c, int R, double* X, double* Y, topo_status* st) {
  const Grid& g = c->g;
  const long long nx1 = g.nnx, ny1 = g.nny, nz1 = g.nnz;
  const double* Vx = c->d_helm;
  const double* Vy = Vx + nx1 * nx1;
  const double* Vz = Vy + ny1 * ny1;
  // along x: every row of nx1 values times Vx (V symmetric: row q of V = column q)
  *st = gemm(c, (int)(R * nz1 * ny1), (int)nx1, (int)nx1, X, nx1, 0, Vx, nx1, 0, Y, nx1, 0, 1);
  if (*st) return nullptr;
  // along y: Vy times each (ny1 x nx1) slab
  *st = gemm(c, (int)ny1, (int)nx1, (int)ny1, Vy, ny1, 0, Y, nx1, ny1 * nx1, X, nx1, ny1 * nx1, (int)(R * nz1));
  if (*st) return nullptr;
  if (g.dim == 2) return X;
  // along z: Vz times each field's (nz1 x ny1 nx1) block
  *st = gemm(c, (int)nz1, (int)(ny1 * nx1), (int)nz1, Vz, nz1, 0, X, ny1 * nx1, nz1 * ny1 * nx1, Y, ny1 * nx1,
             nz1 * ny1 * nx1, R);
  if (*st) return nullptr;
  return Y;
}

// Cosine matrices, the diagonal and two R-field work buffers in the context's own allocation
// (the filter runs inside other calls that hold the generic scratch).
static topo_status helm_prepare(topo_ctx* c, int R) {
  const Grid& g = c->g;
  const double r = c->helm_r > 0.0 ? c->helm_r : c->rmin / (2.0 * std::sqrt(3.0));
  const long long nx1 = g.nnx, ny1 = g.nny, nz1 = g.nnz;
  const size_t fixed = (size_t)(nx1 * nx1 + ny1 * ny1 + (g.dim == 3 ? nz1 * nz1 : 0) + g.nnodes);
  const size_t need = fixed + 2 * (size_t)R * g.nnodes;
  if (need * sizeof(double) > c->helm_bytes) {
    TOPO_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->d_helm) cudaFree(c->d_helm);
    c->d_helm = nullptr;
    c->helm_bytes = 0;
    TOPO_CUDA_TRY(c, cudaMalloc(&c->d_helm, need * sizeof(double)));
    c->helm_bytes = need * sizeof(double);
    c->helm_r_built = -1.0;
  }
  if (c->helm_r_built != r) {
    double* Vx = c->d_helm;
    double* Vy = Vx + nx1 * nx1;
    double* Vz = Vy + ny1 * ny1;
    double* D = Vz + (g.dim == 3 ? nz1 * nz1 : 0);
    helm_cos_kernel<<<(int)grid_cap(c, nx1 * nx1), 256, 0, c->stream>>>(g.nx, Vx);
    note_launch();
    helm_cos_kernel<<<(int)grid_cap(c, ny1 * ny1), 256, 0, c->stream>>>(g.ny, Vy);
    note_launch();
    if (g.dim == 3) {
      helm_cos_kernel<<<(int)grid_cap(c, nz1 * nz1), 256, 0, c->stream>>>(g.nz, Vz);
      note_launch();
    }
    helm_diag_kernel<<<(int)grid_cap(c, g.nnodes), 256, 0, c->stream>>>(g, r * r, D);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    c->helm_r_built = r;
  }
  return TOPO_OK;
}

// The Helmholtz filter of R fields (its own adjoint): field r at in + r ldin -> out + r ldout.
topo_status helmholtz_apply(topo_ctx* c, const double* in, long long ldin, double* out, long long ldout, int R) {
  const Grid& g = c->g;
  if (R < 1) return TOPO_OK;
  constexpr int RMAX = 32;  // fields per pass (bounds the work buffers)
  for (int r0 = 0; r0 < R; r0 += RMAX) {
    const int nr = std::min(RMAX, R - r0);
    topo_status s = helm_prepare(c, nr);
    if (s) return s;
    const long long nx1 = g.nnx, ny1 = g.nny, nz1 = g.nnz;
    const double* D = c->d_helm + nx1 * nx1 + ny1 * ny1 + (g.dim == 3 ? nz1 * nz1 : 0);
    double* X = const_cast<double*>(D) + g.nnodes;
    double* Y = X + (size_t)nr * g.nnodes;
    helm_load_kernel<<<(int)grid_cap(c, g.nnodes * nr), 256, 0, c->stream>>>(g, in + (long long)r0 * ldin, ldin, nr, X);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
    double* T = helm_transform(c, nr, X, Y, &s);
    if (s) return s;
    helm_scale_kernel<<<(int)grid_cap(c, g.nnodes * nr), 256, 0, c->stream>>>(g.nnodes, nr, D, T);
    note_launch();
    double* U = T == X ? Y : X;
    double* P = helm_transform(c, nr, T, U, &s);
    if (s) return s;
    helm_avg_kernel<<<(int)grid_cap(c, g.nel * nr), 256, 0, c->stream>>>(g, P, nr, out + (long long)r0 * ldout, ldout);
    note_launch();
    TOPO_CUDA_TRY(c, cudaGetLastError());
  }
  return TOPO_OK;
}

}  // namespace topo
