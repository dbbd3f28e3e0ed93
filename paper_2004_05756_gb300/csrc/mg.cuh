// Geometric multigrid preconditioner of the FP64 stencil PCG (pcg2.cu): level data and the
// per-node operations of one V-cycle.
//
// Levels. Level 0 is the mesh's node grid with K(rho) assembled per node (3^d blocks of
// d x d). Each coarser level keeps, per direction, the fine nodes at even positions and the
// last node: coarse node I sits on fine node min(2I, n_f - 1), so n_c = n_f / 2 + 1 and a
// direction of 1 or 2 nodes stops coarsening. The prolongation P is linear interpolation per
// direction (tensor product, every displacement component alike): a fine node on a coarse
// position copies it, any other fine node averages its two coarse neighbours. Rows of P for
// Dirichlet DOFs are zero, so a coarse correction never moves a fixed DOF.
//
// Coarse operators are Galerkin products K_{l+1} = P^T K_l P, formed in FP64 from the FP64
// stencil of the finer level (again 3^d blocks of d x d per node). A coarse DOF whose whole
// fine support is fixed has an all-zero row and column; it becomes an identity row, the same
// convention as the Dirichlet rows of level 0. The coarsest level (at most MG_COARSE_MAX DOFs)
// is solved exactly with its dense inverse, computed in FP64 once per solve.
//
// Smoothing: d steps of the Chebyshev iteration for D^-1 K on [lambda_max / ratio,
// lambda_max], lambda_max the Gershgorin bound of D^-1 K of that level, before the coarse
// correction (from a zero guess) and the same d steps after it, so the V-cycle is a symmetric
// operator. The V-cycle runs in FP32 on FP32 copies of every stencil; the CG around it, its
// residuals and its stopping test stay FP64.
#pragma once

#include "common.cuh"

namespace topo {

constexpr int MG_MAX_LEVELS = 12;
constexpr int MG_MAX_DEG = 4;          // Chebyshev smoothing steps per side
constexpr int MG_COARSE_MAX = 160;     // DOFs of the coarsest level (dense inverse)
constexpr double MG_RATIO = 30.0;      // Chebyshev interval [lambda_max / 30, lambda_max]

struct MgLevel {
  int nnx, nny, nnz;
  long long nnodes, ndof, nunits;  // nunits: ceil(nnx / 32) * nny * nnz (32 nodes of an x-row each)
  double* C;            // FP64 stencil [NC][nnodes] (coefficient-major; level 0: the solve's stencil)
  float* C32;           // FP32 copy
  float* dinv;          // FP32 D^-1 [ndof]
  unsigned char* fix;   // identity-row DOFs [ndof] (levels >= 1; level 0 uses the grid's bitmask)
  float* v;             // V-cycle vectors: slots of ndof x m floats (column stride ndof)
};

struct MgArgs {
  int L;          // levels (L >= 2)
  int ls;         // levels ls .. L - 1 run on CTA 0 alone (1 <= ls <= L - 1)
  int deg;        // Chebyshev smoothing steps per side (1 .. MG_MAX_DEG)
  int nc;         // DOFs of the coarsest level
  double* A;      // coarsest operator, dense nc x nc FP64 (row-major), Cholesky factor in place
  float* Ainv;    // its inverse, nc x nc FP32
  double* lmax;   // per-level Gershgorin partials [MG_MAX_LEVELS][G]
  int* coarse_ok; // 1 when the coarsest factorisation succeeded (else no coarse correction)
  MgLevel lv[MG_MAX_LEVELS];
};

// Vector slots of a level (deg = d): pre-smoothing iterates x_0 .. x_{d-1} in slots 0 .. d-1,
// the residual after pre-smoothing in slot d, post-smoothing iterates y_0 .. y_d in slots
// d + 1 .. 2d + 1 (y_0 = x_{d-1} + P x_coarse), the restricted right-hand side in slot 2d + 2.
// The coarsest level keeps its solution in slot 0 and its right-hand side in slot 2d + 2.
__host__ __device__ constexpr int mg_slots(int deg) { return 2 * deg + 3; }
__host__ __device__ constexpr int mg_slot_res(int deg) { return deg; }
__host__ __device__ constexpr int mg_slot_post(int deg, int j) { return deg + 1 + j; }
__host__ __device__ constexpr int mg_slot_b(int deg) { return 2 * deg + 2; }

__host__ __device__ inline int mg_coarse_n(int nf) { return nf / 2 + 1; }

// Fine position of coarse node I on a direction of nf fine nodes.
__device__ __forceinline__ int mg_pos(int I, int nf) { return min(2 * I, nf - 1); }
// Is fine node i a coarse position?
__device__ __forceinline__ bool mg_is_cpos(int i, int nf) { return (i & 1) == 0 || i == nf - 1; }
// 1D interpolation weight of coarse node I at fine node i (0, 1/2 or 1).
__device__ __forceinline__ float mg_w1(int i, int I, int nf) {
  const int p = mg_pos(I, nf);
  if (i == p) return 1.f;
  if ((i == p - 1 || i == p + 1) && !mg_is_cpos(i, nf)) return 0.5f;
  return 0.f;
}

// A Grid describing level L's node grid (only the fields the stencil applies read).
__device__ __forceinline__ Grid mg_grid(const Grid& g0, const MgLevel& L) {
  Grid g = g0;
  g.nnx = L.nnx;
  g.nny = L.nny;
  g.nnz = L.nnz;
  g.nnodes = L.nnodes;
  g.ndof = L.ndof;
  return g;
}

// Unit index of node (i, j, k) on a level.
__device__ __forceinline__ long long mg_unit(const MgLevel& L, int i, int j, int k) {
  const long long ux = (L.nnx + 31) / 32;
  return (long long)(i / 32) + ux * (j + (long long)L.nny * k);
}

// Owner of unit u among G CTAs that split n units into contiguous ranges [n r / G, n (r+1) / G).
__device__ __forceinline__ long long mg_owner(long long u, long long n, long long G) {
  long long b = u * G / n;
  while (b + 1 < G && n * (b + 1) / G <= u) ++b;
  while (b > 0 && n * b / G > u) --b;
  return b;
}

// Galerkin row block of coarse node (I, J, K) of level Lc from fine level Lf: for every coarse
// neighbour offset (3^d blocks), sum over fine nodes i in the support of the coarse node and
// fine neighbours j of i in the support of the coarse neighbour of
// w(i, coarse) (1 - fixed(i, a)) K_f[(i, a), (j, b)] w(j, neighbour).
// Writes the FP64 block row (identity rows where the row is all zero) and its FP32 copy, the
// identity-row flags, D^-1 (FP32), and returns the Gershgorin ratio max_a sum_b |K_ab| / K_aa.
template <int DIM>
__device__ double mg_galerkin_node(const Grid& g0, const MgLevel& F, const MgLevel& Cl, bool fine0, int I, int J,
                                   int K, long long n) {
  constexpr int NB = DIM == 2 ? 9 : 27, DD = DIM * DIM;
  const int nfx = F.nnx, nfy = F.nny, nfz = F.nnz;
  const int px = mg_pos(I, nfx), py = mg_pos(J, nfy), pz = DIM == 3 ? mg_pos(K, nfz) : 0;
  double rowabs[DIM], diag[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) rowabs[a] = diag[a] = 0.0;
  const int centre = DIM == 2 ? 4 : 13;
  // first pass computes the blocks; identity rows are decided from the diagonal, so the
  // blocks are written, then patched in a second pass if a row is all zero
#pragma unroll 1
  for (int oc = 0; oc < NB; ++oc) {
    const int ox = oc % 3 - 1, oy = (oc / 3) % 3 - 1, oz = DIM == 3 ? oc / 9 - 1 : 0;
    const int I2 = I + ox, J2 = J + oy, K2 = K + oz;
    double acc[DD];
#pragma unroll
    for (int q = 0; q < DD; ++q) acc[q] = 0.0;
    const bool cin = I2 >= 0 && I2 < Cl.nnx && J2 >= 0 && J2 < Cl.nny && (DIM == 2 || (K2 >= 0 && K2 < Cl.nnz));
    if (cin) {
      const int qx = mg_pos(I2, nfx), qy = mg_pos(J2, nfy), qz = DIM == 3 ? mg_pos(K2, nfz) : 0;
      for (int iz = (DIM == 3 ? max(pz - 1, 0) : 0); iz <= (DIM == 3 ? min(pz + 1, nfz - 1) : 0); ++iz) {
        const float wz = DIM == 3 ? mg_w1(iz, K, nfz) : 1.f;
        if (wz == 0.f) continue;
        for (int iy = max(py - 1, 0); iy <= min(py + 1, nfy - 1); ++iy) {
          const float wy = mg_w1(iy, J, nfy);
          if (wy == 0.f) continue;
          for (int ix = max(px - 1, 0); ix <= min(px + 1, nfx - 1); ++ix) {
            const float wx = mg_w1(ix, I, nfx);
            if (wx == 0.f) continue;
            const double wi = (double)wx * wy * wz;
            const long long ni = ix + (long long)nfx * (iy + (long long)nfy * iz);
            bool rowfree[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
              rowfree[a] = fine0 ? !is_fixed(g0, DIM * ni + a) : (__ldcg(F.fix + DIM * ni + a) == 0);
            // fine neighbours j of i inside the support of the coarse neighbour
            for (int jz = (DIM == 3 ? max(iz - 1, max(qz - 1, 0)) : 0);
                 jz <= (DIM == 3 ? min(iz + 1, min(qz + 1, nfz - 1)) : 0); ++jz) {
              const float vz = DIM == 3 ? mg_w1(jz, K2, nfz) : 1.f;
              if (vz == 0.f) continue;
              for (int jy = max(iy - 1, max(qy - 1, 0)); jy <= min(iy + 1, min(qy + 1, nfy - 1)); ++jy) {
                const float vy = mg_w1(jy, J2, nfy);
                if (vy == 0.f) continue;
                for (int jx = max(ix - 1, max(qx - 1, 0)); jx <= min(ix + 1, min(qx + 1, nfx - 1)); ++jx) {
                  const float vx = mg_w1(jx, I2, nfx);
                  if (vx == 0.f) continue;
                  const double wij = wi * ((double)vx * vy * vz);
                  const int nb = (jx - ix + 1) + 3 * (jy - iy + 1) + (DIM == 3 ? 9 * (jz - iz + 1) : 0);
#pragma unroll
                  for (int a = 0; a < DIM; ++a) {
                    if (!rowfree[a]) continue;
#pragma unroll
                    for (int b = 0; b < DIM; ++b)
                      acc[a * DIM + b] =
                          fma(wij, __ldcg(F.C + (long long)((nb * DIM + a) * DIM + b) * F.nnodes + ni), acc[a * DIM + b]);
                  }
                }
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        const double v = acc[a * DIM + b];
        Cl.C[(long long)((oc * DIM + a) * DIM + b) * Cl.nnodes + n] = v;
        rowabs[a] += fabs(v);
        if (oc == centre && a == b) diag[a] = v;
      }
  }
  double gmax = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const bool ident = !(diag[a] != 0.0);
    Cl.fix[DIM * n + a] = ident ? 1 : 0;
    if (ident) {
      for (int oc = 0; oc < NB; ++oc)
#pragma unroll
        for (int b = 0; b < DIM; ++b)
          Cl.C[(long long)((oc * DIM + a) * DIM + b) * Cl.nnodes + n] = (oc == centre && a == b) ? 1.0 : 0.0;
      diag[a] = 1.0;
      rowabs[a] = 1.0;
    }
    Cl.dinv[DIM * n + a] = (float)(1.0 / diag[a]);
    gmax = fmax(gmax, rowabs[a] / diag[a]);
  }
  for (int q = 0; q < NB * DD; ++q) {
    const long long o = (long long)q * Cl.nnodes + n;
    Cl.C32[o] = (float)Cl.C[o];
  }
  return gmax;
}

}  // namespace topo
