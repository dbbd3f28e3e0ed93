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
constexpr int MG_STALL_ITERS = 64;    // iterations within which the V-cycle must halve ||r||
constexpr int MG_COARSE_MAX = 160;     // DOFs of the coarsest level (dense inverse)
constexpr double MG_RATIO = 30.0;      // Chebyshev interval [lambda_max / 30, lambda_max]
constexpr size_t MG_TAIL_BYTES = 96 * 1024;  // shared memory for the vectors of the levels on CTA 0

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
  float* Ainv;    // inverse of the coarsest operator, nc x nc FP32 (factorised in FP64 per solve)
  double* lmax;   // per-level Gershgorin partials [MG_MAX_LEVELS][G]
  int* coarse_ok; // 1 when the coarsest factorisation succeeded (else no coarse correction)
  int tail_off[MG_MAX_LEVELS];  // levels ls .. L - 1: float offset of their vectors in shared memory
  int tail_floats;              // floats of shared memory those vectors take
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

// Galerkin product K_c = P^T K_f P, one row of one block: entries (oc, a, b), b < DIM, of coarse
// node (I, J, K) of level Cl from fine level F, i.e. the sum over fine nodes i in the support of
// the coarse node and fine neighbours j of i in the support of coarse neighbour oc of
// w(i, coarse) (1 - fixed(i, a)) K_f[(i, a), (j, b)] w(j, neighbour). (A fixed fine column b of
// K_f is already zero, apart from the identity entry, which the row factor removes.) Written to
// the FP64 stencil and its FP32 copy; identity rows are patched afterwards (mg_galerkin_finish).
template <int DIM>
__device__ void mg_galerkin_row(const Grid& g0, const MgLevel& F, const MgLevel& Cl, bool fine0, int I, int J, int K,
                                long long n, int oc, int a) {
  const int nf[3] = {F.nnx, F.nny, F.nnz};
  const int cidx[3] = {I, J, K};
  const int off[3] = {oc % 3 - 1, (oc / 3) % 3 - 1, DIM == 3 ? oc / 9 - 1 : 0};
  const int ncd[3] = {Cl.nnx, Cl.nny, Cl.nnz};
  double acc[DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) acc[b] = 0.0;
  bool cin = true;
#pragma unroll
  for (int d = 0; d < DIM; ++d) cin = cin && cidx[d] + off[d] >= 0 && cidx[d] + off[d] < ncd[d];
  if (cin) {
    // per direction, the fine pairs (i, j) with j - i in {-1, 0, 1}, i in the support of the
    // coarse node and j in the support of its neighbour, and the weight w(i) w(j) of the pair
    short pi[3][7], pj[3][7];
    float pw[3][7];
    int np[3] = {1, 1, 1};
    pi[2][0] = pj[2][0] = 0;
    pw[2][0] = 1.f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int p = mg_pos(cidx[d], nf[d]), c2 = cidx[d] + off[d];
      int cnt = 0;
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int i = p + di;
        const float wi = (i >= 0 && i < nf[d]) ? mg_w1(i, cidx[d], nf[d]) : 0.f;
#pragma unroll
        for (int e = -1; e <= 1; ++e) {
          const int j = i + e;
          const float wj = (wi != 0.f && j >= 0 && j < nf[d]) ? mg_w1(j, c2, nf[d]) : 0.f;
          if (wj != 0.f && cnt < 7) {
            pi[d][cnt] = (short)i;
            pj[d][cnt] = (short)j;
            pw[d][cnt] = wi * wj;
            ++cnt;
          }
        }
      }
      np[d] = cnt;
    }
    for (int qz = 0; qz < np[2]; ++qz) {
      for (int qy = 0; qy < np[1]; ++qy) {
        for (int qx = 0; qx < np[0]; ++qx) {
          const int ix = pi[0][qx], iy = pi[1][qy], iz = pi[2][qz];
          const long long ni = ix + (long long)F.nnx * (iy + (long long)F.nny * iz);
          const bool rowfree = fine0 ? !is_fixed(g0, DIM * ni + a) : (__ldcg(F.fix + DIM * ni + a) == 0);
          if (!rowfree) continue;
          const double w = (double)pw[0][qx] * pw[1][qy] * pw[2][qz];
          const int nb = (pj[0][qx] - ix + 1) + 3 * (pj[1][qy] - iy + 1) + (DIM == 3 ? 9 * (pj[2][qz] - iz + 1) : 0);
#pragma unroll
          for (int b = 0; b < DIM; ++b)
            acc[b] = fma(w, __ldcg(F.C + (long long)((nb * DIM + a) * DIM + b) * F.nnodes + ni), acc[b]);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const long long o = (long long)((oc * DIM + a) * DIM + b) * Cl.nnodes + n;
    Cl.C[o] = acc[b];
    Cl.C32[o] = (float)acc[b];
  }
}

// After every block of coarse node n is written (by threads of the same CTA): row a becomes an
// identity row when its diagonal is zero (its whole fine support is fixed); writes the flag and
// D^-1 and returns the Gershgorin ratio sum_b |K_ab| / K_aa of the row.
template <int DIM>
__device__ double mg_galerkin_finish(const MgLevel& Cl, long long n, int a) {
  constexpr int NB = DIM == 2 ? 9 : 27;
  const int centre = DIM == 2 ? 4 : 13;
  double diag = Cl.C[(long long)((centre * DIM + a) * DIM + a) * Cl.nnodes + n];
  const bool ident = !(diag != 0.0);
  double rowabs = 0.0;
  for (int oc = 0; oc < NB; ++oc)
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      const long long o = (long long)((oc * DIM + a) * DIM + b) * Cl.nnodes + n;
      if (ident) {
        const double v = (oc == centre && a == b) ? 1.0 : 0.0;
        Cl.C[o] = v;
        Cl.C32[o] = (float)v;
      } else {
        rowabs += fabs(Cl.C[o]);
      }
    }
  if (ident) {
    diag = 1.0;
    rowabs = 1.0;
  }
  Cl.fix[DIM * n + a] = ident ? 1 : 0;
  Cl.dinv[DIM * n + a] = (float)(1.0 / diag);
  return rowabs / diag;
}

}  // namespace topo
