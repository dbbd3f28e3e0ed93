// FP64 state solve K(rho) u = f with K assembled per node, Chronopoulos-Gear PCG, one persistent
// cooperative launch.
//
// GB300's FP64 rate is 1/61 of its FP32 rate, so in FP64 the element-by-element product
// (72 FMAs per node in 2D, 600 in 3D) is the bottleneck of every CG iteration. The density is
// fixed during a solve, so this kernel first assembles the stencil of K(rho) once per node:
// for each of the 3^d neighbour offsets a dim x dim block sum_e E(rho_e) K_e[node, neighbour],
// stored structure-of-arrays (coefficient-major, node fastest) so that warps read it coalesced.
// Every CG iteration then costs 36 (2D) / 243 (3D) FMAs per node instead of 72 / 600. The
// Dirichlet convention (identity rows and columns) is folded into the stencil.
//
// Work split: a unit is 32 consecutive nodes of one x-row, one warp. Each CTA owns a contiguous,
// equal share of the units (balanced to one unit), so partial sums are accumulated in a fixed
// order and every result is deterministic. Each iteration has two grid-wide barriers; after
// each one every CTA reduces the per-CTA partial dot products itself, in a fixed order
// (Chronopoulos-Gear: both dot products of an iteration in one reduction). The pipelined CG
// recurrences (one barrier per iteration) were tried and rejected: on these high-contrast
// designs they diverge, and periodic residual replacement makes them stagnate.
#include <algorithm>
#include <type_traits>

#include "pcg2.cuh"

namespace topo {

__device__ __forceinline__ void unit_coords(const Grid& g, long long u, int& i0, int& j, int& kz) {
  const int ux = (g.nnx + 31) / 32;
  i0 = (int)(u % ux) * 32;
  const long long r = u / ux;
  j = (int)(r % g.nny);
  kz = (int)(r / g.nny);
}

// Assemble the stencil rows of node (i, j, k). Element (a, b, c) in {0,1}^d has its lower
// corner at node - 1 + (a, b, c); the node is its local corner (1-a, 1-b, 1-c), and the
// neighbour at offset (dx, dy, dz) is its local corner (dx+1-a, dy+1-b, dz+1-c) when that lies
// in {0,1}^d. Each neighbour block sums E_e K_e[node rows, neighbour columns] over those
// elements. Dirichlet convention: a fixed row is the identity, a fixed neighbour column zero.
template <int DIM>
__device__ void assemble_node(const Grid& g, const typename KeOf<DIM, double>::type& ke, const double* rho,
                              int i, int j, int k, long long n, double* C, float* C32 = nullptr) {
  constexpr int NB = StencilGeom<DIM>::NB, ND = DIM == 2 ? 8 : 24, NE = DIM == 2 ? 4 : 8;
  double E[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
    const int ei = i - 1 + a, ej = j - 1 + b, ek = k - 1 + c;
    const bool in = ei >= 0 && ei < g.nx && ej >= 0 && ej < g.ny && (DIM == 2 || (ek >= 0 && ek < g.nz));
    const long long e = in ? ei + (long long)g.nx * (ej + (long long)g.ny * (DIM == 3 ? ek : 0)) : 0;
    E[q] = in ? young<double>(__ldg(rho + e), g.E0, g.Emin, g.ipenal) : 0.0;
  }
  const int centre = DIM == 2 ? 4 : 13;
  bool rfix[DIM];
#pragma unroll
  for (int r = 0; r < DIM; ++r) rfix[r] = is_fixed(g, DIM * n + r);
#pragma unroll 1
  for (int nb = 0; nb < NB; ++nb) {
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = DIM == 3 ? nb / 9 - 1 : 0;
    double acc[DIM * DIM];
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) acc[q] = 0.0;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
      const int cx = dx + 1 - a, cy = dy + 1 - b, cz = DIM == 3 ? dz + 1 - c : 0;
      if (cx < 0 || cx > 1 || cy < 0 || cy > 1 || cz < 0 || cz > 1) continue;
      const int L = DIM == 2 ? lidx2(1 - a, 1 - b) : lidx3(1 - a, 1 - b, 1 - c);
      const int M = DIM == 2 ? lidx2(cx, cy) : lidx3(cx, cy, cz);
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int d = 0; d < DIM; ++d) acc[r * DIM + d] = fma(E[q], ke.k[(DIM * L + r) * ND + DIM * M + d], acc[r * DIM + d]);
    }
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny && (DIM == 2 || (kk >= 0 && kk < g.nnz));
    const long long m = nin ? ii + (long long)g.nnx * (jj + (long long)g.nny * kk) : 0;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double v = acc[r * DIM + d];
        if (!nin || is_fixed(g, DIM * m + d)) v = 0.0;
        if (rfix[r]) v = (nb == centre && r == d) ? 1.0 : 0.0;
        C[(long long)((nb * DIM + r) * DIM + d) * g.nnodes + n] = v;
        if (C32) C32[(long long)((nb * DIM + r) * DIM + d) * g.nnodes + n] = (float)v;
      }
  }
}

// y = C v for node (i, j, k); neighbour values read from L2 (written by other CTAs).
// y = C v and yabs = |C| |v| (the scale of the rounding error of y).
template <int DIM>
__device__ __forceinline__ void stencil_apply_abs(const Grid& g, const double* __restrict__ C, const double* v, int i,
                                                  int j, int k, long long n, double* y, double* yabs) {
  constexpr int NB = StencilGeom<DIM>::NB;
#pragma unroll
  for (int r = 0; r < DIM; ++r) y[r] = yabs[r] = 0.0;
#pragma unroll 1
  for (int nb = 0; nb < NB; ++nb) {
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = DIM == 3 ? nb / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny && (DIM == 2 || (kk >= 0 && kk < g.nnz));
    if (!nin) continue;
    const long long m = ii + (long long)g.nnx * (jj + (long long)g.nny * kk);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double vv = __ldcg(v + DIM * m + d);
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        const double cc = __ldcg(C + (long long)((nb * DIM + r) * DIM + d) * g.nnodes + n);
        y[r] = fma(cc, vv, y[r]);
        yabs[r] = fma(fabs(cc), fabs(vv), yabs[r]);
      }
    }
  }
}

// y = C v for node (i, j, k); vown = v at the node itself.
template <int DIM>
__device__ __forceinline__ void stencil_apply(const Grid& g, const double* __restrict__ C, const double* v, int i,
                                              int j, int k, long long n, double* y, double* vown) {
  constexpr int NB = StencilGeom<DIM>::NB;
  if constexpr (DIM == 2) {
    // Branch-free: a neighbour outside the grid has all-zero coefficients (assembly), so its
    // value is read at the node itself and contributes fma(0, v, y) = y exactly. A node's two
    // components are one 16-byte load (half the L2 sectors of two 8-byte loads at stride 16 B).
    // All 18 values and 36 coefficients are loaded before the first FMA.
    double vv[NB][2];
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      const int ii = i + nb % 3 - 1, jj = j + nb / 3 - 1;
      const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny;
      const long long m = nin ? ii + (long long)g.nnx * jj : n;
      const double2 t = __ldcg(reinterpret_cast<const double2*>(v) + m);  // (x, y) of node m: 16 B
      vv[nb][0] = t.x;
      vv[nb][1] = t.y;
    }
    // each block's 4 coefficients are used as they arrive
    const double* gp = C + n;
    y[0] = y[1] = 0.0;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      double cc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cc[q] = __ldcg(gp + (long long)(nb * 4 + q) * g.nnodes);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int d = 0; d < 2; ++d) y[r] = fma(cc[r * 2 + d], vv[nb][d], y[r]);
    }
    vown[0] = vv[4][0];  // the centre block (nb = 4) is the node itself
    vown[1] = vv[4][1];
    return;
  }
#pragma unroll
  for (int r = 0; r < DIM; ++r) y[r] = 0.0;
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = DIM == 3 ? nb / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny && (DIM == 2 || (kk >= 0 && kk < g.nnz));
    if (!nin) continue;
    const long long m = ii + (long long)g.nnx * (jj + (long long)g.nny * kk);
    double vv[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) vv[d] = __ldcg(v + DIM * m + d);
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int d = 0; d < DIM; ++d) y[r] = fma(__ldcg(C + (long long)((nb * DIM + r) * DIM + d) * g.nnodes + n), vv[d], y[r]);
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d) vown[d] = __ldcg(v + DIM * n + d);
}

// y = C32 v in FP32 for node (i, j, k) (the FP32 preconditioners); vown: v at the node. In 2D
// the coefficients (read-only after the setup, written by the reading thread or before a grid
// barrier for levels run by one CTA) stay in L1: a CTA's share of a level fits there. In 3D
// (243 per node) they do not, and come from L2 like v, which other CTAs write during the solve.
template <int DIM, bool SMEMV = false>
__device__ __forceinline__ void stencil_apply32(const Grid& g, const float* __restrict__ C, const float* v, int i,
                                                int j, int k, long long n, float* y, float* vown) {
  constexpr int NB = StencilGeom<DIM>::NB;
#pragma unroll
  for (int r = 0; r < DIM; ++r) y[r] = 0.f;
  if constexpr (DIM == 2) {
    // as the FP64 form: a neighbour outside the grid has zero coefficients and reads the node
    float2 vv[NB];
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      const int ii = i + nb % 3 - 1, jj = j + nb / 3 - 1;
      const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny;
      const long long m = nin ? ii + (long long)g.nnx * jj : n;
      vv[nb] = SMEMV ? reinterpret_cast<const float2*>(v)[m] : __ldcg(reinterpret_cast<const float2*>(v) + m);
    }
    const float* gp = C + n;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      float cc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cc[q] = __ldca(gp + (long long)(nb * 4 + q) * g.nnodes);
      y[0] = fmaf(cc[0], vv[nb].x, y[0]);
      y[0] = fmaf(cc[1], vv[nb].y, y[0]);
      y[1] = fmaf(cc[2], vv[nb].x, y[1]);
      y[1] = fmaf(cc[3], vv[nb].y, y[1]);
    }
    vown[0] = vv[4].x;
    vown[1] = vv[4].y;
    return;
  }
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = DIM == 3 ? nb / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    const bool nin = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny && (DIM == 2 || (kk >= 0 && kk < g.nnz));
    if (!nin) continue;
    const long long m = ii + (long long)g.nnx * (jj + (long long)g.nny * kk);
    float vv[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) vv[d] = SMEMV ? v[DIM * m + d] : __ldcg(v + DIM * m + d);
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int d = 0; d < DIM; ++d) y[r] = fmaf(__ldcg(C + (long long)((nb * DIM + r) * DIM + d) * g.nnodes + n), vv[d], y[r]);
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d) vown[d] = SMEMV ? v[DIM * n + d] : __ldcg(v + DIM * n + d);
}

// The solver, run by a group of G co-resident CTAs (this CTA is number `rank` of the group)
// that share the barrier state gb.
// PK selects the preconditioner compiled in: 0 Jacobi (the batched kernel); 1 Jacobi or the
// FP32 Chebyshev polynomial of degree a.poly; 2 the FP32 geometric multigrid V-cycle (mg.cuh).
template <int DIM, int PK>
__device__ __forceinline__ void pcg2_body(const Pcg2Args<DIM>& a, const unsigned G, const unsigned rank,
                                          GridBar* gb) {
  __shared__ double red[96];
  __shared__ double sh_gamma[P2_MAX_COLS], sh_alpha[P2_MAX_COLS], sh_beta[P2_MAX_COLS], sh_tol2[P2_MAX_COLS],
      sh_ff[P2_MAX_COLS], sh_rr[P2_MAX_COLS], sh_den[P2_MAX_COLS];
  __shared__ int sh_done[P2_MAX_COLS];
  __shared__ double sh_sum[P2_SLOTS * P2_MAX_COLS];
  __shared__ double sh_floor2[P2_MAX_COLS];
  __shared__ double sh_c1[P2_MAX_POLY], sh_c2[P2_MAX_POLY], sh_itheta;  // Chebyshev coefficients
  // multigrid: per-level smoother coefficients and the CTA ranges each exchange waits for
  __shared__ float mg_ith[MG_MAX_LEVELS], mg_c1[MG_MAX_LEVELS][MG_MAX_DEG], mg_c2[MG_MAX_LEVELS][MG_MAX_DEG];
  __shared__ int mg_halo[MG_MAX_LEVELS][2], mg_rest[MG_MAX_LEVELS][2], mg_prol[MG_MAX_LEVELS][2];
  __shared__ int mg_okc;
  __shared__ int sh_fallback;  // multigrid: the FP32 V-cycle lost positive definiteness
  __shared__ double sh_rrchk[P2_MAX_COLS];  // multigrid: r.r at the last stagnation checkpoint
  __shared__ int s_okw;
  const Grid& g = a.g;
  const int m = a.m;
  const long long N = a.N;
  GridSync* gs = a.gs;
  unsigned long long bar = 0;  // grid barriers passed
  double* part = a.partial;
  // Partials written before barrier number bar + 1 go to buffer (bar + 1) & 1 and are read
  // after it; a CTA can only reuse a buffer after the next barrier, i.e. after every CTA has
  // finished reading it.
  auto P = [&](int slot, int c) -> double* {
    return part + ((size_t)((((bar + 1) & 1) * P2_SLOTS + slot) * m + c)) * G + rank;
  };
  auto R = [&](int slot, int c) -> double { return sh_sum[slot * m + c]; };
  // grid barrier, then every CTA reduces the per-CTA partials of nred slots itself
  auto sync_reduce = [&](int nred) -> bool {
    if (!grid_barrier(gb, &gs->status, bar, a.wait_cycles, G)) return false;
    if (nred > 0) reduce_slots(part + (size_t)((bar & 1) * P2_SLOTS * m) * G, G, nred, sh_sum);
    return true;
  };
  // this CTA's units: a contiguous, balanced range
  const long long u0 = a.nunits * rank / G, u1 = a.nunits * (rank + 1) / G;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // iterate over the owned nodes of this CTA: fn(i, j, k, n)
  // iterate over the owned nodes of this CTA: fn(i, j, k, n)
  auto for_owned = [&](auto fn) {
    for (long long u = u0 + warp; u < u1; u += nwarps) {
      int i0, j, kz;
      unit_coords(g, u, i0, j, kz);
      const int i = i0 + lane;
      if (i >= g.nnx) continue;
      const long long n = i + (long long)g.nnx * (j + (long long)g.nny * kz);
      fn(i, j, kz, n);
    }
  };
  // CTAs owning the nodes whose z the apply of this CTA's nodes reads: units within `span` of
  // the own range (one x-row (and one z-plane) plus one unit on either side).
  const long long ux = (g.nnx + 31) / 32;
  const long long span = DIM == 2 ? ux + 1 : ux * g.nny + ux + 1;
  auto owner = [&](long long u) -> long long {
    long long b = u * (long long)G / a.nunits;
    while (b + 1 < (long long)G && a.nunits * (b + 1) / G <= u) ++b;
    while (b > 0 && a.nunits * b / G > u) --b;
    return b;
  };
  const long long nb_lo = u1 > u0 ? owner(max(0LL, u0 - span)) : (long long)rank;
  const long long nb_hi = u1 > u0 ? owner(min(a.nunits - 1, u1 - 1 + span)) : (long long)rank;
  unsigned long long zseq = 0;  // phase-U completions so far (the same on every CTA)
  // after phase U: z of the owned nodes is complete
  auto publish_z = [&]() {
    __syncthreads();
    ++zseq;
    if (threadIdx.x == 0) {
      __threadfence();
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> f(a.zflag[rank]);
      f.store(zseq, cuda::memory_order_release);
    }
  };
  // before phase W: every neighbour has published the same z (bounded wait)
  auto wait_z = [&]() -> bool {
    if (threadIdx.x == 0) s_okw = 1;
    __syncthreads();
    for (long long q = nb_lo + threadIdx.x; q <= nb_hi; q += blockDim.x) {
      if (q == (long long)rank) continue;
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> f(a.zflag[q]);
      const long long t0 = clock64();
      while (f.load(cuda::memory_order_acquire) < zseq) {
        if (*(volatile int*)&gb->abort) {
          s_okw = 0;
          break;
        }
        if (clock64() - t0 > a.wait_cycles) {
          atomicCAS(&gs->status, 0, (int)TOPO_ERR_TIMEOUT);
          atomicExch(&gb->abort, 1);
          s_okw = 0;
          break;
        }
      }
    }
    __syncthreads();
    return s_okw != 0;
  };

  // --- multigrid setup (PK == 2), once per solve after the level-0 stencil -------------------
  // 1. Galerkin levels 1 .. L-1 (all CTAs split each level's units; a grid barrier after each),
  // 2. the coarsest operator as a dense matrix, factorised by CTA 0 (Cholesky, FP64),
  // 3. its inverse, one column per CTA, 4. the smoother coefficients of every level and the
  // ranges of CTAs each exchange of the V-cycle waits for.
  auto block_max = [&](double v) -> double {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double bm = 0.0;
    for (int q = 0; q < nwarps; ++q) bm = fmax(bm, red[q]);
    __syncthreads();
    return bm;
  };
  auto mg_setup = [&]() -> bool {
    const MgArgs& M = a.mg;
    for (int l = 0; l + 1 < M.L; ++l) {
      const MgLevel& F = M.lv[l];
      const MgLevel& Cc = M.lv[l + 1];
      const long long c0 = Cc.nunits * rank / G, c1 = Cc.nunits * (rank + 1) / G;
      const int ux = (Cc.nnx + 31) / 32;
      constexpr int NB = StencilGeom<DIM>::NB;
      // one thread per (node, neighbour block, row); nodes fastest, so stores coalesce
      const long long items = (c1 - c0) * 32 * NB * DIM;
      for (long long t = threadIdx.x; t < items; t += blockDim.x) {
        const int ln = (int)(t % 32);
        const long long rest = t / 32;
        const int ar = (int)(rest % DIM);
        const int oc = (int)((rest / DIM) % NB);
        const long long u = c0 + rest / (DIM * NB);
        const int i = (int)(u % ux) * 32 + ln;
        const long long r = u / ux;
        const int j = (int)(r % Cc.nny), k = (int)(r / Cc.nny);
        if (i >= Cc.nnx) continue;
        const long long n = i + (long long)Cc.nnx * (j + (long long)Cc.nny * k);
        mg_galerkin_row<DIM>(g, F, Cc, l == 0, i, j, k, n, oc, ar);
      }
      __syncthreads();
      double gm = 0.0;
      for (long long t = threadIdx.x; t < (c1 - c0) * 32 * DIM; t += blockDim.x) {
        const int ln = (int)(t % 32);
        const int ar = (int)((t / 32) % DIM);
        const long long u = c0 + t / (32 * DIM);
        const int i = (int)(u % ux) * 32 + ln;
        const long long r = u / ux;
        const int j = (int)(r % Cc.nny), k = (int)(r / Cc.nny);
        if (i >= Cc.nnx) continue;
        const long long n = i + (long long)Cc.nnx * (j + (long long)Cc.nny * k);
        gm = fmax(gm, mg_galerkin_finish<DIM>(Cc, n, ar));
      }
      const double bm = block_max(gm);
      if (threadIdx.x == 0) M.lmax[(size_t)(l + 1) * G + rank] = bm;
      if (!sync_reduce(0)) return false;
    }
    // Coarsest level: every CTA that owns a column of the inverse (q = rank, rank + G, ...)
    // builds the dense operator itself from the coarsest stencil, as a packed lower triangle in
    // shared memory, factorises it (Cholesky, FP64; a non-positive pivot disables the coarse
    // correction instead of failing the solve) and solves L L^T x = e_q column-wise: no grid
    // barrier and no global round trip between the steps, and the same factor on every CTA.
    const int nc = M.nc;
    if ((int)rank < nc) {
      extern __shared__ __align__(16) unsigned char mg_dyn[];
      double* Ap = reinterpret_cast<double*>(mg_dyn);      // packed lower triangle, nc (nc + 1) / 2
      double* yv = Ap + (size_t)nc * (nc + 1) / 2;          // [nc]: the column being solved
      auto pk = [&](int i, int j) -> double& { return Ap[(size_t)i * (i + 1) / 2 + j]; };
      const MgLevel& Cc = M.lv[M.L - 1];
      constexpr int NB = StencilGeom<DIM>::NB;
      for (int t = threadIdx.x; t < nc * (nc + 1) / 2; t += blockDim.x) Ap[t] = 0.0;
      __syncthreads();
      for (int row = threadIdx.x; row < nc; row += blockDim.x) {
        const long long n = row / DIM;
        const int ar = row % DIM;
        const int i = (int)(n % Cc.nnx), j = (int)((n / Cc.nnx) % Cc.nny), k = (int)(n / ((long long)Cc.nnx * Cc.nny));
        for (int nb = 0; nb < NB; ++nb) {
          const int ii = i + nb % 3 - 1, jj = j + (nb / 3) % 3 - 1, kk = DIM == 3 ? k + nb / 9 - 1 : 0;
          if (ii < 0 || ii >= Cc.nnx || jj < 0 || jj >= Cc.nny || kk < 0 || kk >= Cc.nnz) continue;
          const long long mm = ii + (long long)Cc.nnx * (jj + (long long)Cc.nny * kk);
          for (int b = 0; b < DIM; ++b) {
            const int col = (int)(DIM * mm + b);
            if (col <= row) pk(row, col) = __ldcg(Cc.C + (long long)((nb * DIM + ar) * DIM + b) * Cc.nnodes + n);
          }
        }
      }
      if (threadIdx.x == 0) mg_okc = 1;
      __syncthreads();
      for (int kq = 0; kq < nc; ++kq) {  // right-looking Cholesky, a warp per trailing row
        if (threadIdx.x == 0) {
          const double d = pk(kq, kq);
          if (!(d > 0.0) || !isfinite(d)) mg_okc = 0;
          pk(kq, kq) = mg_okc ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (!mg_okc) break;
        const double inv = 1.0 / pk(kq, kq);
        for (int i = kq + 1 + threadIdx.x; i < nc; i += blockDim.x) pk(i, kq) *= inv;
        __syncthreads();
        for (int i = kq + 1 + warp; i < nc; i += nwarps) {
          const double lik = pk(i, kq);
          for (int j = kq + 1 + lane; j <= i; j += 32) pk(i, j) = fma(-lik, pk(j, kq), pk(i, j));
        }
        __syncthreads();
      }
      if (rank == 0 && threadIdx.x == 0) *M.coarse_ok = mg_okc;
      for (int q = rank; q < nc; q += G) {  // L y = e_q, then L^T x = y (column-oriented)
        if (warp == 0) {
          for (int i = lane; i < nc; i += 32) yv[i] = (i == q) ? 1.0 : 0.0;
          __syncwarp();
          if (mg_okc) {
            for (int jc = q; jc < nc; ++jc) {
              const double yj = yv[jc] / pk(jc, jc);
              __syncwarp();
              for (int i = jc + 1 + lane; i < nc; i += 32) yv[i] = fma(-pk(i, jc), yj, yv[i]);
              if (lane == 0) yv[jc] = yj;
              __syncwarp();
            }
            for (int jc = nc - 1; jc >= 0; --jc) {
              const double xj = yv[jc] / pk(jc, jc);
              __syncwarp();
              for (int i = lane; i < jc; i += 32) yv[i] = fma(-pk(jc, i), xj, yv[i]);
              if (lane == 0) yv[jc] = xj;
              __syncwarp();
            }
          } else {
            for (int i = lane; i < nc; i += 32) yv[i] = 0.0;
            __syncwarp();
          }
          for (int i = lane; i < nc; i += 32) M.Ainv[(size_t)q * nc + i] = (float)yv[i];
          __syncwarp();
        }
      }
    }
    if (!sync_reduce(0)) return false;
    // Chebyshev coefficients of every level (as in the polynomial preconditioner above)
    if (warp < M.L) {
      double lm = 0.0;
      for (unsigned q = lane; q < G; q += 32) lm = fmax(lm, __ldcg(M.lmax + (size_t)warp * G + q));
      for (int o = 16; o; o >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
      if (lane == 0) {
        if (!(lm > 0.0) || !isfinite(lm)) lm = 1.0;
        lm *= 1.001;
        const double lmin = lm / MG_RATIO;
        const double th = 0.5 * (lm + lmin), de = 0.5 * (lm - lmin), sigma = th / de;
        mg_ith[warp] = (float)(1.0 / th);
        double ro = 1.0 / sigma;
        for (int j = 1; j < M.deg; ++j) {
          const double rn = 1.0 / (2.0 * sigma - ro);
          mg_c1[warp][j] = (float)(rn * ro);
          mg_c2[warp][j] = (float)(2.0 * rn / de);
          ro = rn;
        }
      }
    }
    // exchange ranges of the levels run by all CTAs (0 .. ls - 1)
    if (threadIdx.x < M.ls) {
      const int l = threadIdx.x;
      const MgLevel& Lv = M.lv[l];
      const long long u0 = Lv.nunits * rank / G, u1 = Lv.nunits * (rank + 1) / G;
      const long long ux = (Lv.nnx + 31) / 32;
      if (u1 > u0) {
        const long long sp = DIM == 2 ? ux + 1 : ux * Lv.nny + ux + 1;
        mg_halo[l][0] = (int)mg_owner(max(0LL, u0 - sp), Lv.nunits, G);
        mg_halo[l][1] = (int)mg_owner(min(Lv.nunits - 1, u1 - 1 + sp), Lv.nunits, G);
        // first and last owned node positions
        const int i0 = (int)(u0 % ux) * 32, j0 = (int)((u0 / ux) % Lv.nny), k0 = (int)(u0 / ux / Lv.nny);
        const long long ul = u1 - 1;
        const int i1 = min((int)(ul % ux) * 32 + 31, Lv.nnx - 1), j1 = (int)((ul / ux) % Lv.nny),
                  k1 = (int)(ul / ux / Lv.nny);
        if (l >= 1) {  // restriction from level l - 1: its owners of the fine support
          const MgLevel& F = M.lv[l - 1];
          const long long fmin = mg_unit(F, max(0, 2 * i0 - 2), max(0, 2 * j0 - 2), DIM == 3 ? max(0, 2 * k0 - 2) : 0);
          const long long fmaxu = mg_unit(F, min(F.nnx - 1, 2 * i1 + 1), min(F.nny - 1, 2 * j1 + 1),
                                          DIM == 3 ? min(F.nnz - 1, 2 * k1 + 1) : 0);
          mg_rest[l][0] = (int)mg_owner(fmin, F.nunits, G);
          mg_rest[l][1] = (int)mg_owner(fmaxu, F.nunits, G);
        }
        if (l + 1 < M.ls) {  // prolongation from level l + 1: its owners of the coarse parents
          // parents of fine node i lie in [i / 2, i / 2 + 1]; a range of owned nodes that spans
          // more than one row (plane) reaches whole coarse rows (planes), so the bounds take
          // x from 0 to the row end (and y likewise when planes are spanned)
          const MgLevel& Cc = M.lv[l + 1];
          const bool planes = DIM == 3 && k1 > k0;
          const long long cmin = mg_unit(Cc, 0, planes ? 0 : j0 / 2, DIM == 3 ? k0 / 2 : 0);
          const long long cmaxu = mg_unit(Cc, Cc.nnx - 1, planes ? Cc.nny - 1 : min(Cc.nny - 1, j1 / 2 + 1),
                                          DIM == 3 ? min(Cc.nnz - 1, k1 / 2 + 1) : 0);
          mg_prol[l][0] = (int)mg_owner(cmin, Cc.nunits, G);
          mg_prol[l][1] = (int)mg_owner(cmaxu, Cc.nunits, G);
        } else {  // level ls is run by CTA 0
          mg_prol[l][0] = mg_prol[l][1] = 0;
        }
      } else {
        mg_halo[l][0] = mg_halo[l][1] = mg_rest[l][0] = mg_rest[l][1] = mg_prol[l][0] = mg_prol[l][1] = (int)rank;
      }
    }
    __syncthreads();
    return true;
  };

  // --- stencil assembly and Jacobi diagonal ----------------------------------------------
  // With a polynomial preconditioner, also the Gershgorin bound max_i sum_j |K_ij| / K_ii of the
  // spectrum of D^-1 K (an upper bound, so the polynomial stays positive on the spectrum).
  // poly: degree of the polynomial preconditioner (the multigrid solve's fallback for PK == 2)
  const int poly = PK >= 1 ? a.poly : 1;
  // the preconditioner in use: 2 multigrid, 1 polynomial, 0 Jacobi. The multigrid solve drops
  // to the polynomial if its FP32 V-cycle stops being positive definite (r.z <= 0 or p.K p <= 0:
  // designs whose conditioning is beyond the V-cycle's FP32 arithmetic, e.g. loads on void)
  // (an instance of a batched multigrid launch whose mesh is too small to coarsen, mg.L < 2, runs
  // the polynomial from the start)
  const bool mg_on = PK == 2 && a.mg.L >= 2;
  int mode = mg_on ? 2 : (poly > 1 ? 1 : 0);
  const bool f32pre = mode != 0;  // an FP32 preconditioner on an FP32 copy of the stencil
  if (threadIdx.x == 0) sh_fallback = 0;
  double gmax = 0.0;
  for_owned([&](int i, int j, int k, long long n) {
    assemble_node<DIM>(g, a.ke, a.rho, i, j, k, n, a.C, f32pre ? a.C32 : nullptr);
    const int centre = DIM == 2 ? 4 : 13;
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      const double d = a.C[(long long)((centre * DIM + r) * DIM + r) * g.nnodes + n];
      a.dinv[DIM * n + r] = 1.0 / d;
      if (f32pre) {
        a.dinv32[DIM * n + r] = (float)(1.0 / d);
        double rs = 0.0;
        for (int q = 0; q < StencilGeom<DIM>::NB * DIM; ++q) rs += fabs(a.C[(long long)(r * DIM + (q / DIM) * DIM * DIM + q % DIM) * g.nnodes + n]);
        gmax = fmax(gmax, rs / d);
      }
    }
  });
  if (f32pre) {
    for (int o = 16; o; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if (lane == 0) red[warp] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double bm = 0.0;
      for (int q = 0; q < nwarps; ++q) bm = fmax(bm, red[q]);
      if (mg_on)
        a.mg.lmax[rank] = bm;  // level 0 (an instance without levels has no mg.lmax)
      else
        *P(0, 0) = bm;
    }
  }
  if (!sync_reduce(0)) return;
  if constexpr (PK == 2) {
    if (mg_on && !mg_setup()) return;
  }
  if (poly > 1) {
    // (the multigrid solve keeps these for its fallback; its level-0 bound is in mg.lmax)
    // Chebyshev iteration for D^-1 K z = D^-1 r on [lmax / ratio, lmax], from z = 0, poly steps:
    // z_0 = b / theta, then d_j = c1_j d_{j-1} + c2_j res_{j-1}, z_j = z_{j-1} + d_j, with
    // rho_0 = 1 / sigma, rho_j = 1 / (2 sigma - rho_{j-1}), c1_j = rho_j rho_{j-1},
    // c2_j = 2 rho_j / delta (theta, delta: centre and half-width of the interval).
    if (threadIdx.x == 0) {
      const double* bpart = mg_on ? a.mg.lmax : part + (size_t)((bar & 1) * P2_SLOTS * m) * G;
      double lmax = 0.0;
      for (unsigned q = 0; q < G; ++q) lmax = fmax(lmax, bpart[q]);
      if (!(lmax > 0.0) || !isfinite(lmax)) lmax = 1.0;
      lmax *= 1.001;  // margin for the FP32 rounding of the stencil the polynomial applies
      const double lmin = lmax / a.cheb_ratio;
      const double th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin), sigma = th / de;
      sh_itheta = 1.0 / th;
      double ro = 1.0 / sigma;
      for (int j = 1; j < poly; ++j) {
        const double rn = 1.0 / (2.0 * sigma - ro);
        sh_c1[j] = rn * ro;
        sh_c2[j] = 2.0 * rn / de;
        ro = rn;
      }
    }
    __syncthreads();
  }

  // gamma = r.z and r.r of the last phase U, per thread, until phase W reduces them
  double accg[P2_MAX_COLS], accr[P2_MAX_COLS];

  // Polynomial preconditioner z = p(D^-1 K) D^-1 r (poly > 1), r complete for the owned nodes,
  // evaluated in FP32 (a preconditioner needs no FP64 accuracy, and GB300 runs FP32 at 64x the
  // FP64 rate): poly Chebyshev steps, of which the last poly - 1 apply the FP32 stencil to the
  // previous direction. Step 0 stores b = D^-1 r as the residual, so every step updates
  // res -= D^-1 K t. Each direction is published to the neighbouring CTAs with the release
  // flags and read through their halo, in alternating buffers: a CTA can only overwrite a
  // buffer after every neighbour has published the next step, i.e. has finished reading it.
  // The last step converts z to FP64 and accumulates the per-thread r.z into accg; z itself is
  // published by the caller. all_cols: every column (the true residual, whose convergence
  // flags are not set yet), else the open ones.
  auto precond = [&](bool all_cols) -> bool {
    const float it = (float)sh_itheta;
    for (int c = 0; c < m; ++c) {
      if (!all_cols && sh_done[c]) continue;
      const long long o0 = (long long)c * N;
      for_owned([&](int i, int j, int k, long long n) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const long long dof = DIM * n + d, o = o0 + dof;
          const float b = __ldca(a.dinv32 + dof) * (float)a.r[o];
          const float zv = b * it;
          a.res[o] = b;
          a.t0[o] = zv;
          a.z32[o] = zv;
        }
      });
    }
    publish_z();
    for (int c = 0; c < m; ++c) accg[c] = 0.0;
    for (int st = 1; st < poly; ++st) {
      if (!wait_z()) return false;
      const float* tin = (st & 1) ? a.t0 : a.t1;
      float* tout = (st & 1) ? a.t1 : a.t0;
      const bool last = st == poly - 1;
      const float c1 = (float)sh_c1[st], c2 = (float)sh_c2[st];
      for (int c = 0; c < m; ++c) {
        if (!all_cols && sh_done[c]) continue;
        const long long o0 = (long long)c * N;
        double ag = 0.0;
        for_owned([&](int i, int j, int k, long long n) {
          float y[DIM], tn[DIM];
          stencil_apply32<DIM>(g, a.C32, tin + o0, i, j, k, n, y, tn);
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const long long dof = DIM * n + d, o = o0 + dof;
            const float rs = fmaf(-__ldca(a.dinv32 + dof), y[d], a.res[o]);
            const float dv = fmaf(c1, tn[d], c2 * rs);
            const float zv = a.z32[o] + dv;
            if (last) {
              const double zd = (double)zv;
              a.z[o] = zd;
              ag = fma(a.r[o], zd, ag);
            } else {
              a.z32[o] = zv;
              tout[o] = dv;
              a.res[o] = rs;
            }
          }
        });
        if (last) accg[c] = ag;
      }
      if (!last) publish_z();
    }
    return true;
  };

  // --- multigrid V-cycle z = M r (PK == 2) ---------------------------------------------------
  // Levels 0 .. ls - 1 are split over all G CTAs like level 0 (units of 32 nodes of an x-row);
  // every step that reads neighbouring nodes first waits for the CTAs that own them to publish
  // the previous step (per-CTA release flags, as the z halo of phase W). Levels ls .. L - 1
  // (small) run on CTA 0 alone with block barriers. Every vector slot is written once per
  // V-cycle, and V-cycles are separated by the CG's grid barrier, so no step overwrites data a
  // slower neighbour still reads.
  auto wait_seq = [&](long long lo, long long hi, unsigned long long seq) -> bool {
    if (threadIdx.x == 0) s_okw = 1;
    __syncthreads();
    for (long long q = lo + threadIdx.x; q <= hi; q += blockDim.x) {
      if (q == (long long)rank) continue;
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> f(a.zflag[q]);
      const long long t0 = clock64();
      while (f.load(cuda::memory_order_acquire) < seq) {
        if (*(volatile int*)&gb->abort) {
          s_okw = 0;
          break;
        }
        if (clock64() - t0 > a.wait_cycles) {
          atomicCAS(&gs->status, 0, (int)TOPO_ERR_TIMEOUT);
          atomicExch(&gb->abort, 1);
          s_okw = 0;
          break;
        }
      }
    }
    __syncthreads();
    return s_okw != 0;
  };
  auto for_lv = [&](int l, bool single, auto fn) {
    const MgLevel& Lv = a.mg.lv[l];
    long long lo = 0, hi = Lv.nunits;
    if (single) {
      if (rank != 0) return;
    } else {
      lo = Lv.nunits * rank / G;
      hi = Lv.nunits * (rank + 1) / G;
    }
    const int ux = (Lv.nnx + 31) / 32;
    for (long long u = lo + warp; u < hi; u += nwarps) {
      const int i = (int)(u % ux) * 32 + lane;
      const long long r = u / ux;
      const int j = (int)(r % Lv.nny), k = (int)(r / Lv.nny);
      if (i >= Lv.nnx) continue;
      fn(i, j, k, i + (long long)Lv.nnx * (j + (long long)Lv.nny * k));
    }
  };
  // vectors of the levels run by CTA 0 (ls and coarser) live in its dynamic shared memory
  extern __shared__ __align__(16) unsigned char mg_tail_dyn[];
  float* const tail_s = reinterpret_cast<float*>(mg_tail_dyn);
  auto in_tail = [&](int l) -> bool { return PK == 2 && l >= a.mg.ls; };
  auto mgv_g = [&](int l, int slot, int c) -> float* {  // the global copy
    const MgLevel& Lv = a.mg.lv[l];
    return Lv.v + ((size_t)slot * m + c) * Lv.ndof;
  };
  auto mgv = [&](int l, int slot, int c) -> float* {
    const MgLevel& Lv = a.mg.lv[l];
    if (in_tail(l) && rank == 0) return tail_s + a.mg.tail_off[l] + ((size_t)slot * m + c) * Lv.ndof;
    return mgv_g(l, slot, c);
  };
  auto ldv = [&](int l, const float* p) -> float { return in_tail(l) ? *p : __ldcg(p); };
  auto apply_lv = [&](int l, const Grid& gl, const float* C32, const float* v, int i, int j, int k, long long n,
                      float* y, float* own) {
    if (in_tail(l))
      stencil_apply32<DIM, true>(gl, C32, v, i, j, k, n, y, own);
    else
      stencil_apply32<DIM, false>(gl, C32, v, i, j, k, n, y, own);
  };
  auto colskip = [&](bool all_cols, int c) -> bool { return !all_cols && sh_done[c]; };
  // b at coarse node (I, J, K) of level l = P^T r of level l - 1 (its residual slot). The 3^d
  // fine support positions are unrolled with predicates, so all loads are issued at once.
  auto restrict_node = [&](int l, const float* src, int I, int J, int K, float* out) {
    const MgLevel& F = a.mg.lv[l - 1];
    constexpr int NZ = DIM == 3 ? 3 : 1;
    const int px = mg_pos(I, F.nnx), py = mg_pos(J, F.nny), pz = DIM == 3 ? mg_pos(K, F.nnz) : 0;
#pragma unroll
    for (int q = 0; q < DIM; ++q) out[q] = 0.f;
#pragma unroll 1
    for (int dz = 0; dz < NZ; ++dz) {  // one plane of the support at a time (register budget)
      const int iz = DIM == 3 ? pz + dz - 1 : 0;
      const float wz = DIM == 3 ? ((iz >= 0 && iz < F.nnz) ? mg_w1(iz, K, F.nnz) : 0.f) : 1.f;
      if (wz == 0.f) continue;
      float v[3][3][DIM], wt[3][3];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int ix = px + dx - 1, iy = py + dy - 1;
          const bool in = ix >= 0 && ix < F.nnx && iy >= 0 && iy < F.nny;
          const float w = in ? mg_w1(ix, I, F.nnx) * mg_w1(iy, J, F.nny) * wz : 0.f;
          wt[dy][dx] = w;
          const long long ni = w != 0.f ? ix + (long long)F.nnx * (iy + (long long)F.nny * iz) : 0;
#pragma unroll
          for (int q = 0; q < DIM; ++q) v[dy][dx][q] = w != 0.f ? ldv(l - 1, src + DIM * ni + q) : 0.f;
        }
#pragma unroll
      for (int q = 0; q < DIM; ++q) {
        float t = out[q];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) t = fmaf(wt[dy][dx], v[dy][dx][q], t);
        out[q] = t;
      }
    }
  };
  // (P x_c) at fine node (i, j, k) of level l from level l + 1: parents in [i/2, i/2 + 1] per
  // direction, unrolled the same way
  auto prolong_node = [&](int l, const float* src, int i, int j, int k, float* out) {
    const MgLevel& F = a.mg.lv[l];
    const MgLevel& Cc = a.mg.lv[l + 1];
    constexpr int NZ = DIM == 3 ? 2 : 1;
    float v[NZ][2][2][DIM], wt[NZ][2][2];
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int Ix = i / 2 + dx, Jy = j / 2 + dy, Kz = DIM == 3 ? k / 2 + dz : 0;
          const bool in = Ix < Cc.nnx && Jy < Cc.nny && Kz < Cc.nnz;
          const float w = in ? mg_w1(i, Ix, F.nnx) * mg_w1(j, Jy, F.nny) * (DIM == 3 ? mg_w1(k, Kz, F.nnz) : 1.f) : 0.f;
          wt[dz][dy][dx] = w;
          const long long mc = w != 0.f ? Ix + (long long)Cc.nnx * (Jy + (long long)Cc.nny * Kz) : 0;
#pragma unroll
          for (int q = 0; q < DIM; ++q) v[dz][dy][dx][q] = w != 0.f ? ldv(l, src + DIM * mc + q) : 0.f;
        }
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      float t = 0.f;
#pragma unroll
      for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) t = fmaf(wt[dz][dy][dx], v[dz][dy][dx][q], t);
      out[q] = t;
    }
  };
  auto fixed_lv = [&](int l, long long dof) -> bool {
    return l == 0 ? is_fixed(g, dof) : __ldcg(a.mg.lv[l].fix + dof) != 0;
  };
  // right-hand side of level l at a DOF: the CG residual (level 0) or the restricted residual
  auto rhs = [&](int l, int c, long long dof) -> float {
    return l == 0 ? (float)a.r[(size_t)c * N + dof] : ldv(l, mgv(l, mg_slot_b(a.mg.deg), c) + dof);
  };
  // pre-smoothing step 0 (from zero): x_0 = D^-1 b / theta; for l >= 1 b is restricted first
  auto mg_pre0 = [&](int l, bool single, bool all_cols) {
    const MgLevel& Lv = a.mg.lv[l];
    const float ith = mg_ith[l];
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      float* x0 = mgv(l, 0, c);
      float* bb = mgv(l, mg_slot_b(a.mg.deg), c);
      const float* r2f = l ? mgv(l - 1, mg_slot_res(a.mg.deg), c) : nullptr;
      for_lv(l, single, [&](int i, int j, int k, long long n) {
        float b[DIM];
        if (l == 0) {
#pragma unroll
          for (int q = 0; q < DIM; ++q) b[q] = (float)a.r[(size_t)c * N + DIM * n + q];
        } else {
          restrict_node(l, r2f, i, j, k, b);
#pragma unroll
          for (int q = 0; q < DIM; ++q) bb[DIM * n + q] = b[q];
        }
#pragma unroll
        for (int q = 0; q < DIM; ++q) x0[DIM * n + q] = __ldca(Lv.dinv + DIM * n + q) * b[q] * ith;
      });
    }
  };
  // pre-smoothing step jj >= 1: x_jj = x_{jj-1} + c1 (x_{jj-1} - x_{jj-2}) + c2 D^-1 (b - K x_{jj-1})
  auto mg_pre = [&](int l, int jj, bool single, bool all_cols) {
    const MgLevel& Lv = a.mg.lv[l];
    const Grid gl = mg_grid(g, Lv);
    const float c1 = mg_c1[l][jj], c2 = mg_c2[l][jj];
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      const float* xin = mgv(l, jj - 1, c);
      const float* xpp = jj >= 2 ? mgv(l, jj - 2, c) : nullptr;
      float* xout = mgv(l, jj, c);
      for_lv(l, single, [&](int i, int j, int k, long long n) {
        float y[DIM], own[DIM];
        apply_lv(l, gl, Lv.C32, xin, i, j, k, n, y, own);
#pragma unroll
        for (int q = 0; q < DIM; ++q) {
          const long long dof = DIM * n + q;
          const float prev = xpp ? ldv(l, xpp + dof) : 0.f;
          const float d = fmaf(c1, own[q] - prev, c2 * __ldca(Lv.dinv + dof) * (rhs(l, c, dof) - y[q]));
          xout[dof] = own[q] + d;
        }
      });
    }
  };
  // residual after pre-smoothing: r = b - K x_{deg-1}
  auto mg_res = [&](int l, bool single, bool all_cols) {
    const MgLevel& Lv = a.mg.lv[l];
    const Grid gl = mg_grid(g, Lv);
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      const float* xin = mgv(l, a.mg.deg - 1, c);
      float* res = mgv(l, mg_slot_res(a.mg.deg), c);
      for_lv(l, single, [&](int i, int j, int k, long long n) {
        float y[DIM], own[DIM];
        apply_lv(l, gl, Lv.C32, xin, i, j, k, n, y, own);
#pragma unroll
        for (int q = 0; q < DIM; ++q) res[DIM * n + q] = rhs(l, c, DIM * n + q) - y[q];
      });
    }
  };
  // coarse correction: y_0 = x_{deg-1} + P x_coarse (no correction on identity rows)
  auto mg_post0 = [&](int l, bool single, bool all_cols) {
    const int deg = a.mg.deg;
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      // level l + 1's result: for l + 1 == ls the global copy CTA 0 leaves for the other CTAs
      const int so = (l + 1 == a.mg.L - 1) ? 0 : mg_slot_post(deg, deg);
      const float* xc = (l + 1 == a.mg.ls) ? mgv_g(l + 1, so, c) : mgv(l + 1, so, c);
      const float* xin = mgv(l, deg - 1, c);
      float* y0 = mgv(l, mg_slot_post(deg, 0), c);
      for_lv(l, single, [&](int i, int j, int k, long long n) {
        float p[DIM];
        prolong_node(l, xc, i, j, k, p);
#pragma unroll
        for (int q = 0; q < DIM; ++q) {
          const long long dof = DIM * n + q;
          y0[dof] = ldv(l, xin + dof) + (fixed_lv(l, dof) ? 0.f : p[q]);
        }
      });
    }
  };
  // post-smoothing step jj (0 .. deg-1): y_{jj+1} from y_jj (and y_{jj-1}); the last step of
  // level 0 writes z (FP64) and accumulates r.z per thread
  auto mg_post = [&](int l, int jj, bool single, bool all_cols) {
    const MgLevel& Lv = a.mg.lv[l];
    const Grid gl = mg_grid(g, Lv);
    const int deg = a.mg.deg;
    const float ith = mg_ith[l];
    const float c1 = jj ? mg_c1[l][jj] : 0.f, c2 = jj ? mg_c2[l][jj] : 0.f;
    const bool last0 = l == 0 && jj == deg - 1;
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      const float* yin = mgv(l, mg_slot_post(deg, jj), c);
      const float* yprev = jj ? mgv(l, mg_slot_post(deg, jj - 1), c) : nullptr;
      float* yout = last0 ? nullptr : mgv(l, mg_slot_post(deg, jj + 1), c);
      double ag = 0.0;
      for_lv(l, single, [&](int i, int j, int k, long long n) {
        float y[DIM], own[DIM];
        apply_lv(l, gl, Lv.C32, yin, i, j, k, n, y, own);
#pragma unroll
        for (int q = 0; q < DIM; ++q) {
          const long long dof = DIM * n + q;
          const float dr = __ldca(Lv.dinv + dof) * (rhs(l, c, dof) - y[q]);
          const float d = jj ? fmaf(c1, own[q] - ldv(l, yprev + dof), c2 * dr) : dr * ith;
          const float out = own[q] + d;
          if (last0) {
            const double zd = (double)out;
            const size_t o = (size_t)c * N + dof;
            a.z[o] = zd;
            ag = fma(a.r[o], zd, ag);
          } else {
            yout[dof] = out;
          }
        }
      });
      if (last0) accg[c] = ag;
    }
  };
  // coarsest level on CTA 0: b = P^T r (restricted), x = A^-1 b (dense, one warp per row)
  auto mg_coarsest = [&](bool all_cols) {
    const int l = a.mg.L - 1, nc = a.mg.nc, deg = a.mg.deg;
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      float* bc = mgv(l, mg_slot_b(deg), c);
      const float* r2f = mgv(l - 1, mg_slot_res(deg), c);
      for_lv(l, true, [&](int i, int j, int k, long long n) {
        float b[DIM];
        restrict_node(l, r2f, i, j, k, b);
#pragma unroll
        for (int q = 0; q < DIM; ++q) bc[DIM * n + q] = b[q];
      });
    }
    __syncthreads();
    for (int c = 0; c < m; ++c) {
      if (colskip(all_cols, c)) continue;
      const float* bc = mgv(l, mg_slot_b(deg), c);
      float* xs = mgv(l, 0, c);
      for (int row = warp; row < nc; row += nwarps) {
        float t = 0.f;
#pragma unroll 5
        for (int q = lane; q < nc; q += 32) t = fmaf(__ldca(a.mg.Ainv + (size_t)row * nc + q), bc[q], t);
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) xs[row] = t;
      }
    }
    __syncthreads();
  };
  auto mg_vcycle = [&](bool all_cols) -> bool {
    const int deg = a.mg.deg, L = a.mg.L, ls = a.mg.ls;
    unsigned long long seq_res[MG_MAX_LEVELS], seq_out[MG_MAX_LEVELS];
    for (int c = 0; c < m; ++c) accg[c] = 0.0;
    for (int l = 0; l < ls; ++l) {  // descend (all CTAs)
      if (l >= 1 && !wait_seq(mg_rest[l][0], mg_rest[l][1], seq_res[l - 1])) return false;
      mg_pre0(l, false, all_cols);
      publish_z();
      for (int jj = 1; jj < deg; ++jj) {
        if (!wait_seq(mg_halo[l][0], mg_halo[l][1], zseq)) return false;
        mg_pre(l, jj, false, all_cols);
        publish_z();
      }
      if (!wait_seq(mg_halo[l][0], mg_halo[l][1], zseq)) return false;
      mg_res(l, false, all_cols);
      publish_z();
      seq_res[l] = zseq;
    }
    bool ok = true;
    if (rank == 0) {  // levels ls .. L - 1 on CTA 0
      ok = wait_seq(0, (long long)G - 1, seq_res[ls - 1]);
      if (ok) {
        for (int l = ls; l < L - 1; ++l) {
          mg_pre0(l, true, all_cols);
          __syncthreads();
          for (int jj = 1; jj < deg; ++jj) {
            mg_pre(l, jj, true, all_cols);
            __syncthreads();
          }
          mg_res(l, true, all_cols);
          __syncthreads();
        }
        mg_coarsest(all_cols);
        for (int l = L - 2; l >= ls; --l) {
          mg_post0(l, true, all_cols);
          __syncthreads();
          for (int jj = 0; jj < deg; ++jj) {
            mg_post(l, jj, true, all_cols);
            __syncthreads();
          }
        }
        // level ls's result, from shared memory to its global copy, for level ls - 1
        const int so = (ls == L - 1) ? 0 : mg_slot_post(deg, deg);
        for (int c = 0; c < m; ++c) {
          if (colskip(all_cols, c)) continue;
          const float* src = mgv(ls, so, c);
          float* dst = mgv_g(ls, so, c);
          for (long long t = threadIdx.x; t < a.mg.lv[ls].ndof; t += blockDim.x) dst[t] = src[t];
        }
      }
    }
    if (!ok) return false;
    publish_z();
    const unsigned long long seq_tail = zseq;
    for (int l = ls - 1; l >= 0; --l) {  // ascend (all CTAs)
      if (!wait_seq(mg_prol[l][0], mg_prol[l][1], l + 1 == ls ? seq_tail : seq_out[l + 1])) return false;
      mg_post0(l, false, all_cols);
      publish_z();
      for (int jj = 0; jj < deg; ++jj) {
        if (!wait_seq(mg_halo[l][0], mg_halo[l][1], zseq)) return false;
        mg_post(l, jj, false, all_cols);
        publish_z();
      }
      seq_out[l] = zseq;
    }
    return true;
  };

  // --- true residual r = f - K x, z = D^-1 r -----------------------------------------------
  // r, z for owned nodes (x = caller's U, Dirichlet entries zeroed), partial gamma, r.r, f.f,
  // (|K||x|)^2; one barrier (it also publishes z to every CTA).
  auto true_residual = [&](bool first) -> bool {
    double acc[4][P2_MAX_COLS];
    for (int c = 0; c < m; ++c) acc[0][c] = acc[1][c] = acc[2][c] = acc[3][c] = 0.0;
    for (int c = 0; c < m; ++c) {
      double* x = a.U + c * a.ld;
      const double* f = a.F + c * a.ld;
      double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;  // register accumulators
      for_owned([&](int i, int j, int k, long long n) {
        double y[DIM], yabs[DIM];
        stencil_apply_abs<DIM>(g, a.C, x, i, j, k, n, y, yabs);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const long long dof = DIM * n + d;
          double rv = 0.0;
          if (!is_fixed(g, dof)) {
            const double fv = f[dof];
            rv = fv - y[d];
            t1 = fma(rv, rv, t1);
            t2 = fma(fv, fv, t2);
            t3 = fma(yabs[d], yabs[d], t3);
          } else if (first) {
            x[dof] = 0.0;  // Dirichlet entries of the solution are zero (their columns are zero)
          }
          a.r[c * N + dof] = rv;
          if (mode == 0) {
            const double zv = __ldcg(a.dinv + dof) * rv;
            a.z[c * N + dof] = zv;
            t0 = fma(rv, zv, t0);
          }
        }
      });
      acc[0][c] = t0;
      acc[1][c] = t1;
      acc[2][c] = t2;
      acc[3][c] = t3;
    }
    if (mode != 0) {  // z = p(D^-1 K) D^-1 r or the V-cycle: their halo steps need every CTA's r
      if (!(mode == 2 ? mg_vcycle(true) : precond(true))) return false;
      for (int c = 0; c < m; ++c) acc[0][c] = accg[c];
    }
    for (int c = 0; c < m; ++c)
      for (int q = 0; q < 4; ++q) {
        const double t = block_sum(acc[q][c], red);
        if (threadIdx.x == 0) *P(q, c) = t;
      }
    if (!sync_reduce(4 * m)) return false;
    if (threadIdx.x == 0) {
      for (int c = 0; c < m; ++c) {
        sh_gamma[c] = R(0, c);
        sh_rr[c] = R(1, c);
        if (first) sh_ff[c] = R(2, c);
        // no FP64 evaluation of f - K x can be trusted below ~eps |K||x|: accept the larger
        // of rtol and 2 eps |K||x| / |f|
        const double fl = 2.0 * 2.220446049250313e-16;
        sh_floor2[c] = fl * fl * R(3, c);
        sh_tol2[c] = fmax(a.rtol * a.rtol * sh_ff[c], sh_floor2[c]);
        sh_done[c] = sh_rr[c] <= sh_tol2[c];
      }
    }
    __syncthreads();
    return true;
  };


  // Phase W: w = K z for owned nodes and partial delta = w.z; one grid barrier reduces delta
  // together with gamma and r.r of the preceding phase U (Chronopoulos-Gear: one reduction
  // per iteration). Then beta = gamma_new / gamma, the convergence test on r.r, and
  // alpha = gamma / den with den = delta - beta gamma / alpha_old = delta - beta^2 den_old
  // (alpha_old = gamma_old / den_old; two FP64 divisions per step). Restart: beta = 0,
  // den = delta; gamma and r.r come from the true residual.
  //
  // With the polynomial preconditioner (poly > 1), which is symmetric only up to its FP32
  // rounding, the recurrence for den assumes a symmetry the preconditioner lacks, and den can
  // turn negative. So the same reduction also carries e = z.s_old and f = p_old.w, and
  // den = p.K p for the new p = z + beta p_old is formed directly, exact for any preconditioner:
  //   den = delta + beta (e + f) + beta^2 den_old (> 0: K is SPD).
  // beta stays gamma_new / gamma (measured at 600x200: 1,432 iterations at degree 8, against
  // 1,658 with the flexible choice -alpha_old e / gamma_old).
  auto phase_w = [&](bool restart) -> bool {
    if (!restart && !wait_z()) return false;
    const bool flex = f32pre;
    double acc[P2_MAX_COLS], acce[P2_MAX_COLS], accf[P2_MAX_COLS];  // per column
    for (int c = 0; c < m; ++c) acc[c] = acce[c] = accf[c] = 0.0;
    for (int c = 0; c < m; ++c) {
      if (sh_done[c]) continue;
      const double* zc = a.z + c * N;
      double ad = 0.0, ae = 0.0, af = 0.0;  // register accumulators
      for_owned([&](int i, int j, int k, long long n) {
        double y[DIM], zn[DIM];
        stencil_apply<DIM>(g, a.C, zc, i, j, k, n, y, zn);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const long long dof = DIM * n + d;
          a.w[c * N + dof] = y[d];
          ad = fma(y[d], zn[d], ad);
          if (flex && !restart) {  // p and s of the previous iteration (stale on a restart)
            ae = fma(zn[d], a.s[c * N + dof], ae);
            af = fma(a.p[c * N + dof], y[d], af);
          }
        }
      });
      acc[c] = ad;
      acce[c] = ae;
      accf[c] = af;
    }
    for (int c = 0; c < m; ++c) {
      double t0 = acc[c], t1 = restart ? 0.0 : accg[c], t2 = restart ? 0.0 : accr[c];
      block_sum3(t0, t1, t2, red);
      if (threadIdx.x == 0) {
        *P(0, c) = t0;
        *P(1, c) = t1;
        *P(2, c) = t2;
      }
      if (flex) {
        double t3 = acce[c], t4 = accf[c], t5 = 0.0;
        block_sum3(t3, t4, t5, red);
        if (threadIdx.x == 0) {
          *P(3, c) = t3;
          *P(4, c) = t4;
        }
      }
    }
    if (!sync_reduce((flex ? 5 : 3) * m)) return false;
    if (threadIdx.x == 0) {
      for (int c = 0; c < m; ++c) {
        if (sh_done[c]) continue;
        if (flex) {
          const double delta = R(0, c);
          if (restart) {
            sh_beta[c] = 0.0;
            sh_den[c] = delta;
          } else {
            const double gnew = R(1, c), e = R(3, c), f = R(4, c);
            sh_beta[c] = gnew / sh_gamma[c];
            sh_gamma[c] = gnew;
            sh_rr[c] = R(2, c);
            if (sh_rr[c] <= sh_tol2[c]) {
              sh_done[c] = 1;
              continue;
            }
            const double be = sh_beta[c];
            sh_den[c] = delta + be * (e + f) + be * be * sh_den[c];
          }
          sh_alpha[c] = sh_gamma[c] / sh_den[c];
          if (!(sh_alpha[c] > 0.0) || !isfinite(sh_alpha[c])) {
            if (PK == 2 && mode == 2) {
              sh_fallback = 1;  // restart from the true residual with the polynomial
            } else {
              set_status(&gs->status, TOPO_ERR_NOT_SPD);
              sh_done[c] = 1;
            }
          }
          continue;
        }
        if (!restart) {
          const double gnew = R(1, c);
          sh_beta[c] = gnew / sh_gamma[c];
          sh_gamma[c] = gnew;
          sh_rr[c] = R(2, c);
          if (sh_rr[c] <= sh_tol2[c]) {
            sh_done[c] = 1;
            continue;
          }
        }
        const double delta = R(0, c);
        if (restart) {
          sh_beta[c] = 0.0;
          sh_den[c] = delta;
        } else {
          sh_den[c] = delta - sh_beta[c] * sh_beta[c] * sh_den[c];
        }
        sh_alpha[c] = sh_gamma[c] / sh_den[c];
        if (!(sh_alpha[c] > 0.0) || !isfinite(sh_alpha[c])) {
          set_status(&gs->status, TOPO_ERR_NOT_SPD);
          sh_done[c] = 1;
        }
      }
    }
    __syncthreads();
    return true;
  };

  // Phase U: p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s, z = D^-1 r (Jacobi) or
  // the polynomial preconditioner; per-thread gamma = r.z and r.r (reduced by the next phase W);
  // then z is published to the neighbours.
  auto phase_u = [&](bool restart) -> bool {
    const bool jac = mode == 0;
    for (int c = 0; c < m; ++c) accg[c] = accr[c] = 0.0;
    for (int c = 0; c < m; ++c) {
      if (sh_done[c]) continue;
      const double al = sh_alpha[c], be = restart ? 0.0 : sh_beta[c];
      double* x = a.U + c * a.ld;
      double ag = 0.0, ar = 0.0;  // register accumulators of r.z and r.r
      for_owned([&](int i, int j, int k, long long n) {
        if constexpr (DIM == 2) {
          // the node's two DOFs as 16-byte accesses (scratch vectors are 16-byte aligned; x, the
          // caller's array, may have an odd leading dimension and stays scalar)
          const long long o2 = (c * N) / 2 + n;
          const double2 zz = reinterpret_cast<const double2*>(a.z)[o2];
          const double2 ww = reinterpret_cast<const double2*>(a.w)[o2];
          const double2 rr = reinterpret_cast<const double2*>(a.r)[o2];
          const double2 di = __ldcg(reinterpret_cast<const double2*>(a.dinv) + n);
          double2 pv, sv;
          if (restart) {  // p and s hold stale (possibly non-finite) data: take z and w exactly
            pv = zz;
            sv = ww;
          } else {
            const double2 pp = reinterpret_cast<const double2*>(a.p)[o2];
            const double2 ss = reinterpret_cast<const double2*>(a.s)[o2];
            pv = make_double2(fma(be, pp.x, zz.x), fma(be, pp.y, zz.y));
            sv = make_double2(fma(be, ss.x, ww.x), fma(be, ss.y, ww.y));
          }
          reinterpret_cast<double2*>(a.p)[o2] = pv;
          reinterpret_cast<double2*>(a.s)[o2] = sv;
          x[2 * n] = fma(al, pv.x, x[2 * n]);
          x[2 * n + 1] = fma(al, pv.y, x[2 * n + 1]);
          const double2 rv = make_double2(fma(-al, sv.x, rr.x), fma(-al, sv.y, rr.y));
          reinterpret_cast<double2*>(a.r)[o2] = rv;
          if (jac) {
            const double2 zv = make_double2(di.x * rv.x, di.y * rv.y);
            reinterpret_cast<double2*>(a.z)[o2] = zv;
            ag = fma(rv.x, zv.x, ag);
            ag = fma(rv.y, zv.y, ag);
          }
          ar = fma(rv.x, rv.x, ar);
          ar = fma(rv.y, rv.y, ar);
        } else {
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const long long dof = DIM * n + d, o = c * N + dof;
            // on a restart p and s hold stale (possibly non-finite) data: take z and w exactly
            const double pv = restart ? a.z[o] : fma(be, a.p[o], a.z[o]);
            const double sv = restart ? a.w[o] : fma(be, a.s[o], a.w[o]);
            a.p[o] = pv;
            a.s[o] = sv;
            x[dof] = fma(al, pv, x[dof]);
            const double rv = fma(-al, sv, a.r[o]);
            a.r[o] = rv;
            if (jac) {
              const double zv = __ldcg(a.dinv + dof) * rv;
              a.z[o] = zv;
              ag = fma(rv, zv, ag);
            }
            ar = fma(rv, rv, ar);
          }
        }
      });
      accg[c] = ag;
      accr[c] = ar;
    }
    if constexpr (PK == 2) {
      if (mode == 2) return mg_vcycle(false);  // publishes z as its last step
      if (!precond(false)) return false;
      publish_z();
      return true;
    } else {
      if (!jac && !precond(false)) return false;
      publish_z();
      return true;
    }
  };

  int iters = 0;
  if (!true_residual(true)) return;
  for (int rep = 0; rep < 50; ++rep) {
    bool all = true;
    for (int c = 0; c < m; ++c) all = all && sh_done[c];
    if (all || iters >= a.maxit) break;
    bool restart = true;
    // multigrid stagnation: a V-cycle in FP32 cannot resolve every stiffness contrast (a stiff
    // island held only by void elements); when r.r of a column still in progress has not fallen
    // to a quarter within MG_STALL_ITERS iterations, the solve continues with the polynomial.
    // Every CTA tests the same reduced values, so all switch at the same iteration.
    int chk_it = iters;
    if (PK == 2 && mode == 2) {
      __syncthreads();
      if (threadIdx.x == 0)
        for (int c = 0; c < m; ++c) sh_rrchk[c] = sh_rr[c];
      __syncthreads();
    }
    while (true) {
      if (!phase_w(restart)) return;
      if (PK == 2 && mode == 2 && sh_fallback) {
        mode = 1;  // every CTA reduced the same values: all switch here
        break;
      }
      if (PK == 2 && mode == 2 && iters - chk_it >= MG_STALL_ITERS) {
        bool stalled = false;
        for (int c = 0; c < m; ++c) stalled = stalled || (!sh_done[c] && sh_rr[c] > 0.25 * sh_rrchk[c]);
        __syncthreads();
        if (threadIdx.x == 0)
          for (int c = 0; c < m; ++c) sh_rrchk[c] = sh_rr[c];
        __syncthreads();
        chk_it = iters;
        if (stalled) {
          mode = 1;
          break;
        }
      }
      bool any = false;
      for (int c = 0; c < m; ++c) any = any || !sh_done[c];
      if (!any || iters >= a.maxit) break;
      if (!phase_u(restart)) return;
      restart = false;
      ++iters;
    }
    // residual replacement: restart from the true residual (the last phase W's barrier has
    // made every CTA's x visible)
    if (!true_residual(false)) return;
  }
  if (rank == 0 && threadIdx.x == 0) {
    double worst = 0.0, wfloor = 0.0;
    bool conv = true;
    for (int c = 0; c < m; ++c) {
      worst = fmax(worst, sh_ff[c] > 0 ? sh_rr[c] / sh_ff[c] : 0.0);
      wfloor = fmax(wfloor, sh_ff[c] > 0 ? sh_floor2[c] / sh_ff[c] : 0.0);
      conv = conv && (sh_rr[c] <= sh_tol2[c]);
    }
    a.info_rr[1] = wfloor;
    a.info[0] = iters;
    a.info[1] = 0;
    a.info[2] = conv ? 0 : TOPO_ERR_NOT_CONVERGED;
    a.info[3] = (mg_on && mode != 2) ? 1 : 0;  // multigrid fell back to the polynomial
    a.info_rr[0] = worst;
  }
}

template <int DIM>
__global__ void __launch_bounds__(P2_THREADS_SOLO, 1) pcg2_kernel(const __grid_constant__ Pcg2Args<DIM> a) {
  pcg2_body<DIM, 1>(a, gridDim.x, blockIdx.x, a.gb);
}

// The same solver with the multigrid V-cycle as its preconditioner.
template <int DIM>
__global__ void __launch_bounds__(P2_THREADS_SOLO, 1) pcg2_mg_kernel(const __grid_constant__ Pcg2Args<DIM> a) {
  pcg2_body<DIM, 2>(a, gridDim.x, blockIdx.x, a.gb);
}

// Batched form: CTA b works on instance cta_inst[b] as number cta_rank[b] of that instance's
// group of grp_size[instance] CTAs; every instance has its own barrier state and progresses on
// its own (no barrier spans instances).
template <int DIM>
__global__ void __launch_bounds__(P2_THREADS, 4) pcg2_batch_kernel(const Pcg2Args<DIM>* __restrict__ args,
                                                                const int* __restrict__ cta_inst,
                                                                const int* __restrict__ cta_rank,
                                                                const int* __restrict__ grp_size) {
  const int inst = cta_inst[blockIdx.x];
  pcg2_body<DIM, 0>(args[inst], (unsigned)grp_size[inst], (unsigned)cta_rank[blockIdx.x], args[inst].gb);
}
template __global__ void pcg2_batch_kernel<2>(const Pcg2Args<2>*, const int*, const int*, const int*);


template <int DIM>
topo_status build_pcg2_args(topo_ctx* c, const double* rho, const double* F, double* U, int m, int ld, double rtol,
                            int maxit, int G, Pcg2Args<DIM>* out, GridSync* status, int poly, bool mg) {
  const Grid& g = c->g;
  const long long N = g.ndof;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oC = take((size_t)StencilGeom<DIM>::NC * g.nnodes * 8), oD = take(N * 8);
  size_t ov[5];
  for (int t = 0; t < 5; ++t) ov[t] = take(N * m * 8);
  size_t oC32 = 0, oD32 = 0, of[4] = {0, 0, 0, 0};
  if (poly > 1 || mg) {  // FP32 stencil and D^-1 (the FP32 preconditioners)
    oC32 = take((size_t)StencilGeom<DIM>::NC * g.nnodes * 4);
    oD32 = take(N * 4);
  }
  if (poly > 1 || mg)  // the four vectors of the polynomial preconditioner (multigrid: its fallback)
    for (int t = 0; t < 4; ++t) of[t] = take(N * m * 4);
  // multigrid levels: sizes, then FP64/FP32 stencils, D^-1, identity-row flags and V-cycle
  // vectors of every level, the dense coarsest operator and its inverse
  MgArgs mga = {};
  size_t omg[MG_MAX_LEVELS][5] = {};
  size_t oAi = 0, olm = 0, ook = 0;
  if (mg) {
    const int deg = c->mg_deg;
    int nn[3] = {g.nnx, g.nny, g.nnz};
    int L = 0;
    while (true) {
      MgLevel& Lv = mga.lv[L];
      Lv.nnx = nn[0];
      Lv.nny = nn[1];
      Lv.nnz = nn[2];
      Lv.nnodes = (long long)nn[0] * nn[1] * nn[2];
      Lv.ndof = DIM * Lv.nnodes;
      Lv.nunits = (long long)((nn[0] + 31) / 32) * nn[1] * nn[2];
      ++L;
      const int nx2 = mg_coarse_n(nn[0]), ny2 = mg_coarse_n(nn[1]), nz2 = DIM == 3 ? mg_coarse_n(nn[2]) : 1;
      const bool shrinks = nx2 < nn[0] || ny2 < nn[1] || nz2 < nn[2];
      if (Lv.ndof <= MG_COARSE_MAX || !shrinks || L == MG_MAX_LEVELS) break;
      nn[0] = nx2;
      nn[1] = ny2;
      nn[2] = nz2;
    }
    mga.L = L;
    mga.deg = deg;
    mga.nc = (int)mga.lv[L - 1].ndof;
    if (L >= 2 && mga.nc <= MG_COARSE_MAX) {
      // Levels ls .. L - 1 run on CTA 0 with their vectors in its shared memory: the first level
      // (never level 0) with at most mg_single_nodes nodes whose vectors, with those of all
      // coarser levels, fit MG_TAIL_BYTES; at least the coarsest level.
      auto tail_floats = [&](int l0) {
        size_t t = 0;
        for (int l = l0; l < L; ++l) t += (((size_t)mg_slots(deg) * m * mga.lv[l].ndof + 3) & ~(size_t)3);
        return t;
      };
      // -1: 1024 nodes in 2D (measured best at 600x200); in 3D only the coarsest level, whose
      // 243-coefficient stencils do not stay in one SM's L1 at coarse sizes
      const long long single = c->mg_single_nodes >= 0 ? c->mg_single_nodes : (DIM == 2 ? 1024 : 0);
      int ls = L - 1;
      for (int l = 1; l < L; ++l)
        if (mga.lv[l].nnodes <= single && tail_floats(l) * 4 <= MG_TAIL_BYTES) {
          ls = l;
          break;
        }
      mga.ls = ls;
      size_t toff = 0;
      for (int l = 0; l < MG_MAX_LEVELS; ++l) mga.tail_off[l] = 0;
      for (int l = ls; l < L; ++l) {
        mga.tail_off[l] = (int)toff;
        toff += ((size_t)mg_slots(deg) * m * mga.lv[l].ndof + 3) & ~(size_t)3;
      }
      mga.tail_floats = (int)toff;
      for (int l = 0; l < L; ++l) {
        const MgLevel& Lv = mga.lv[l];
        if (l > 0) {
          omg[l][0] = take((size_t)StencilGeom<DIM>::NC * Lv.nnodes * 8);
          omg[l][1] = take((size_t)StencilGeom<DIM>::NC * Lv.nnodes * 4);
          omg[l][2] = take((size_t)Lv.ndof * 4);
          omg[l][3] = take((size_t)Lv.ndof);
        }
        omg[l][4] = take((size_t)mg_slots(deg) * m * Lv.ndof * 4);
      }
      oAi = take((size_t)mga.nc * mga.nc * 4);
      olm = take((size_t)MG_MAX_LEVELS * G * 8);
      ook = take(16);
    } else {
      mg = false;  // a mesh too small to coarsen: the polynomial / Jacobi path
      mga.L = 0;
    }
  }

  const size_t opart = take(sizeof(double) * 2 * P2_SLOTS * m * G), oflag = take(sizeof(unsigned long long) * G),
               oinfo = take(64);
  topo_status st = ensure_scratch(c, off);
  if (st) return st;
  char* base = (char*)c->d_scratch;
  Pcg2Args<DIM>& a = *out;
  a.g = g;
  if (DIM == 2)
    memcpy(&a.ke, &c->q4_64, sizeof(a.ke));
  else
    memcpy(&a.ke, &c->h8_64, sizeof(a.ke));
  a.rho = rho;
  a.F = F;
  a.U = U;
  a.ld = ld;
  a.m = m;
  a.N = N;
  a.nunits = (long long)((g.nnx + 31) / 32) * g.nny * g.nnz;
  a.C = (double*)(base + oC);
  a.dinv = (double*)(base + oD);
  double** vecs[5] = {&a.r, &a.z, &a.w, &a.p, &a.s};
  for (int t = 0; t < 5; ++t) *vecs[t] = (double*)(base + ov[t]);
  float** fvecs[4] = {&a.t0, &a.t1, &a.res, &a.z32};
  for (int t = 0; t < 4; ++t) *fvecs[t] = (poly > 1 || mg) ? (float*)(base + of[t]) : nullptr;
  a.C32 = (poly > 1 || mg) ? (float*)(base + oC32) : nullptr;
  a.dinv32 = (poly > 1 || mg) ? (float*)(base + oD32) : nullptr;
  a.poly = poly > 1 ? poly : 1;
  if (mg && a.poly < 2) a.poly = 2;  // the multigrid solve's fallback is a real polynomial
  a.mg = mga;
  if (mg) {
    for (int l = 0; l < mga.L; ++l) {
      MgLevel& Lv = a.mg.lv[l];
      if (l == 0) {
        Lv.C = a.C;
        Lv.C32 = a.C32;
        Lv.dinv = a.dinv32;
        Lv.fix = nullptr;
      } else {
        Lv.C = (double*)(base + omg[l][0]);
        Lv.C32 = (float*)(base + omg[l][1]);
        Lv.dinv = (float*)(base + omg[l][2]);
        Lv.fix = (unsigned char*)(base + omg[l][3]);
      }
      Lv.v = (float*)(base + omg[l][4]);
    }
    a.mg.Ainv = (float*)(base + oAi);
    a.mg.lmax = (double*)(base + olm);
    a.mg.coarse_ok = (int*)(base + ook);
  }
  a.cheb_ratio = 100.0;  // interval [lambda_max / 100, lambda_max]
  a.partial = (double*)(base + opart);
  a.zflag = (unsigned long long*)(base + oflag);
  a.info = (int*)(base + oinfo);
  a.info_rr = (double*)(base + oinfo + 16);
  a.gs = status;
  a.gb = c->d_bar;
  a.rtol = rtol;
  a.maxit = maxit;
  a.wait_cycles = c->wait_cycles;
  return TOPO_OK;
}

cudaError_t launch_pcg2_batch2(unsigned ctas, cudaStream_t stream, const Pcg2Args<2>* args, const int* cta_inst,
                               const int* cta_rank, const int* grp_size) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(P2_THREADS);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pcg2_batch_kernel<2>, args, cta_inst, cta_rank, grp_size);
}

int pcg2_occupancy() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg2_batch_kernel<2>, P2_THREADS, 0);
  return occ;
}

// Degree of the polynomial preconditioner when TOPO_PARAM_PCG_POLY is 0.
static int pcg_poly_auto(int dim) { return dim == 2 ? 8 : 4; }

// One 2D solve staged for a share of at most max_ctas CTAs, to be launched on any stream: the
// same preconditioner choice, grid size and arguments as topo_solve_hdm (the batched multigrid
// form launches many such solves concurrently, one stream each).
topo_status stage_solo2(topo_ctx* c, const double* rho, const double* F, double* U, int m, int ld, double rtol,
                        int maxit, int max_ctas, SoloLaunch2* out) {
  const Grid& g = c->g;
  const long long nunits = (long long)((g.nnx + 31) / 32) * g.nny * g.nnz;
  const bool want_mg = c->pcg_mg != 0;
  int occ = 0;
  if (want_mg)
    TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg2_mg_kernel<2>, P2_THREADS_SOLO, 0));
  else
    TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg2_kernel<2>, P2_THREADS_SOLO, 0));
  if (occ < 1) return fail(c, TOPO_ERR_CUDA, "pcg2 kernel cannot be resident");
  const int per_sm = c->pcg_blocks_per_sm > 0 ? std::min(c->pcg_blocks_per_sm, occ) : std::min(occ, 2);
  long long G = std::min<long long>((long long)per_sm * c->num_sms, std::max(1, max_ctas));
  const long long maxG = (nunits + P2_THREADS_SOLO / 32 - 1) / (P2_THREADS_SOLO / 32);
  if (G > maxG) G = std::max(1LL, maxG);
  const int poly = c->pcg_poly > 0 ? c->pcg_poly : pcg_poly_auto(2);
  topo_status st = build_pcg2_args<2>(c, rho, F, U, m, ld, rtol, maxit, (int)G, &out->a, c->d_sync, poly, want_mg);
  if (st) return st;
  out->mg = want_mg && out->a.mg.L >= 2;
  if (want_mg && !out->mg) {
    st = build_pcg2_args<2>(c, rho, F, U, m, ld, rtol, maxit, (int)G, &out->a, c->d_sync, poly, false);
    if (st) return st;
  }
  out->G = (unsigned)G;
  out->dyn = 0;
  if (out->mg) {
    const MgArgs& M = out->a.mg;
    out->dyn = std::max(((size_t)M.nc * (M.nc + 1) / 2 + M.nc) * sizeof(double), (size_t)M.tail_floats * sizeof(float));
    constexpr size_t dyn_max = std::max(((size_t)MG_COARSE_MAX * (MG_COARSE_MAX + 1) / 2 + MG_COARSE_MAX) * sizeof(double),
                                        MG_TAIL_BYTES);
    if (out->dyn > dyn_max) return fail(c, TOPO_ERR_INVALID, "multigrid shared memory %zu B above %zu B", out->dyn, dyn_max);
    // one value for every launch (see solve_stencil_fp64); set here, never while launching
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(pcg2_mg_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)dyn_max));
  }
  return TOPO_OK;
}

// The staged solve's state resets and its cooperative launch on stream (no host synchronisation,
// no attribute or occupancy calls: capturable in a CUDA graph).
cudaError_t launch_solo2(topo_ctx* c, const SoloLaunch2& s, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(c->d_bar, 0, sizeof(GridBar), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.a.zflag, 0, sizeof(unsigned long long) * s.G, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.a.info, 0, 32, stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s.G);
  cfg.blockDim = dim3(P2_THREADS_SOLO);
  cfg.dynamicSmemBytes = s.dyn;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = s.mg ? cudaLaunchKernelEx(&cfg, pcg2_mg_kernel<2>, s.a) : cudaLaunchKernelEx(&cfg, pcg2_kernel<2>, s.a);
  if (e == cudaSuccess) note_launch();
  return e;
}

template <int DIM>
topo_status solve_stencil_fp64(topo_ctx* c, const double* rho, const double* F, double* U, int m, int ld, double rtol,
                               int maxit, topo_solve_info* info_host) {
  const Grid& g = c->g;
  const long long nunits = (long long)((g.nnx + 31) / 32) * g.nny * g.nnz;
  const bool want_mg = c->pcg_mg != 0;
  int occ = 0;
  if (want_mg)
    TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg2_mg_kernel<DIM>, P2_THREADS_SOLO, 0));
  else
    TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg2_kernel<DIM>, P2_THREADS_SOLO, 0));
  if (occ < 1) return fail(c, TOPO_ERR_CUDA, "pcg2 kernel cannot be resident");
  const int per_sm = c->pcg_blocks_per_sm > 0 ? std::min(c->pcg_blocks_per_sm, occ) : std::min(occ, 2);
  long long G = (long long)per_sm * c->num_sms;
  if (c->pcg_max_ctas > 0 && G > c->pcg_max_ctas) G = c->pcg_max_ctas;  // a share of the GPU
  const long long maxG = (nunits + P2_THREADS_SOLO / 32 - 1) / (P2_THREADS_SOLO / 32);  // >= 1 unit per warp
  if (G > maxG) G = std::max(1LL, maxG);
  Pcg2Args<DIM> a;
  const int poly = c->pcg_poly > 0 ? c->pcg_poly : pcg_poly_auto(DIM);
  topo_status st = build_pcg2_args<DIM>(c, rho, F, U, m, ld, rtol, maxit, (int)G, &a, c->d_sync, poly, want_mg);
  if (st) return st;
  const bool use_mg = want_mg && a.mg.L >= 2;  // a mesh too small to coarsen keeps the polynomial
  if (want_mg && !use_mg) {
    st = build_pcg2_args<DIM>(c, rho, F, U, m, ld, rtol, maxit, (int)G, &a, c->d_sync, poly, false);
    if (st) return st;
  }
  TOPO_CUDA_TRY(c, cudaMemsetAsync(c->d_bar, 0, sizeof(GridBar), c->stream));  // counter, generation, abort
  TOPO_CUDA_TRY(c, cudaMemsetAsync(a.zflag, 0, sizeof(unsigned long long) * G, c->stream));
  TOPO_CUDA_TRY(c, cudaMemsetAsync(a.info, 0, 32, c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(P2_THREADS_SOLO);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (use_mg) {
    // shared memory: the coarsest operator's packed factor and one column (setup), then the
    // vectors of the levels CTA 0 runs alone (the V-cycle)
    const size_t dyn = std::max(((size_t)a.mg.nc * (a.mg.nc + 1) / 2 + a.mg.nc) * sizeof(double),
                                (size_t)a.mg.tail_floats * sizeof(float));
    // the attribute is the kernel's largest request, whatever this launch needs: host threads that
    // launch concurrently then never lower it under one another's launch
    constexpr size_t dyn_max = std::max(((size_t)MG_COARSE_MAX * (MG_COARSE_MAX + 1) / 2 + MG_COARSE_MAX) * sizeof(double),
                                        MG_TAIL_BYTES);
    if (dyn > dyn_max) return fail(c, TOPO_ERR_INVALID, "multigrid shared memory %zu B above %zu B", dyn, dyn_max);
    TOPO_CUDA_TRY(c, cudaFuncSetAttribute(pcg2_mg_kernel<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)dyn_max));
    cfg.dynamicSmemBytes = dyn;
    TOPO_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, pcg2_mg_kernel<DIM>, a));
  } else
    TOPO_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, pcg2_kernel<DIM>, a));
  note_launch();
  if (info_host) {
    int hinfo[4];
    double hrr[2];
    TOPO_CUDA_TRY(c, cudaMemcpyAsync(hinfo, a.info, 16, cudaMemcpyDeviceToHost, c->stream));
    TOPO_CUDA_TRY(c, cudaMemcpyAsync(hrr, a.info_rr, 16, cudaMemcpyDeviceToHost, c->stream));
    TOPO_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int dev_status = 0;
    TOPO_CUDA_TRY(c, cudaMemcpy(&dev_status, &c->d_sync->status, sizeof(int), cudaMemcpyDeviceToHost));
    info_host->iters = hinfo[0];
    info_host->outer = 0;
    info_host->relres = sqrt(hrr[0]);
    info_host->floor = sqrt(hrr[1]);
    info_host->poly = use_mg ? (hinfo[3] ? a.poly : 0) : a.poly;
    info_host->mg_levels = use_mg ? a.mg.L : 0;
    info_host->fallback = use_mg ? hinfo[3] : 0;
    info_host->status = dev_status ? dev_status : hinfo[2];
    if (dev_status) {
      int zero = 0;
      cudaMemcpy(&c->d_sync->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return fail(c, (topo_status)dev_status, "topo_solve_hdm: device status %d", dev_status);
    }
    if (hinfo[2])
      return fail(c, TOPO_ERR_NOT_CONVERGED, "topo_solve_hdm: relres %.3e after %d iterations", info_host->relres,
                  hinfo[0]);
  }
  return TOPO_OK;
}

template topo_status solve_stencil_fp64<2>(topo_ctx*, const double*, const double*, double*, int, int, double, int,
                                           topo_solve_info*);
template topo_status solve_stencil_fp64<3>(topo_ctx*, const double*, const double*, double*, int, int, double, int,
                                           topo_solve_info*);

}  // namespace topo

template topo_status topo::build_pcg2_args<2>(topo_ctx*, const double*, const double*, double*, int, int, double, int,
                                              int, topo::Pcg2Args<2>*, topo::GridSync*, int, bool);
