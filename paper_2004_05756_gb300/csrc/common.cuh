// Internal definitions shared by the libtopo translation units (sm_103a).
//
// Operator: K(rho) = sum_e E(rho_e) P_e K_e P_e^T (Section 2.1, Eq. linelast-res1) applied
// node-centrically on a structured grid: the thread that owns node n sums, over the 4 (Q4)
// or 8 (H8) elements that touch n, E_e times the rows of K_e that belong to n, times the
// element's nodal values. Every node therefore gathers a 3x3 (3x3x3) neighbourhood from a
// shared-memory tile with a one-node halo: no atomics, no scatter, deterministic results.
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>

#include "../../include/topo.h"

namespace topo {

// ---------------------------------------------------------------------------------------
// Optional self-checking build (-DTOPO_BOUNDS_CHECK): every checked global access verifies
// its index against the array length, records the first violation (tag, index, length)
// and skips the access instead of faulting. Off in normal builds.
// ---------------------------------------------------------------------------------------
#ifdef TOPO_BOUNDS_CHECK
struct BoundsLog {
  int hit;
  int tag;
  long long idx;
  long long n;
};
static __device__ BoundsLog g_bounds_log;  // one per translation unit
__device__ inline bool bounds_ok(long long idx, long long n, int tag) {
  if (idx >= 0 && idx < n) return true;
  if (atomicCAS(&g_bounds_log.hit, 0, 1) == 0) {
    g_bounds_log.tag = tag;
    g_bounds_log.idx = idx;
    g_bounds_log.n = n;
  }
  return false;
}
#define TOPO_OK_IDX(idx, n, tag) topo::bounds_ok((long long)(idx), (long long)(n), (tag))
#else
#define TOPO_OK_IDX(idx, n, tag) true
#endif

// ---------------------------------------------------------------------------------------
// Element matrices passed by value as __grid_constant__ kernel parameters, so that the
// FMAs read K_e straight from the constant bank (no load instructions).
// ---------------------------------------------------------------------------------------
template <typename T> struct KeQ4 { T k[64]; };
template <typename T> struct KeH8 { T k[576]; };

template <int DIM, typename T> struct KeOf;
template <typename T> struct KeOf<2, T> { using type = KeQ4<T>; };
template <typename T> struct KeOf<3, T> { using type = KeH8<T>; };

// Grid description used by every kernel.
struct Grid {
  int dim;
  int nx, ny, nz;     // elements per direction (nz = 1 in 2D)
  int nnx, nny, nnz;  // nodes per direction (nnz = 1 in 2D)
  long long nnodes, ndof, nel;
  const uint32_t* fixed_bits;  // Dirichlet mask, one bit per DOF
  double E0, Emin;
  int ipenal;
};

__host__ __device__ inline bool is_fixed(const Grid& g, long long dof) {
#ifdef __CUDA_ARCH__
  return (__ldg(g.fixed_bits + (dof >> 5)) >> (dof & 31)) & 1u;
#else
  return (g.fixed_bits[dof >> 5] >> (dof & 31)) & 1u;
#endif
}

// E(rho) = Emin + rho^p (E0 - Emin), integer p by repeated multiplication.
template <typename T>
__device__ __forceinline__ T young(T rho, T E0, T Emin, int p) {
  T rp = rho;
  for (int i = 1; i < p; ++i) rp *= rho;
  return Emin + rp * (E0 - Emin);
}
template <typename T>
__device__ __forceinline__ T dyoung(T rho, T E0, T Emin, int p) {
  T rp = (T)1;
  for (int i = 1; i < p; ++i) rp *= rho;
  return (T)p * rp * (E0 - Emin);
}

// Local node numbering of a Q1 element: counter-clockwise from (0,0) on z = 0, then z = 1.
__host__ __device__ constexpr int lidx2(int cx, int cy) { return cy ? (cx ? 2 : 3) : (cx ? 1 : 0); }
__host__ __device__ constexpr int lidx3(int cx, int cy, int cz) { return lidx2(cx, cy) + 4 * cz; }

// ---------------------------------------------------------------------------------------
// Tile geometry. A CTA owns a box of TX x TY (x TZ) nodes; shared memory holds the box
// plus a one-node halo of vector values and the (TX+1) x (TY+1) (x (TZ+1)) elements that
// touch the box.
// ---------------------------------------------------------------------------------------
template <int DIM> struct TileShape;
template <> struct TileShape<2> {
  static constexpr int TX = 32, TY = 8, TZ = 1;
  static constexpr int NT = TX * TY;  // threads per CTA: one node each
};
template <> struct TileShape<3> {
  static constexpr int TX = 8, TY = 8, TZ = 4;
  static constexpr int NT = TX * TY * TZ;
};

template <int DIM, typename T> struct TileSmem {
  using S = TileShape<DIM>;
  static constexpr int HX = S::TX + 2, HY = S::TY + 2, HZ = (DIM == 3) ? S::TZ + 2 : 1;
  static constexpr int EX = S::TX + 1, EY = S::TY + 1, EZ = (DIM == 3) ? S::TZ + 1 : 1;
  static constexpr int NH = HX * HY * HZ;  // halo nodes
  static constexpr int NE = EX * EY * EZ;  // elements
  T v[NH * DIM];
  T E[NE];
};

struct TileCoord {
  int i0, j0, k0;
};

template <int DIM>
__host__ __device__ inline long long num_tiles(const Grid& g) {
  using S = TileShape<DIM>;
  long long tx = (g.nnx + S::TX - 1) / S::TX, ty = (g.nny + S::TY - 1) / S::TY;
  long long tz = (DIM == 3) ? (g.nnz + S::TZ - 1) / S::TZ : 1;
  return tx * ty * tz;
}

template <int DIM>
__device__ inline TileCoord tile_coord(const Grid& g, long long t) {
  using S = TileShape<DIM>;
  int ntx = (g.nnx + S::TX - 1) / S::TX, nty = (g.nny + S::TY - 1) / S::TY;
  TileCoord c;
  c.i0 = (int)(t % ntx) * S::TX;
  long long r = t / ntx;
  c.j0 = (int)(r % nty) * S::TY;
  c.k0 = (DIM == 3) ? (int)(r / nty) * S::TZ : 0;
  return c;
}

// Stage the element moduli of a tile: E for elements inside the grid, 0 outside, so that
// boundary nodes need no special case. getE(e) returns E for a valid element index.
template <int DIM, typename T, typename GetE>
__device__ inline void stage_E(TileSmem<DIM, T>& s, const Grid& g, TileCoord c, GetE getE) {
  using TS = TileSmem<DIM, T>;
  for (int idx = threadIdx.x; idx < TS::NE; idx += blockDim.x) {
    int ex = idx % TS::EX;
    int rest = idx / TS::EX;
    int ey = rest % TS::EY;
    int ez = rest / TS::EY;
    int ei = c.i0 - 1 + ex, ej = c.j0 - 1 + ey, ek = c.k0 - 1 + ez;
    bool in = ei >= 0 && ei < g.nx && ej >= 0 && ej < g.ny;
    long long e = (long long)ei + (long long)g.nx * ej;
    if (DIM == 3) {
      in = in && ek >= 0 && ek < g.nz;
      e += (long long)g.nx * g.ny * ek;
    }
    if (TOPO_OK_IDX(idx, TS::NE, 20)) s.E[idx] = in ? getE(e) : (T)0;
  }
}

// Stage vector values of the halo'd node box: getV(dof) for free DOFs inside the grid, 0 for
// Dirichlet DOFs (their columns of K act as zero on free rows) and for nodes outside.
// Consecutive threads read consecutive DOFs of one node row: coalesced.
template <int DIM, typename T, typename GetV>
__device__ inline void stage_V(TileSmem<DIM, T>& s, const Grid& g, TileCoord c, GetV getV) {
  using TS = TileSmem<DIM, T>;
  for (int idx = threadIdx.x; idx < TS::NH * DIM; idx += blockDim.x) {
    int comp = idx % DIM;
    int nidx = idx / DIM;
    int hx = nidx % TS::HX;
    int rest = nidx / TS::HX;
    int hy = rest % TS::HY;
    int hz = rest / TS::HY;
    int i = c.i0 - 1 + hx, j = c.j0 - 1 + hy, k = c.k0 - 1 + hz;
    bool in = i >= 0 && i < g.nnx && j >= 0 && j < g.nny;
    long long n = (long long)i + (long long)g.nnx * j;
    if (DIM == 3) {
      in = in && k >= 0 && k < g.nnz;
      n += (long long)g.nnx * g.nny * k;
    }
    T val = (T)0;
    if (in) {
      long long dof = DIM * n + comp;
      if (TOPO_OK_IDX(dof, g.ndof, 23) && !is_fixed(g, dof)) val = getV(dof);
    }
    if (TOPO_OK_IDX(idx, TS::NH * DIM, 19)) s.v[idx] = val;
  }
}

// Thread -> owned node of the tile. Returns false if the node lies outside the grid.
template <int DIM>
__device__ inline bool owned_node(const Grid& g, TileCoord c, int& tx, int& ty, int& tz, long long& n) {
  using S = TileShape<DIM>;
  int t = threadIdx.x;
  tx = t % S::TX;
  ty = (t / S::TX) % S::TY;
  tz = (DIM == 3) ? t / (S::TX * S::TY) : 0;
  int i = c.i0 + tx, j = c.j0 + ty, k = c.k0 + tz;
  if (i >= g.nnx || j >= g.nny || (DIM == 3 && k >= g.nnz)) return false;
  n = (long long)i + (long long)g.nnx * (j + (long long)g.nny * k);
  return true;
}

// Node-centric Q4 product for the node at tile position (tx, ty): y = sum over the four
// adjacent elements of E_e K_e[rows of this node] v_e. Element (a, b) in {0,1}^2 sits at
// element-tile (tx+a, ty+b); the node is its local corner (1-a, 1-b).
template <typename T>
__device__ __forceinline__ void q4_node(const TileSmem<2, T>& s, int tx, int ty, const KeQ4<T>& ke,
                                        T y[2]) {
  using TS = TileSmem<2, T>;
  y[0] = (T)0;
  y[1] = (T)0;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int L = lidx2(1 - a, 1 - b);
      T s0 = (T)0, s1 = (T)0;
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const int M = lidx2(cx, cy);
          const int h = (ty + b + cy) * TS::HX + (tx + a + cx);
          const T vx = s.v[2 * h], vy = s.v[2 * h + 1];
          s0 = fma(ke.k[(2 * L) * 8 + 2 * M], vx, s0);
          s0 = fma(ke.k[(2 * L) * 8 + 2 * M + 1], vy, s0);
          s1 = fma(ke.k[(2 * L + 1) * 8 + 2 * M], vx, s1);
          s1 = fma(ke.k[(2 * L + 1) * 8 + 2 * M + 1], vy, s1);
        }
      }
      const T e = s.E[(ty + b) * TS::EX + (tx + a)];
      y[0] = fma(e, s0, y[0]);
      y[1] = fma(e, s1, y[1]);
    }
  }
}

// Node-centric H8 product, same construction over the eight adjacent elements.
template <typename T>
__device__ __forceinline__ void h8_node(const TileSmem<3, T>& s, int tx, int ty, int tz,
                                        const KeH8<T>& ke, T y[3]) {
  using TS = TileSmem<3, T>;
  y[0] = y[1] = y[2] = (T)0;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int L = lidx3(1 - a, 1 - b, 1 - c);
        T s0 = (T)0, s1 = (T)0, s2 = (T)0;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
#pragma unroll
          for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
              const int M = lidx3(cx, cy, cz);
              const int h = ((tz + c + cz) * TS::HY + (ty + b + cy)) * TS::HX + (tx + a + cx);
              const T v0 = s.v[3 * h], v1 = s.v[3 * h + 1], v2 = s.v[3 * h + 2];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                const T vd = d == 0 ? v0 : (d == 1 ? v1 : v2);
                s0 = fma(ke.k[(3 * L + 0) * 24 + 3 * M + d], vd, s0);
                s1 = fma(ke.k[(3 * L + 1) * 24 + 3 * M + d], vd, s1);
                s2 = fma(ke.k[(3 * L + 2) * 24 + 3 * M + d], vd, s2);
              }
            }
          }
        }
        const T e = s.E[((tz + c) * TS::EY + (ty + b)) * TS::EX + (tx + a)];
        y[0] = fma(e, s0, y[0]);
        y[1] = fma(e, s1, y[1]);
        y[2] = fma(e, s2, y[2]);
      }
    }
  }
}

template <int DIM, typename T>
__device__ __forceinline__ void node_apply(const TileSmem<DIM, T>& s, int tx, int ty, int tz,
                                           const typename KeOf<DIM, T>::type& ke, T* y);
template <>
__device__ __forceinline__ void node_apply<2, double>(const TileSmem<2, double>& s, int tx, int ty, int,
                                                      const KeQ4<double>& ke, double* y) {
  q4_node<double>(s, tx, ty, ke, y);
}
template <>
__device__ __forceinline__ void node_apply<2, float>(const TileSmem<2, float>& s, int tx, int ty, int,
                                                     const KeQ4<float>& ke, float* y) {
  q4_node<float>(s, tx, ty, ke, y);
}
template <>
__device__ __forceinline__ void node_apply<3, double>(const TileSmem<3, double>& s, int tx, int ty, int tz,
                                                      const KeH8<double>& ke, double* y) {
  h8_node<double>(s, tx, ty, tz, ke, y);
}
template <>
__device__ __forceinline__ void node_apply<3, float>(const TileSmem<3, float>& s, int tx, int ty, int tz,
                                                     const KeH8<float>& ke, float* y) {
  h8_node<float>(s, tx, ty, tz, ke, y);
}

// ---------------------------------------------------------------------------------------
// Block reduction in a fixed order (warp shuffle tree, then warp partials in index order).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sums v over the block; result valid in thread 0. red must hold blockDim.x/32 doubles.
__device__ inline double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    t = (l < nw) ? red[l] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// Three block sums at once (result in thread 0; blockDim.x <= 512, a multiple of 32; red holds
// 3 * 32 doubles). Within a warp the values are reduced by a butterfly that halves the number
// of values each lane carries at the first two levels, so the warp spends 6 FP64 additions on
// all three sums instead of 15 (FP64 issue is scarce on GB300); the order is fixed, so
// the result is deterministic.
__device__ inline void block_sum3(double& a, double& b, double& c, double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  // level 16: lanes 0-15 carry values (0, 1), lanes 16-31 carry (2, 3 = 0)
  const bool lo = l < 16;
  const double ka = lo ? a : c, kb = lo ? b : 0.0;
  const double sa = lo ? c : a, sb = lo ? 0.0 : b;
  double x = ka + __shfl_xor_sync(0xffffffffu, sa, 16);
  double y = kb + __shfl_xor_sync(0xffffffffu, sb, 16);
  // level 8: lanes with bit 3 clear keep x, the others y
  const bool lo8 = (l & 8) == 0;
  double v = (lo8 ? x : y) + __shfl_xor_sync(0xffffffffu, lo8 ? y : x, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  // lane 0: value 0, lane 8: value 1, lane 16: value 2 (lane 24: the zero pad)
  if (l == 0) red[w] = v;
  if (l == 8) red[32 + w] = v;
  if (l == 16) red[64 + w] = v;
  __syncthreads();
  if (w == 0) {
    // lanes 0-15: value 0 of warp l; lanes 16-31: value 1 of warp l - 16; then value 2
    const int ww = l & 15;
    double t = ww < nw ? red[(l >> 4) * 32 + ww] : 0.0;
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 8);
    double u = l < nw ? red[64 + l] : 0.0;
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 4);
    u += __shfl_xor_sync(0xffffffffu, u, 8);
    a = __shfl_sync(0xffffffffu, t, 0);
    b = __shfl_sync(0xffffffffu, t, 16);
    c = __shfl_sync(0xffffffffu, u, 0);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier for cooperative (co-resident) launches, with a deterministic reduction
// folded in: each CTA has written partial[j * G + cta] for j < nred; the last CTA to arrive
// sums them in CTA order into result[j], then releases the others. Every wait is bounded by
// wait_cycles; on expiry the device status becomes TOPO_ERR_TIMEOUT and false is returned.
// ---------------------------------------------------------------------------------------
struct GridSync {
  unsigned int count;  // arrivals at the current barrier (reset before every launch)
  int abort;           // set when a CTA gives up; every waiter leaves (reset before every launch)
  unsigned int gen;    // barrier generation
  int status;          // sticky device status (topo_status), cleared by topo_check
};

__device__ inline void set_status(int* status, int code) { atomicCAS(status, 0, code); }

__device__ inline bool grid_sync_reduce(GridSync* gs, unsigned int& my_gen, const double* partial, double* result,
                                        int nred, long long wait_cycles) {
  __shared__ int s_last;
  __shared__ int s_ok;
  const unsigned int G = gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int arrived = atomicAdd(&gs->count, 1u);
    s_last = (arrived == G - 1);
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    // fixed-order sum of each reduction slot: lane l of warp j sums CTAs l, l+32, ... then a
    // shuffle tree; the order depends only on G.
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = w; j < nred; j += nw) {
      double t = 0.0;
      for (unsigned int c = l; c < G; c += 32) t += __ldcg(partial + (size_t)j * G + c);
      t = warp_sum(t);
      if (l == 0) __stcg(result + j, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      gs->count = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    long long t0 = clock64();
    while (true) {
      unsigned int g = *(volatile unsigned int*)&gs->gen;
      if (g != my_gen) break;
      if (*(volatile int*)&gs->abort != 0) {
        s_ok = 0;
        break;
      }
      if (clock64() - t0 > wait_cycles) {
        set_status(&gs->status, TOPO_ERR_TIMEOUT);
        atomicExch(&gs->abort, 1);
        s_ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  my_gen += 1u;
  return s_ok && (*(volatile int*)&gs->abort == 0);
}

// ---------------------------------------------------------------------------------------
// Grid barrier, second form: a monotonically increasing 64-bit arrival counter with release
// semantics and a generation word polled with acquire semantics (both reset before every
// launch), so no CTA resets anything inside the launch. Barrier number b completes when the
// counter reaches b * G. Bounded wait as above; on expiry a per-launch abort word is set.
// Reductions are not folded in: after the barrier every CTA reduces the per-CTA partials
// itself (reduce_slots), in parallel, in a fixed order.
// ---------------------------------------------------------------------------------------
struct GridBar {
  unsigned long long count;
  unsigned long long gen;
  int abort;
  int pad;
};

// Barrier over a group of `group` co-resident CTAs sharing one GridBar (the whole grid, or one
// instance's CTAs in a batched launch).
__device__ inline bool grid_barrier(GridBar* gb, int* status, unsigned long long& b, long long wait_cycles,
                                    unsigned group) {
  __shared__ int s_ok;
  __syncthreads();
  b += 1;
  if (threadIdx.x == 0) {
    s_ok = 1;
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> cnt(gb->count);
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> gen(gb->gen);
    const unsigned long long target = b * (unsigned long long)group;
    const unsigned long long old = cnt.fetch_add(1ull, cuda::memory_order_release);
    if (old == target - 1) {
      gen.store(b, cuda::memory_order_release);
    } else {
      const long long t0 = clock64();
      while (gen.load(cuda::memory_order_acquire) < b) {
        __nanosleep(20);
        if (*(volatile int*)&gb->abort) {
          s_ok = 0;
          break;
        }
        if (clock64() - t0 > wait_cycles) {
          atomicCAS(status, 0, (int)TOPO_ERR_TIMEOUT);
          atomicExch(&gb->abort, 1);
          s_ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// out[j] = sum over g < G of partial[j * G + g], j < nslots, summed lane-strided then by a
// shuffle tree (an order fixed by G alone). One warp per slot. Result in shared memory.
__device__ inline void reduce_slots(const double* partial, unsigned G, int nslots, double* out) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = w; j < nslots; j += nw) {
    const double* pj = partial + (size_t)j * G;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    unsigned g = l;
    for (; g + 96 < G; g += 128) {
      t0 += __ldcg(pj + g);
      t1 += __ldcg(pj + g + 32);
      t2 += __ldcg(pj + g + 64);
      t3 += __ldcg(pj + g + 96);
    }
    for (; g < G; g += 32) t0 += __ldcg(pj + g);
    double t = warp_sum((t0 + t1) + (t2 + t3));
    if (l == 0) out[j] = t;
  }
  __syncthreads();
}

}  // namespace topo

// ---------------------------------------------------------------------------------------
// Context (host side).
// ---------------------------------------------------------------------------------------
struct topo_ctx {
  topo::Grid g;           // device pointers inside
  double E0, Emin, nu, penal, rmin;
  int ipenal;
  cudaStream_t stream;
  int device, num_sms;
  uint32_t* d_fixed_bits;
  int* d_fixed_list;      // Dirichlet DOF indices, ascending
  int nfixed;
  topo::KeQ4<double> q4_64;
  topo::KeQ4<float> q4_32, q4_bf;
  topo::KeH8<double> h8_64;
  topo::KeH8<float> h8_32, h8_bf;
  double bf_scale;  // K_e = bf_scale * (BF16 table); folded into E(rho) by the BF16 form
  int bf_exact;     // 1 when the BF16 table holds K_e / bf_scale exactly
  // filter stencil (host-computed offsets and weights, device copy)
  int nstencil;
  int* d_stencil_off;     // [nstencil * 3]
  double* d_stencil_w;    // [nstencil]
  double* d_Hsinv;        // [nel]: 1 / Hs_e, the reciprocal filter normaliser
  // device status word + grid barrier state
  topo::GridSync* d_sync;
  topo::GridBar* d_bar;    // state of the second barrier form
  // generic scratch (grown on demand)
  void* d_scratch;
  size_t scratch_bytes;
  unsigned long long scratch_gen;  // bumped whenever d_scratch is (re)allocated
  double* d_red;          // small reduction buffer (partials)
  size_t red_bytes;
  // parameters
  double inner_rtol;
  int max_outer;
  long long wait_cycles;
  int rom_refine;
  int pcg_blocks_per_sm;
  int inner_cap;
  int hdm_kernel;  // 0: assembled-stencil Chronopoulos-Gear PCG (FP64); 1: element-form PCG
  int pcg_max_ctas;  // cap on the CTAs of one persistent solve (0 = none)
  int rom_tensor;    // FP32 projection contraction: 1 tensor cores (tcgen05), 0 SIMT FP32
  int rom_asm_tensor;  // per-density reduced assembly of many candidates: 1 tensor cores (Ozaki digits), 0 FP64 SIMT
  int apply_cols;    // columns per CTA of the 2D node-centric apply (0 = default split)
  int apply_stages;  // 2D FP32 block apply: 0 cp.async staging, 2-4 TMA units in flight per CTA
  int pcg_poly;      // FP64 stencil PCG: degree of the Chebyshev polynomial preconditioner (0 = auto)
  int pcg_mg;        // FP64 stencil PCG: 1 = multigrid V-cycle preconditioner, 0 = polynomial / Jacobi
  int mg_deg;        // multigrid: Chebyshev smoothing steps per side (1 .. 4)
  long long mg_single_nodes;  // multigrid: levels with at most this many nodes run on one CTA
  int filter_kind;   // 0 = linear cone filter, 1 = Helmholtz filter
  double helm_r;     // Helmholtz length r (element lengths; 0 = rmin / (2 sqrt 3))
  double helm_r_built;  // the r the cosine and diagonal data were built for (-1 = none)
  double* d_helm;    // Helmholtz filter: cosine matrices, diagonal, work buffers
  size_t helm_bytes;
  char err[512];
};

namespace topo {

topo_status fail(topo_ctx* c, topo_status s, const char* fmt, ...);
void note_launch();  // counts kernel launches issued by the library (diagnostics)
topo_status cuda_fail(topo_ctx* c, cudaError_t e, const char* where);
topo_status ensure_scratch(topo_ctx* c, size_t bytes);
topo_status ensure_red(topo_ctx* c, size_t bytes);
bool dev_ptr_ok(const void* p);

// Launch helpers implemented in apply.cu (used by the ROM code as well).
topo_status launch_apply(topo_ctx* c, const double* rho, const void* V, void* Y, int m, int ld, topo_prec prec,
                         const int* gate = nullptr);
// The filter of R fields (forward, or adjoint when adjoint != 0) in one launch (ctx.cu).
topo_status launch_filter_batch(topo_ctx* c, const double* in, long long ldin, double* out, long long ldout, int R,
                                int adjoint);
// Compliance gradients of R designs with one state each (ctx.cu).
// Residual norms ||f - K(rho_r) u_r|| (and / ||f||) of R designs in one launch (apply.cu): out2 +
// 2 r receives them; partial holds 2 x tiles x R doubles.
size_t cgs2_scratch_doubles(topo_ctx* c);
topo_status launch_cgs2(topo_ctx* c, const double* U, int m, long long ld, double* Phi, const double* f, double* b,
                        double drop_rel, double* scratch, int* k_dev);
topo_status launch_residual64_batch(topo_ctx* c, const double* rho, long long ldr, const double* U, long long ldu,
                                    const double* f, double* out2, int R, double* partial, double* dc = nullptr,
                                    long long ldd = 0);
long long residual_tiles(topo_ctx* c);
// Residual r = f - K(rho) u on free DOFs (0 on Dirichlet DOFs), FP64, with ||r||^2 and ||f||^2
// partials reduced to out2[0..1] (device). r may be NULL (norms only).
topo_status launch_residual64(topo_ctx* c, const double* rho, const double* u, const double* f, double* r,
                              double* out2);
// One reduced solve of a batch of different problems (k <= 32): the FP64 Cholesky of H (k x k,
// row-major, overwritten by L), y = H^-1 b, *J = b^T y, *ok = 1 (0 and NOT_SPD in *status on a
// non-positive pivot). launch_chol_small_multi runs n of them, one warp each (rom.cu).
struct RedSolve {
  double* H;
  const double* b;
  double* y;
  double* J;
  int* status;
  int* ok;
  int k;
  int pad;
};
cudaError_t launch_chol_small_multi(const RedSolve* tab, int n, cudaStream_t stream);
// The Helmholtz filter of R fields (its own adjoint): field r at in + r ldin -> out + r ldout
// (helmholtz.cu).
topo_status helmholtz_apply(topo_ctx* c, const double* in, long long ldin, double* out, long long ldout, int R);
// Deterministic sum of n doubles -> *out (device), two passes.
topo_status launch_sum(topo_ctx* c, const double* x, long long n, double* out);
// Tensor-core contraction (tcgen05, kind::tf32 with an exact hi/lo split of each FP32 operand):
// per-CTA FP64 partials of A^T B into partial[g * k1 * k2 + i * k2 + j], g < *G_out. A, B are
// FP32 column-major N x k1 / N x k2, 16-byte aligned, lda and ldb multiples of 4; k1, k2 <= 128.
topo_status launch_atb_tc_partial(topo_ctx* c, const float* A, long long lda, int k1, const float* B, long long ldb,
                                  int k2, long long N, double* partial, size_t partial_cap, int* G_out);

#define TOPO_CUDA_TRY(ctx, expr)                         \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return topo::cuda_fail((ctx), _e, #expr); \
  } while (0)

}  // namespace topo
