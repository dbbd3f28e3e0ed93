// Matrix-free K(rho) V (Section 2.1, Eq. linelast-res1) and the FP64 residual
// r = f - K(rho) u with its norms (Section 3.3).
//
// One CTA per node tile; the element moduli of the tile are staged once and reused for
// every column the CTA processes; each column's halo'd node box is staged in shared memory
// with coalesced loads (Dirichlet DOFs zeroed), then every thread forms its node's rows.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace topo {

template <int DIM, typename T>
struct ApplyArgs {
  Grid g;
  typename KeOf<DIM, T>::type ke;
  const double* rho;
  const T* V;
  T* Y;
  long long ld;
  int m;
  int cols_per_cta;
  T escale;         // folded into E(rho): 1, or the BF16 table's scale
  const int* gate;  // optional device flag: the launch does nothing when *gate == 0
};

template <int DIM, typename T>
__global__ void __launch_bounds__(TileShape<DIM>::NT) apply_kernel(const __grid_constant__ ApplyArgs<DIM, T> a) {
  __shared__ TileSmem<DIM, T> s;
  if (a.gate && *a.gate == 0) return;
  const Grid& g = a.g;
  const TileCoord tc = tile_coord<DIM>(g, blockIdx.x);
  const T E0 = (T)g.E0, Emin = (T)g.Emin, es = a.escale;
  stage_E<DIM, T>(s, g, tc, [&](long long e) { return es * young<T>((T)a.rho[e], E0, Emin, g.ipenal); });
  int tx, ty, tz;
  long long n = 0;
  const bool own = owned_node<DIM>(g, tc, tx, ty, tz, n);
  const int c0 = blockIdx.y * a.cols_per_cta;
  const int c1 = min(a.m, c0 + a.cols_per_cta);
  for (int col = c0; col < c1; ++col) {
    const T* v = a.V + (long long)col * a.ld;
    T* y = a.Y + (long long)col * a.ld;
    stage_V<DIM, T>(s, g, tc, [&](long long dof) { return v[dof]; });
    __syncthreads();
    if (own) {
      T out[DIM];
      node_apply<DIM, T>(s, tx, ty, tz, a.ke, out);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const long long dof = DIM * n + c;
        y[dof] = is_fixed(g, dof) ? v[dof] : out[c];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Node-centric 2D apply for blocks of columns. A CTA owns a 32 x 8 node tile, one node per
// thread. Each thread forms its node's 3 x 3-block stencil row (36 coefficients, kept in
// registers) once from the moduli of the 4 elements around it, with the Dirichlet convention
// folded in (a fixed row is the identity, a fixed neighbour column zero). The columns are
// then processed in batches of AB: the tile's 34 x 10 halo box of every column of a batch is
// copied into shared memory with asynchronous copies (zero-filled outside the grid), two
// batches ahead of the one being computed (a ring of NBUF = 3 buffers); per node and column
// that is 9 shared loads, 36 FMAs and one vector store. Half the flops of the element form, V read from DRAM
// about once, and the copies of a whole batch in flight at once.
// Needs an even leading dimension and V, Y aligned to a (x, y) pair.
// ---------------------------------------------------------------------------------------
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// acc += c * v componentwise, each component one fused multiply-add rounded to nearest: one
// packed FP32x2 instruction on sm_100 and later, two FP64 FMAs for double.
__device__ __forceinline__ void fma_pair(float2 c, float2 v, float2& acc) { acc = __ffma2_rn(c, v, acc); }
__device__ __forceinline__ void fma_pair(double2 c, double2 v, double2& acc) {
  acc.x = fma(c.x, v.x, acc.x);
  acc.y = fma(c.y, v.y, acc.y);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;  // 0: the BYTES destination bytes are zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(n) : "memory");
}

// Stencil row of node (i, j) of a 2D Q4 grid: C[nb][2 r + d] couples DOF r of the node with
// DOF d of neighbour nb = (dx + 1) + 3 (dy + 1), summed over the up to four elements around
// the node with their SIMP moduli; Dirichlet rows are the identity, Dirichlet columns and
// neighbours outside the grid zero. Returns the 9-bit mask of neighbours outside the grid.
template <typename T>
__device__ __forceinline__ unsigned node_stencil_q4(const ApplyArgs<2, T>& a, int i, int j, bool own, long long n,
                                                    T (&C)[9][4]) {
  const Grid& g = a.g;
  unsigned outside = 0;
  const T E0 = (T)g.E0, Emin = (T)g.Emin, es = a.escale;
  // moduli of the elements around the node: q = qa + 2 qb is element (i - 1 + qa, j - 1 + qb)
  T E[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int ei = i - 1 + (q & 1), ej = j - 1 + (q >> 1);
    const bool in = own && ei >= 0 && ei < g.nx && ej >= 0 && ej < g.ny;
    E[q] = in ? es * young<T>((T)a.rho[ei + (long long)g.nx * ej], E0, Emin, g.ipenal) : (T)0;
  }
  const bool rfix0 = own && is_fixed(g, 2 * n), rfix1 = own && is_fixed(g, 2 * n + 1);
#pragma unroll
  for (int nb = 0; nb < 9; ++nb) {
    const int dx = nb % 3 - 1, dy = nb / 3 - 1;
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int qa = q & 1, qb = q >> 1;
      const int cx = dx + 1 - qa, cy = dy + 1 - qb;
      if (cx < 0 || cx > 1 || cy < 0 || cy > 1) continue;
      const int L = lidx2(1 - qa, 1 - qb), M = lidx2(cx, cy);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int d = 0; d < 2; ++d)
          acc[r * 2 + d] = fma(E[q], a.ke.k[(2 * L + r) * 8 + 2 * M + d], acc[r * 2 + d]);
    }
    const int ii = i + dx, jj = j + dy;
    const bool nin = own && ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny;
    if (own && !nin) outside |= 1u << nb;
    const long long m = nin ? ii + (long long)g.nnx * jj : 0;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        T v = acc[r * 2 + d];
        if (!nin || is_fixed(g, 2 * m + d)) v = (T)0;
        if (r == 0 ? rfix0 : rfix1) v = (nb == 4 && r == d) ? (T)1 : (T)0;
        C[nb][r * 2 + d] = v;
      }
  }
  return outside;
}

template <typename T>
__global__ void __launch_bounds__(256) apply2_kernel(const __grid_constant__ ApplyArgs<2, T> a) {
  using V2 = typename Vec2<T>::type;
  constexpr int AB = 32 / (int)sizeof(T);  // columns per batch: 8 (FP32) or 4 (FP64)
  constexpr int HX = 34, HB = 340;         // halo box: 34 x 10 nodes
  constexpr int NBUF = 3;
  extern __shared__ __align__(16) unsigned char apply2_smem[];
  V2 (*sv)[AB][HB] = reinterpret_cast<V2 (*)[AB][HB]>(apply2_smem);  // [NBUF][AB][HB]
  if (a.gate && *a.gate == 0) return;
  const Grid& g = a.g;
  const int tiles_x = (g.nnx + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = (int)(blockIdx.x % tiles_x) * 32, j0 = (int)(blockIdx.x / tiles_x) * 8;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < g.nnx && j < g.nny;
  const long long n = own ? i + (long long)g.nnx * j : 0;
  V2 Cp[9][2];  // (C[nb][0], C[nb][1]) and (C[nb][2], C[nb][3]): the x and y parts of both rows
  {
    T C[9][4];
    node_stencil_q4(a, i, j, own, n, C);
#pragma unroll
    for (int nb = 0; nb < 9; ++nb) {
      Cp[nb][0].x = C[nb][0];
      Cp[nb][0].y = C[nb][1];
      Cp[nb][1].x = C[nb][2];
      Cp[nb][1].y = C[nb][3];
    }
  }
  const int c0 = blockIdx.y * a.cols_per_cta;
  const int c1 = min(a.m, c0 + a.cols_per_cta);
  const int nbatch = c1 > c0 ? (c1 - c0 + AB - 1) / AB : 0;
  // copies: warp w moves halo rows (column, row) = w, w + 8, ... of a batch, lane = x offset
  // (lanes 0 and 1 also take the last two nodes of the 34-node row)
  const int lane = tx, warp = ty;
  const int gi0 = i0 - 1 + lane, gi1 = i0 + 31 + lane;
  const bool xin0 = gi0 >= 0 && gi0 < g.nnx, xin1 = lane < 2 && gi1 < g.nnx;
  const long long pitch = a.ld / 2;  // column stride in (x, y) pairs
  const V2* V2base = reinterpret_cast<const V2*>(a.V);
  auto issue = [&](int b, int buf) {
    const int cb = c0 + b * AB;
    V2* dst = &sv[buf][0][0];
    for (int pr = warp; pr < AB * 10; pr += 8) {
      const int col = pr / 10, hy = pr - col * 10;
      const int gj = j0 - 1 + hy;
      const bool yin = cb + col < c1 && gj >= 0 && gj < g.nny;
      const V2* row = V2base + (long long)(cb + col) * pitch + (long long)g.nnx * gj;
      V2* d = dst + col * HB + hy * HX;
      cp_async_zfill<sizeof(V2)>(d + lane, (yin && xin0) ? row + gi0 : V2base, yin && xin0);
      if (lane < 2) cp_async_zfill<sizeof(V2)>(d + 32 + lane, (yin && xin1) ? row + gi1 : V2base, yin && xin1);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  V2* ybase = reinterpret_cast<V2*>(a.Y) + n;
  if (nbatch > 0) issue(0, 0);
  if (nbatch > 1) issue(1, 1);
  int buf = 0;
  for (int b = 0; b < nbatch; ++b) {
    if (b + 2 < nbatch) {
      issue(b + 2, buf == 0 ? NBUF - 1 : buf - 1);  // the buffer after the next one
      asm volatile("cp.async.wait_group 2;" ::: "memory");  // batch b has landed
    } else if (b + 1 < nbatch) {
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const int cb = c0 + b * AB;
    if (own) {
      const V2* sb = &sv[buf][0][ty * HX + tx];  // the node's 3 x 3 neighbourhood starts here
#pragma unroll
      for (int col = 0; col < AB; ++col) {
        if (cb + col >= c1) break;
        V2 o;
        if constexpr (std::is_same<T, float>::value) {
          // row r of the node: sum over neighbours of the x part C[nb][2r] t.x and, separately,
          // of the y part C[nb][2r+1] t.y (one packed FMA each); the two partial sums are added
          // at the end. The TMA-staged form uses the same order.
          V2 p0, p1;
          p0.x = p0.y = p1.x = p1.y = (T)0;
#pragma unroll
          for (int nb = 0; nb < 9; ++nb) {
            const V2 t = sb[col * HB + (nb / 3) * HX + (nb % 3)];
            fma_pair(Cp[nb][0], t, p0);
            fma_pair(Cp[nb][1], t, p1);
          }
          o.x = p0.x + p0.y;
          o.y = p1.x + p1.y;
        } else {
          // FP64 is bound by the FP64 pipe: one chain per row, no extra additions
          T y0 = (T)0, y1 = (T)0;
#pragma unroll
          for (int nb = 0; nb < 9; ++nb) {
            const V2 t = sb[col * HB + (nb / 3) * HX + (nb % 3)];
            y0 = fma(Cp[nb][0].x, t.x, y0);
            y0 = fma(Cp[nb][0].y, t.y, y0);
            y1 = fma(Cp[nb][1].x, t.x, y1);
            y1 = fma(Cp[nb][1].y, t.y, y1);
          }
          o.x = y0;
          o.y = y1;
        }
        ybase[(long long)(cb + col) * pitch] = o;
      }
    }
    __syncthreads();  // the buffer of batch b is refilled by batch b + 3
    buf = buf == NBUF - 1 ? 0 : buf + 1;
  }
}

template <typename T>
constexpr size_t apply2_smem_bytes() {
  return 3 * (32 / sizeof(T)) * 340 * 2 * sizeof(T);
}

// ---------------------------------------------------------------------------------------
// 2D node-centric block apply in FP32 with the halo rows staged by TMA: the form for 16-byte
// aligned column pitches (ld % 4 == 0, V 16-byte aligned). Same stencil rows and the same
// products in the same order as apply2_kernel, so both forms give identical results.
//
// Work unit = one 32 x 8 node tile times one batch of AB = 8 columns, numbered tile-major.
// A persistent grid (every resident CTA slot of the GPU) splits the units evenly, each CTA a
// contiguous range, so there is no wave tail; a thread forms its node's stencil row again
// only when its CTA's range enters the next tile. Per unit one thread issues ten TMA boxes, one per
// halo row, of 72 floats (36 nodes from the even node at or before the row's first halo node,
// so that x is 16-byte aligned) by AB columns, all completing on the unit's mbarrier; NBUF
// units are in flight per CTA. Rows and columns outside V read as zero. Halo positions
// outside the grid hold whatever lies beside them in V (the end of the previous or the start
// of the next grid row): a thread zeroes each such slot that it reads before reading it, so a
// non-finite value there never enters a product.
// Every mbarrier wait is bounded by wait_cycles; on expiry the status becomes
// TOPO_ERR_TIMEOUT, the CTA stops after the unit in hand and waits for its copies in flight.
// ---------------------------------------------------------------------------------------
namespace tmaapply {
constexpr int AB = 8;                         // columns per unit
constexpr int BOXN = 36;                      // nodes per halo row box
constexpr int ROWS = 10;                      // halo rows of a 32 x 8 tile
constexpr int BOX_BYTES = 2 * BOXN * AB * 4;  // 2304 = 18 x 128: every box 128-byte aligned
constexpr int UNIT_BYTES = ROWS * BOX_BYTES;  // 23040
constexpr size_t smem_bytes(int nbuf) { return 128 + (size_t)nbuf * UNIT_BYTES + 8 * (size_t)nbuf; }
}  // namespace tmaapply

// Resident CTAs per SM that each ring depth is built for: the shared memory of NBUF units
// (23 KB each) and the registers fit 4, 3 and 2 CTAs for NBUF = 2, 3, 4.
template <int NBUF>
__global__ void __launch_bounds__(256, NBUF == 2 ? 4 : (NBUF == 3 ? 3 : 2))
    apply2_tma_kernel(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ ApplyArgs<2, float> a,
                      long long units, int* status, long long wait_cycles) {
  using namespace tmaapply;
  extern __shared__ unsigned char apply2_tma_smem[];
  unsigned char* base = apply2_tma_smem + ((128u - (su32(apply2_tma_smem) & 127u)) & 127u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + NBUF * UNIT_BYTES);
  __shared__ int abort_word;
  if (a.gate && *a.gate == 0) return;
  const Grid& g = a.g;
  const int tiles_x = (g.nnx + 31) / 32;
  const int nb = (a.m + AB - 1) / AB;  // units per tile
  const long long u_begin = units * blockIdx.x / gridDim.x;
  const int nunits = (int)(units * (blockIdx.x + 1) / gridDim.x - u_begin);
  // unit q of this CTA -> its tile t and first column c0
  auto unit_of = [&](int q, int& t, int& c0) {
    const long long u = u_begin + q;
    t = (int)(u / nb);
    c0 = (int)(u - (long long)t * nb) * AB;
  };
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const uint32_t buf0 = su32(base);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NBUF; ++s) mbar_init(su32(&full[s]), 1);
    abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmV) : "memory");
  }
  __syncthreads();
  auto issue = [&](int q) {  // thread 0: the ten halo-row boxes of the CTA's unit q
    int t, c0;
    unit_of(q, t, c0);
    const int i0 = (t % tiles_x) * 32, j0 = (t / tiles_x) * 8;
    const uint32_t bar = su32(&full[q % NBUF]);
    const uint32_t dst = buf0 + (uint32_t)(q % NBUF) * UNIT_BYTES;
    mbar_expect_tx(bar, UNIT_BYTES);
#pragma unroll 1
    for (int hy = 0; hy < ROWS; ++hy) {
      const long long node = (long long)g.nnx * (j0 - 1 + hy) + (i0 - 1);
      tma_load_2d(dst + hy * BOX_BYTES, &tmV, (int)(2 * (node - (node & 1))), c0, bar);
    }
  };
  int issued = 0;
  if (threadIdx.x == 0)
    for (; issued < NBUF - 1 && issued < nunits; ++issued) issue(issued);
  const Ctl ctl{&abort_word, status, wait_cycles};
  const float2* __restrict__ sv = reinterpret_cast<const float2*>(base);
  float2* __restrict__ svw = reinterpret_cast<float2*>(base);
  float2* Y2 = reinterpret_cast<float2*>(a.Y);
  const long long pitch = a.ld / 2;  // column stride in (x, y) pairs
  int cur_tile = -1;
  float2 Cp[9][2];
  int off[3] = {0, 0, 0};  // float2 offset of halo rows ty .. ty + 2 at the node's column, in a unit
  unsigned outside = 0;
  bool own = false;
  long long n = 0;
  int q = 0;
  bool failed = false;
  for (; q < nunits; ++q) {
    if (threadIdx.x == 0 && issued < nunits) issue(issued++);  // into the buffer unit q - 1 released
    int t, c0;
    unit_of(q, t, c0);
    if (t != cur_tile) {
      cur_tile = t;
      const int i0 = (t % tiles_x) * 32, j0 = (t / tiles_x) * 8;
      const int i = i0 + tx, j = j0 + ty;
      own = i < g.nnx && j < g.nny;
      n = own ? i + (long long)g.nnx * j : 0;
      {
        float C[9][4];
        outside = node_stencil_q4(a, i, j, own, n, C);
#pragma unroll
        for (int nbr = 0; nbr < 9; ++nbr) {
          Cp[nbr][0] = make_float2(C[nbr][0], C[nbr][1]);
          Cp[nbr][1] = make_float2(C[nbr][2], C[nbr][3]);
        }
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const long long node = (long long)g.nnx * (j0 - 1 + ty + r) + (i0 - 1);
        off[r] = (ty + r) * (BOXN * AB) + tx + (int)(node & 1);
      }
    }
    const int s = q % NBUF;
    if (!wait_bar(su32(&full[s]), (uint32_t)((q / NBUF) & 1), ctl, false)) failed = true;
    if (!failed && own) {
      const int sb = s * (UNIT_BYTES / 8);
      if (outside) {
#pragma unroll
        for (int nbr = 0; nbr < 9; ++nbr)
          if (outside & (1u << nbr))
#pragma unroll
            for (int col = 0; col < AB; ++col) svw[sb + off[nbr / 3] + col * BOXN + nbr % 3] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int col = 0; col < AB; ++col) {
        if (c0 + col >= a.m) break;
        float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int nbr = 0; nbr < 9; ++nbr) {
          const float2 v = sv[sb + off[nbr / 3] + col * BOXN + nbr % 3];
          fma_pair(Cp[nbr][0], v, p0);
          fma_pair(Cp[nbr][1], v, p1);
        }
        Y2[n + (long long)(c0 + col) * pitch] = make_float2(p0.x + p0.y, p1.x + p1.y);
      }
      // the zeroed slots are generic-proxy writes; the TMA that refills this buffer must see
      // them as ordered before it
      if (outside) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (__syncthreads_or(failed)) break;
  }
  if (failed && threadIdx.x == 0) {
    // copies still in flight: units q .. issued - 1, each in its own buffer
    const Ctl td{&abort_word, status, kTeardownCycles};
    for (int r = q; r < issued; ++r) wait_bar(su32(&full[r % NBUF]), (uint32_t)((r / NBUF) & 1), td, false);
  }
}

template <int NBUF>
static topo_status launch_apply2_tma_n(topo_ctx* c, const CUtensorMap& map, const ApplyArgs<2, float>& a,
                                       long long units) {
  const size_t sm = tmaapply::smem_bytes(NBUF);
  TOPO_CUDA_TRY(c, cudaFuncSetAttribute(apply2_tma_kernel<NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  static int per_sm = 0;  // resident CTAs per SM of this instantiation (the same on every GB300)
  if (per_sm == 0) {
    int v = 0;
    TOPO_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, apply2_tma_kernel<NBUF>, 256, sm));
    per_sm = v > 0 ? v : 1;
  }
  const long long grid = std::min(units, (long long)per_sm * c->num_sms);
  apply2_tma_kernel<NBUF><<<(unsigned)grid, 256, sm, c->stream>>>(map, a, units, &c->d_sync->status, c->wait_cycles);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

static topo_status launch_apply2_tma(topo_ctx* c, const ApplyArgs<2, float>& a) {
  const Grid& g = c->g;
  CUtensorMap map;
  if (!encode_map_f32_2d(&map, a.V, a.ld, g.ndof, a.m, 2 * tmaapply::BOXN, tmaapply::AB, false))
    return fail(c, TOPO_ERR_CUDA, "cuTensorMapEncodeTiled failed for the block apply operand");
  const long long tiles = (long long)((g.nnx + 31) / 32) * ((g.nny + 7) / 8);
  const long long units = tiles * ((a.m + tmaapply::AB - 1) / tmaapply::AB);
  switch (c->apply_stages) {
    case 2: return launch_apply2_tma_n<2>(c, map, a, units);
    case 4: return launch_apply2_tma_n<4>(c, map, a, units);
    default: return launch_apply2_tma_n<3>(c, map, a, units);
  }
}

template <int DIM, typename T>
static topo_status apply_impl(topo_ctx* c, const double* rho, const T* V, T* Y, int m, int ld,
                              const typename KeOf<DIM, T>::type& ke, double escale, const int* gate) {
  ApplyArgs<DIM, T> a;
  a.escale = (T)escale;
  a.gate = gate;
  a.g = c->g;
  a.ke = ke;
  a.rho = rho;
  a.V = V;
  a.Y = Y;
  a.ld = ld;
  a.m = m;
  const bool pairs = DIM == 2 && (ld % 2 == 0) && ((uintptr_t)V % (2 * sizeof(T)) == 0) &&
                     ((uintptr_t)Y % (2 * sizeof(T)) == 0);
  long long tiles = pairs ? (long long)((c->g.nnx + 31) / 32) * ((c->g.nny + 7) / 8) : num_tiles<DIM>(c->g);
  // enough CTAs to fill the GPU several times over, each reusing its staged E for a run
  // of columns
  long long want_ctas = 8LL * c->num_sms;
  long long groups = (want_ctas + tiles - 1) / tiles;
  if (groups > m) groups = m;
  if (groups < 1) groups = 1;
  if (groups > 65535) groups = 65535;
  a.cols_per_cta = (int)((m + groups - 1) / groups);
  // node-centric kernel: 32 columns per CTA amortise the coefficient set-up best at
  // 600x200, m = 64 (measured against 16, 22, 64); TOPO_PARAM_TILE_X overrides
  if (pairs) a.cols_per_cta = std::min(m, c->apply_cols > 0 ? c->apply_cols : 32);
  groups = (m + a.cols_per_cta - 1) / a.cols_per_cta;
  dim3 grid((unsigned)tiles, (unsigned)groups);
  if constexpr (DIM == 2 && std::is_same<T, float>::value) {
    if (pairs && c->apply_stages > 0 && ld % 4 == 0 && ((uintptr_t)V & 15) == 0 && c->g.ndof < (1LL << 30))
      return launch_apply2_tma(c, a);
  }
  if constexpr (DIM == 2) {
    if (pairs) {
      const size_t sm = apply2_smem_bytes<T>();
      TOPO_CUDA_TRY(c, cudaFuncSetAttribute(apply2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      apply2_kernel<T><<<grid, 256, sm, c->stream>>>(a);
      note_launch();
      TOPO_CUDA_TRY(c, cudaGetLastError());
      return TOPO_OK;
    }
  }
  apply_kernel<DIM, T><<<grid, TileShape<DIM>::NT, 0, c->stream>>>(a);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

topo_status launch_apply(topo_ctx* c, const double* rho, const void* V, void* Y, int m, int ld, topo_prec prec,
                         const int* gate) {
  const bool bf = prec == TOPO_FP32_BF16KE_REFINED;
  const double es = bf ? c->bf_scale : 1.0;
  if (c->g.dim == 2) {
    if (prec == TOPO_FP64)
      return apply_impl<2, double>(c, rho, (const double*)V, (double*)Y, m, ld, c->q4_64, 1.0, gate);
    return apply_impl<2, float>(c, rho, (const float*)V, (float*)Y, m, ld, bf ? c->q4_bf : c->q4_32, es, gate);
  }
  if (prec == TOPO_FP64)
    return apply_impl<3, double>(c, rho, (const double*)V, (double*)Y, m, ld, c->h8_64, 1.0, gate);
  return apply_impl<3, float>(c, rho, (const float*)V, (float*)Y, m, ld, bf ? c->h8_bf : c->h8_32, es, gate);
}

// ---------------------------------------------------------------------------------------
// FP64 residual r = f - K u on free DOFs (0 on Dirichlet DOFs) with per-CTA partial sums of
// ||r||^2 and ||f||^2 (free DOFs), then a fixed-order final reduction to sqrt values.
// GRAD: each thread also forms the compliance gradient dc_e = -E'(rho_e) u_e^T K_e u_e of the
// element whose lower-left node it owns, from the tile's staged u (its corners lie in the node
// box and its halo), in the symmetric form and order of grad_kernel, so the values equal that
// kernel's bit for bit without its global gathers of u_e.
// ---------------------------------------------------------------------------------------
template <int DIM>
struct ResArgs {
  Grid g;
  typename KeOf<DIM, double>::type ke;
  const double* rho;
  const double* u;
  const double* f;
  double* r;        // may be null
  double* partial;  // [2 * G] per design
  long long ldr, ldu;  // strides of rho and u between the designs of blockIdx.y (several per launch)
  double* dc;          // GRAD: element gradients, stride ldd between designs
  long long ldd;
};

template <int DIM>
__device__ __forceinline__ void tile_element_grad(const TileSmem<DIM, double>& s, const Grid& g, TileCoord tc, int tx,
                                                  int ty, int tz, const typename KeOf<DIM, double>::type& ke,
                                                  const double* rho, double* dc) {
  using TS = TileSmem<DIM, double>;
  constexpr int NN = DIM == 2 ? 4 : 8, ND = DIM * NN;
  const int i = tc.i0 + tx, j = tc.j0 + ty, k = tc.k0 + tz;
  if (i >= g.nx || j >= g.ny || (DIM == 3 && k >= g.nz)) return;
  const long long e = (long long)i + (long long)g.nx * (j + (long long)g.ny * k);
  double ue[ND];
#pragma unroll
  for (int L = 0; L < NN; ++L) {
    const int cx = (L == 1 || L == 2 || L == 5 || L == 6) ? 1 : 0, cy = (L & 3) >= 2 ? 1 : 0, cz = L >= 4 ? 1 : 0;
    const int h = ((tz + (DIM == 3 ? 1 + cz : 0)) * TS::HY + (ty + 1 + cy)) * TS::HX + (tx + 1 + cx);
#pragma unroll
    for (int c = 0; c < DIM; ++c) ue[DIM * L + c] = s.v[DIM * h + c];
  }
  double ce = 0.0;
#pragma unroll(DIM == 2 ? ND : 1)
  for (int r2 = 0; r2 < ND; ++r2) {
    double t = 0.0;
#pragma unroll
    for (int c2 = r2 + 1; c2 < ND; ++c2) t = fma(ke.k[r2 * ND + c2], ue[c2], t);
    t = fma(ke.k[r2 * ND + r2], ue[r2], t + t);
    ce = fma(ue[r2], t, ce);
  }
  dc[e] = -dyoung<double>(rho[e], g.E0, g.Emin, g.ipenal) * ce;
}

template <int DIM, bool GRAD = false>
__global__ void __launch_bounds__(TileShape<DIM>::NT) residual_kernel(const __grid_constant__ ResArgs<DIM> a) {
  __shared__ TileSmem<DIM, double> s;
  __shared__ double red[32];
  const Grid& g = a.g;
  const TileCoord tc = tile_coord<DIM>(g, blockIdx.x);
  const double* rho = a.rho + blockIdx.y * a.ldr;
  const double* u = a.u + blockIdx.y * a.ldu;
  stage_E<DIM, double>(s, g, tc, [&](long long e) { return young<double>(rho[e], g.E0, g.Emin, g.ipenal); });
  stage_V<DIM, double>(s, g, tc, [&](long long dof) { return u[dof]; });
  __syncthreads();
  int tx, ty, tz;
  long long n = 0;
  double rr = 0.0, ff = 0.0;
  if (owned_node<DIM>(g, tc, tx, ty, tz, n)) {
    double out[DIM];
    node_apply<DIM, double>(s, tx, ty, tz, a.ke, out);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const long long dof = DIM * n + c;
      double rv = 0.0;
      if (!is_fixed(g, dof)) {
        const double fv = a.f[dof];
        rv = fv - out[c];
        rr = fma(rv, rv, rr);
        ff = fma(fv, fv, ff);
      }
      if (a.r) a.r[dof] = rv;
    }
    if (GRAD) tile_element_grad<DIM>(s, g, tc, tx, ty, tz, a.ke, rho, a.dc + blockIdx.y * a.ldd);
  }
  double t1 = block_sum(rr, red);
  double t2 = block_sum(ff, red);
  if (threadIdx.x == 0) {
    double* part = a.partial + (size_t)blockIdx.y * 2 * gridDim.x;
    part[blockIdx.x] = t1;
    part[gridDim.x + blockIdx.x] = t2;
  }
}

__global__ void residual_final_kernel(const double* partial, int G, double* out2) {
  __shared__ double red[32];
  partial += (size_t)blockIdx.x * 2 * G;  // one CTA per design
  out2 += 2 * blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    a += partial[i];
    b += partial[G + i];
  }
  double ta = block_sum(a, red);
  double tb = block_sum(b, red);
  if (threadIdx.x == 0) {
    out2[0] = sqrt(ta);
    out2[1] = tb > 0.0 ? sqrt(ta) / sqrt(tb) : 0.0;
  }
}

template <int DIM>
static topo_status residual_impl(topo_ctx* c, const double* rho, const double* u, const double* f, double* r,
                                 double* out2, const typename KeOf<DIM, double>::type& ke) {
  long long tiles = num_tiles<DIM>(c->g);
  topo_status s = ensure_red(c, sizeof(double) * (size_t)(2 * tiles + 64));
  if (s) return s;
  ResArgs<DIM> a;
  a.g = c->g;
  a.ke = ke;
  a.rho = rho;
  a.u = u;
  a.f = f;
  a.r = r;
  a.partial = c->d_red;
  a.ldr = a.ldu = 0;
  residual_kernel<DIM><<<(unsigned)tiles, TileShape<DIM>::NT, 0, c->stream>>>(a);
  note_launch();
  residual_final_kernel<<<1, 256, 0, c->stream>>>(c->d_red, (int)tiles, out2);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

long long residual_tiles(topo_ctx* c) {
  return c->g.dim == 2 ? num_tiles<2>(c->g) : num_tiles<3>(c->g);
}

template <int DIM>
static topo_status residual_batch_impl(topo_ctx* c, const double* rho, long long ldr, const double* U, long long ldu,
                                       const double* f, double* out2, int R, double* partial, double* dc,
                                       long long ldd, const typename KeOf<DIM, double>::type& ke) {
  const long long tiles = num_tiles<DIM>(c->g);
  ResArgs<DIM> a;
  a.g = c->g;
  a.ke = ke;
  a.rho = rho;
  a.u = U;
  a.f = f;
  a.r = nullptr;
  a.partial = partial;
  a.ldr = ldr;
  a.ldu = ldu;
  a.dc = dc;
  a.ldd = ldd;
  if (dc)
    residual_kernel<DIM, true><<<dim3((unsigned)tiles, (unsigned)R), TileShape<DIM>::NT, 0, c->stream>>>(a);
  else
    residual_kernel<DIM><<<dim3((unsigned)tiles, (unsigned)R), TileShape<DIM>::NT, 0, c->stream>>>(a);
  note_launch();
  residual_final_kernel<<<R, 256, 0, c->stream>>>(partial, (int)tiles, out2);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

topo_status launch_residual64_batch(topo_ctx* c, const double* rho, long long ldr, const double* U, long long ldu,
                                    const double* f, double* out2, int R, double* partial, double* dc, long long ldd) {
  if (c->g.dim == 2) return residual_batch_impl<2>(c, rho, ldr, U, ldu, f, out2, R, partial, dc, ldd, c->q4_64);
  return residual_batch_impl<3>(c, rho, ldr, U, ldu, f, out2, R, partial, dc, ldd, c->h8_64);
}

topo_status launch_residual64(topo_ctx* c, const double* rho, const double* u, const double* f, double* r,
                              double* out2) {
  if (c->g.dim == 2) return residual_impl<2>(c, rho, u, f, r, out2, c->q4_64);
  return residual_impl<3>(c, rho, u, f, r, out2, c->h8_64);
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_apply_K(topo_ctx* c, const double* rho, const void* V, void* Y, int m, int ld,
                                    topo_prec prec) {
  if (!c) return TOPO_ERR_INVALID;
  if (m < 0) return fail(c, TOPO_ERR_INVALID, "topo_apply_K: m < 0");
  if (m == 0) return TOPO_OK;
  if ((long long)ld < c->g.ndof) return fail(c, TOPO_ERR_INVALID, "topo_apply_K: ld < N");
  if (prec != TOPO_FP64 && prec != TOPO_FP32_REFINED && prec != TOPO_FP32_BF16KE_REFINED)
    return fail(c, TOPO_ERR_INVALID, "topo_apply_K: unknown precision");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(V) || !dev_ptr_ok(Y))
    return fail(c, TOPO_ERR_INVALID, "topo_apply_K: null or misaligned pointer");
  if (V == Y) return fail(c, TOPO_ERR_INVALID, "topo_apply_K: V and Y alias");
  return launch_apply(c, rho, V, Y, m, ld, prec);
}
