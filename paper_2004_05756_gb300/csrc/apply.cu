// Matrix-free K(rho) V (Section 2.1, Eq. linelast-res1) and the FP64 residual
// r = f - K(rho) u with its norms (Section 3.3).
//
// One CTA per node tile; the element moduli of the tile are staged once and reused for
// every column the CTA processes; each column's halo'd node box is staged in shared memory
// with coalesced loads (Dirichlet DOFs zeroed), then every thread forms its node's rows.
#include "common.cuh"

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

template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;  // 0: the BYTES destination bytes are zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(n) : "memory");
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
  T C[9][4];
  {
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
      issue(b + 2, buf == 0 ? 2 : buf - 1);  // the buffer after the next one
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
        T y0 = (T)0, y1 = (T)0;
#pragma unroll
        for (int nb = 0; nb < 9; ++nb) {
          const V2 t = sb[col * HB + (nb / 3) * HX + (nb % 3)];
          y0 = fma(C[nb][0], t.x, y0);
          y0 = fma(C[nb][1], t.y, y0);
          y1 = fma(C[nb][2], t.x, y1);
          y1 = fma(C[nb][3], t.y, y1);
        }
        V2 o;
        o.x = y0;
        o.y = y1;
        ybase[(long long)(cb + col) * pitch] = o;
      }
    }
    __syncthreads();  // the buffer of batch b is refilled by batch b + 3
    buf = buf == 2 ? 0 : buf + 1;
  }
}

template <typename T>
constexpr size_t apply2_smem_bytes() {
  return 3 * (32 / sizeof(T)) * 340 * 2 * sizeof(T);
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
// ---------------------------------------------------------------------------------------
template <int DIM>
struct ResArgs {
  Grid g;
  typename KeOf<DIM, double>::type ke;
  const double* rho;
  const double* u;
  const double* f;
  double* r;        // may be null
  double* partial;  // [2 * G]
};

template <int DIM>
__global__ void __launch_bounds__(TileShape<DIM>::NT) residual_kernel(const __grid_constant__ ResArgs<DIM> a) {
  __shared__ TileSmem<DIM, double> s;
  __shared__ double red[32];
  const Grid& g = a.g;
  const TileCoord tc = tile_coord<DIM>(g, blockIdx.x);
  stage_E<DIM, double>(s, g, tc, [&](long long e) { return young<double>(a.rho[e], g.E0, g.Emin, g.ipenal); });
  stage_V<DIM, double>(s, g, tc, [&](long long dof) { return a.u[dof]; });
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
  }
  double t1 = block_sum(rr, red);
  double t2 = block_sum(ff, red);
  if (threadIdx.x == 0) {
    a.partial[blockIdx.x] = t1;
    a.partial[gridDim.x + blockIdx.x] = t2;
  }
}

__global__ void residual_final_kernel(const double* partial, int G, double* out2) {
  __shared__ double red[32];
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
  residual_kernel<DIM><<<(unsigned)tiles, TileShape<DIM>::NT, 0, c->stream>>>(a);
  note_launch();
  residual_final_kernel<<<1, 256, 0, c->stream>>>(c->d_red, (int)tiles, out2);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
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
