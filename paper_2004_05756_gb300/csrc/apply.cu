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
  long long tiles = num_tiles<DIM>(c->g);
  // enough CTAs to fill the GPU several times over, each reusing its staged E for a run
  // of columns
  long long want_ctas = 8LL * c->num_sms;
  long long groups = (want_ctas + tiles - 1) / tiles;
  if (groups > m) groups = m;
  if (groups < 1) groups = 1;
  if (groups > 65535) groups = 65535;
  a.cols_per_cta = (int)((m + groups - 1) / groups);
  groups = (m + a.cols_per_cta - 1) / a.cols_per_cta;
  dim3 grid((unsigned)tiles, (unsigned)groups);
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
