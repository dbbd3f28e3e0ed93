// Context management, the linear density filter, the compliance gradient and deterministic
// reductions of libtopo.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "common.cuh"

namespace topo {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

topo_status fail(topo_ctx* c, topo_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

topo_status cuda_fail(topo_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? TOPO_ERR_OOM : TOPO_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

bool dev_ptr_ok(const void* p) { return p != nullptr && ((uintptr_t)p % 8) == 0; }

topo_status ensure_scratch(topo_ctx* c, size_t bytes) {
  if (bytes <= c->scratch_bytes) return TOPO_OK;
  // stream-ordered: wait for users of the old buffer before freeing it
  TOPO_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->d_scratch) cudaFree(c->d_scratch);
  c->d_scratch = nullptr;
  c->scratch_bytes = 0;
  size_t b = bytes + (bytes >> 3) + 4096;
  cudaError_t e = cudaMalloc(&c->d_scratch, b);
  if (e != cudaSuccess) return cuda_fail(c, e, "scratch cudaMalloc");
  c->scratch_bytes = b;
  c->scratch_gen += 1;
  return TOPO_OK;
}

topo_status ensure_red(topo_ctx* c, size_t bytes) {
  if (bytes <= c->red_bytes) return TOPO_OK;
  TOPO_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->d_red) cudaFree(c->d_red);
  c->d_red = nullptr;
  c->red_bytes = 0;
  cudaError_t e = cudaMalloc(&c->d_red, bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduction cudaMalloc");
  c->red_bytes = bytes;
  return TOPO_OK;
}

// ---------------------------------------------------------------------------------------
// Unit-density element stiffness by 2-point Gauss quadrature per direction (exact for Q1
// on a unit square / cube). Plane stress in 2D, isotropic Lame form in 3D.
// ---------------------------------------------------------------------------------------
static void element_stiffness(int dim, double nu, double* K) {
  const int nn = dim == 2 ? 4 : 8, nd = dim * nn, ns = dim == 2 ? 3 : 6;
  double D[36] = {0};
  if (dim == 2) {
    double f = 1.0 / (1.0 - nu * nu);
    D[0] = f;
    D[1] = f * nu;
    D[3] = f * nu;
    D[4] = f;
    D[8] = f * (1.0 - nu) / 2.0;
  } else {
    double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D[a * 6 + b] = lam;
    for (int a = 0; a < 3; ++a) {
      D[a * 6 + a] = lam + 2.0 * mu;
      D[(a + 3) * 6 + a + 3] = mu;
    }
  }
  const int cx[8] = {0, 1, 1, 0, 0, 1, 1, 0}, cy[8] = {0, 0, 1, 1, 0, 0, 1, 1}, cz[8] = {0, 0, 0, 0, 1, 1, 1, 1};
  const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  const double wq = dim == 2 ? 0.25 : 0.125;
  for (int i = 0; i < nd * nd; ++i) K[i] = 0.0;
  const int nz = dim == 2 ? 1 : 2;
  for (int qz = 0; qz < nz; ++qz)
    for (int qy = 0; qy < 2; ++qy)
      for (int qx = 0; qx < 2; ++qx) {
        double x[3] = {gp[qx], gp[qy], dim == 3 ? gp[qz] : 0.0};
        double dN[8][3];
        for (int a = 0; a < nn; ++a) {
          int c[3] = {cx[a], cy[a], cz[a]};
          for (int d = 0; d < dim; ++d) {
            double v = 1.0;
            for (int e = 0; e < dim; ++e) {
              if (e == d)
                v *= c[e] ? 1.0 : -1.0;
              else
                v *= c[e] ? x[e] : 1.0 - x[e];
            }
            dN[a][d] = v;
          }
        }
        double B[6][24] = {{0}};
        for (int a = 0; a < nn; ++a) {
          if (dim == 2) {
            B[0][2 * a] = dN[a][0];
            B[1][2 * a + 1] = dN[a][1];
            B[2][2 * a] = dN[a][1];
            B[2][2 * a + 1] = dN[a][0];
          } else {
            int o = 3 * a;
            B[0][o] = dN[a][0];
            B[1][o + 1] = dN[a][1];
            B[2][o + 2] = dN[a][2];
            B[3][o] = dN[a][1];
            B[3][o + 1] = dN[a][0];
            B[4][o + 1] = dN[a][2];
            B[4][o + 2] = dN[a][1];
            B[5][o] = dN[a][2];
            B[5][o + 2] = dN[a][0];
          }
        }
        for (int i = 0; i < nd; ++i)
          for (int j = 0; j < nd; ++j) {
            double s = 0.0;
            for (int a = 0; a < ns; ++a)
              for (int b = 0; b < ns; ++b) s += B[a][i] * D[(dim == 2 ? a * 3 : a * 6) + b] * B[b][j];
            K[i * nd + j] += wq * s;
          }
      }
}

// Round to the nearest BF16 value (ties to even) and widen back to FP32.
static float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------------------------------
// Kernels: filter normaliser, filter forward / adjoint, compliance gradient, sums.
// ---------------------------------------------------------------------------------------
struct FilterArgs {
  Grid g;
  const int* off;   // [ns * 3]
  const double* w;  // [ns]
  int ns;
  const double* Hsinv;  // 1 / Hs_e
  const double* in;
  double* out;
  int mode;  // 0 = 1 / Hs, 1 = forward, 2 = adjoint
  long long ldin, ldout;  // strides between the fields of blockIdx.y (several fields per launch)
};

__global__ void filter_kernel(const __grid_constant__ FilterArgs a) {
  extern __shared__ unsigned char smem_raw[];
  int* soff = reinterpret_cast<int*>(smem_raw);
  double* sw = reinterpret_cast<double*>(smem_raw + ((a.ns * 3 * sizeof(int) + 15) & ~15));
  for (int i = threadIdx.x; i < a.ns * 3; i += blockDim.x) soff[i] = a.off[i];
  for (int i = threadIdx.x; i < a.ns; i += blockDim.x) sw[i] = a.w[i];
  __syncthreads();
  const Grid& g = a.g;
  const double* in = a.in + blockIdx.y * a.ldin;
  double* out = a.out + blockIdx.y * a.ldout;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.nel; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % g.nx);
    long long r = e / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    double acc = 0.0;
    for (int s = 0; s < a.ns; ++s) {
      int ii = i + soff[3 * s], jj = j + soff[3 * s + 1], kk = k + soff[3 * s + 2];
      if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.ny || kk < 0 || kk >= g.nz) continue;
      long long en = ii + (long long)g.nx * (jj + (long long)g.ny * kk);
      double v;
      if (a.mode == 0)
        v = 1.0;
      else if (a.mode == 1)
        v = in[en];
      else
        v = in[en] * a.Hsinv[en];  // FP64 division is slow here: multiply by 1 / Hs
      acc = fma(sw[s], v, acc);
    }
    if (a.mode == 0) acc = 1.0 / acc;  // once per context
    if (a.mode == 1) acc *= a.Hsinv[e];
    out[e] = acc;
  }
}

// Element energies and the compliance gradient: dc_e = -E'(rho_e) sum_c u_{c,e}^T K_e u_{c,e}.
template <int DIM>
struct GradArgs {
  Grid g;
  typename KeOf<DIM, double>::type ke;
  const double* rho;
  const double* U;
  long long ld;
  int m;
  double* dc;
  long long ldr, ldu, ldd;  // strides of rho, U and dc between the designs of blockIdx.y
  const double* Lam;        // adjoint states (N x m at ld) for a general output; null: compliance
};

template <int DIM>
__global__ void grad_kernel(const __grid_constant__ GradArgs<DIM> a) {
  constexpr int NN = DIM == 2 ? 4 : 8, ND = DIM * NN;
  const Grid& g = a.g;
  const double* rho = a.rho + blockIdx.y * a.ldr;
  const double* U = a.U + blockIdx.y * a.ldu;
  double* dc = a.dc + blockIdx.y * a.ldd;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.nel; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % g.nx);
    long long r = e / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    long long dofs[ND];
#pragma unroll
    for (int L = 0; L < NN; ++L) {
      const int cxa[8] = {0, 1, 1, 0, 0, 1, 1, 0}, cya[8] = {0, 0, 1, 1, 0, 0, 1, 1}, cza[8] = {0, 0, 0, 0, 1, 1, 1, 1};
      long long n = (i + cxa[L]) + (long long)g.nnx * ((j + cya[L]) + (long long)g.nny * (DIM == 3 ? k + cza[L] : 0));
#pragma unroll
      for (int c = 0; c < DIM; ++c) dofs[DIM * L + c] = DIM * n + c;
    }
    double ce = 0.0;
    for (int col = 0; col < a.m; ++col) {
      const double* u = U + (long long)col * a.ld;
      double ue[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) ue[d] = is_fixed(g, dofs[d]) ? 0.0 : u[dofs[d]];
      if (a.Lam) {  // a general output: the mixed form lambda_e^T K_e u_e
        const double* lam = a.Lam + (long long)col * a.ld;
#pragma unroll(DIM == 2 ? ND : 1)
        for (int r2 = 0; r2 < ND; ++r2) {
          if (is_fixed(g, dofs[r2])) continue;
          double t = 0.0;
#pragma unroll
          for (int c2 = 0; c2 < ND; ++c2) t = fma(a.ke.k[r2 * ND + c2], ue[c2], t);
          ce = fma(lam[dofs[r2]], t, ce);
        }
        continue;
      }
      // u_e^T K_e u_e in the symmetric form: row r2 sums K_e's entries right of the diagonal,
      // doubles that (exactly) and adds the diagonal term, ND (ND + 1) / 2 products instead of ND^2
#pragma unroll(DIM == 2 ? ND : 1)
      for (int r2 = 0; r2 < ND; ++r2) {
        double t = 0.0;
#pragma unroll
        for (int c2 = r2 + 1; c2 < ND; ++c2) t = fma(a.ke.k[r2 * ND + c2], ue[c2], t);
        t = fma(a.ke.k[r2 * ND + r2], ue[r2], t + t);
        ce = fma(ue[r2], t, ce);
      }
    }
    dc[e] = -dyoung<double>(rho[e], g.E0, g.Emin, g.ipenal) * ce;
  }
}

// Deterministic two-pass dot / sum. Pass 1: block b sums the fixed index set
// {b*256 + t + s*G*256}. Pass 2: one block sums the G partials in index order.
__global__ void dot_partial_kernel(const double* x, const double* y, long long n, double* partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc = y ? fma(x[i], y[i], acc) : acc + x[i];
  double t = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void sum_final_kernel(const double* partial, int G, double* out, int sqrt_out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) acc += partial[i];
  double t = block_sum(acc, red);
  if (threadIdx.x == 0) out[0] = sqrt_out ? sqrt(t) : t;
}

static int red_blocks(topo_ctx* c, long long n) {
  long long b = (n + 255) / 256;
  long long cap = 2LL * c->num_sms;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

topo_status launch_sum(topo_ctx* c, const double* x, long long n, double* out) {
  int G = red_blocks(c, n);
  topo_status s = ensure_red(c, sizeof(double) * (size_t)(G + 64));
  if (s) return s;
  dot_partial_kernel<<<G, 256, 0, c->stream>>>(x, nullptr, n, c->d_red);
  note_launch();
  sum_final_kernel<<<1, 256, 0, c->stream>>>(c->d_red, G, out, 0);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

// J = sum over columns of f_c^T u_c: one pass-1 launch per column into consecutive partial
// slots, then a single final sum over all slots (fixed order).
__global__ void dot_cols_partial_kernel(const double* F, const double* U, long long n, long long ld, int m,
                                        double* partial) {
  __shared__ double red[32];
  // blockIdx.y = column
  const double* f = F + (long long)blockIdx.y * ld;
  const double* u = U + (long long)blockIdx.y * ld;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc = fma(f[i], u[i], acc);
  double t = block_sum(acc, red);
  if (threadIdx.x == 0) partial[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

static topo_status filter_launch(topo_ctx* c, const double* in, double* out, int mode, int R = 1,
                                 long long ldin = 0, long long ldout = 0) {
  if (mode != 0 && c->filter_kind == 1)  // the Helmholtz filter is its own adjoint
    return helmholtz_apply(c, in, R > 1 ? ldin : c->g.nel, out, R > 1 ? ldout : c->g.nel, R);
  FilterArgs a;
  a.ldin = ldin;
  a.ldout = ldout;
  a.g = c->g;
  a.off = c->d_stencil_off;
  a.w = c->d_stencil_w;
  a.ns = c->nstencil;
  a.Hsinv = c->d_Hsinv;
  a.in = in;
  a.out = out;
  a.mode = mode;
  size_t sm = ((a.ns * 3 * sizeof(int) + 15) & ~(size_t)15) + a.ns * sizeof(double);
  long long blocks = (c->g.nel + 255) / 256;
  if (blocks > 8LL * c->num_sms) blocks = 8LL * c->num_sms;
  if (R > 1) blocks = std::max(1LL, std::min(blocks, (8LL * c->num_sms + R - 1) / R));
  filter_kernel<<<dim3((unsigned)blocks, (unsigned)R), 256, sm, c->stream>>>(a);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

// The filter (forward or adjoint) of R fields in one launch: field r at in + r ldin -> out + r ldout.
topo_status launch_filter_batch(topo_ctx* c, const double* in, long long ldin, double* out, long long ldout, int R,
                                int adjoint) {
  return filter_launch(c, in, out, adjoint ? 2 : 1, R, ldin, ldout);
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_create(const topo_problem* prob, void* cuda_stream, topo_ctx** out) {
  if (!out) return TOPO_ERR_INVALID;
  *out = nullptr;
  if (!prob) return TOPO_ERR_INVALID;
  const topo_problem& p = *prob;
  if (!(p.dim == 2 || p.dim == 3) || p.nx < 1 || p.ny < 1 || (p.dim == 3 && p.nz < 1)) return TOPO_ERR_INVALID;
  if (!(p.E0 > p.Emin) || !(p.Emin >= 0.0) || !(p.nu >= 0.0 && p.nu < 0.5)) return TOPO_ERR_INVALID;
  int ip = (int)p.penal;
  if ((double)ip != p.penal || ip < 1 || ip > 6) return TOPO_ERR_INVALID;
  if (!(p.rmin > 0.0 && p.rmin <= 6.0)) return TOPO_ERR_INVALID;
  if (!p.fixed_dof_mask) return TOPO_ERR_INVALID;
  const int nz = p.dim == 3 ? p.nz : 1;
  long long nnodes = (long long)(p.nx + 1) * (p.ny + 1) * (p.dim == 3 ? nz + 1 : 1);
  long long ndof = p.dim * nnodes;
  if (ndof >= (1LL << 31)) return TOPO_ERR_INVALID;

  topo_ctx* c = (topo_ctx*)calloc(1, sizeof(topo_ctx));
  if (!c) return TOPO_ERR_OOM;
  c->stream = (cudaStream_t)cuda_stream;
  c->E0 = p.E0;
  c->Emin = p.Emin;
  c->nu = p.nu;
  c->penal = p.penal;
  c->rmin = p.rmin;
  c->ipenal = ip;
  c->inner_rtol = 1e-5;
  c->max_outer = 30;
  c->wait_cycles = 2000000000LL;
  c->rom_tensor = 1;
  c->rom_asm_tensor = 1;
  c->apply_stages = 3;
  c->pcg_poly = 0;
  c->pcg_mg = 1;
  c->mg_deg = 2;
  c->mg_single_nodes = -1;
  c->rom_refine = 8;
  c->pcg_blocks_per_sm = 0;
  c->inner_cap = 2000;
  c->hdm_kernel = 0;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->num_sms <= 0) c->num_sms = 1;

  Grid& g = c->g;
  g.dim = p.dim;
  g.nx = p.nx;
  g.ny = p.ny;
  g.nz = nz;
  g.nnx = p.nx + 1;
  g.nny = p.ny + 1;
  g.nnz = p.dim == 3 ? nz + 1 : 1;
  g.nnodes = nnodes;
  g.ndof = ndof;
  g.nel = (long long)p.nx * p.ny * nz;
  g.E0 = p.E0;
  g.Emin = p.Emin;
  g.ipenal = ip;

  // Dirichlet bitmask
  size_t nwords = (size_t)((ndof + 31) / 32);
  std::vector<uint32_t> bits(nwords, 0u);
  for (long long d = 0; d < ndof; ++d)
    if (p.fixed_dof_mask[d]) bits[d >> 5] |= 1u << (d & 31);
  cudaError_t e = cudaMalloc(&c->d_fixed_bits, nwords * sizeof(uint32_t));
  if (e != cudaSuccess) {
    topo_destroy(c);
    return TOPO_ERR_OOM;
  }
  cudaMemcpy(c->d_fixed_bits, bits.data(), nwords * sizeof(uint32_t), cudaMemcpyHostToDevice);
  g.fixed_bits = c->d_fixed_bits;
  std::vector<int> flist;
  for (long long d = 0; d < ndof; ++d)
    if (p.fixed_dof_mask[d]) flist.push_back((int)d);
  c->nfixed = (int)flist.size();
  e = cudaMalloc(&c->d_fixed_list, std::max<size_t>(1, flist.size()) * sizeof(int));
  if (e != cudaSuccess) {
    topo_destroy(c);
    return TOPO_ERR_OOM;
  }
  if (!flist.empty()) cudaMemcpy(c->d_fixed_list, flist.data(), flist.size() * sizeof(int), cudaMemcpyHostToDevice);

  // element matrices in three arithmetic forms
  double K[576];
  element_stiffness(p.dim, p.nu, K);
  const int nke = p.dim == 2 ? 64 : 576;
  // BF16 form: if K_e = s * N with N an integer matrix of entries |N| <= 256 (exactly
  // representable in BF16), store N and fold s into each element's modulus; otherwise
  // round every entry to BF16 (s = 1).
  c->bf_scale = 1.0;
  c->bf_exact = 0;
  for (int n = 1; n <= 256 && !c->bf_exact; ++n) {
    const double s = K[0] / n;
    bool ok = true;
    for (int i = 0; i < nke && ok; ++i) {
      const double q = K[i] / s, r = nearbyint(q);
      ok = fabs(q - r) < 1e-9 && fabs(r) <= 256.0;
    }
    if (ok) {
      c->bf_exact = 1;
      c->bf_scale = s;
    }
  }
  for (int i = 0; i < nke; ++i) {
    const float bf = c->bf_exact ? round_bf16((float)nearbyint(K[i] / c->bf_scale)) : round_bf16((float)K[i]);
    if (p.dim == 2) {
      c->q4_64.k[i] = K[i];
      c->q4_32.k[i] = (float)K[i];
      c->q4_bf.k[i] = bf;
    } else {
      c->h8_64.k[i] = K[i];
      c->h8_32.k[i] = (float)K[i];
      c->h8_bf.k[i] = bf;
    }
  }

  // filter stencil: all offsets with positive cone weight
  std::vector<int> off;
  std::vector<double> w;
  int R = (int)ceil(p.rmin);
  int RZ = p.dim == 3 ? R : 0;
  for (int dz = -RZ; dz <= RZ; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        double wt = p.rmin - sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (wt > 0.0) {
          off.push_back(dx);
          off.push_back(dy);
          off.push_back(dz);
          w.push_back(wt);
        }
      }
  c->nstencil = (int)w.size();
  e = cudaMalloc(&c->d_stencil_off, off.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_stencil_w, w.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_Hsinv, g.nel * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_sync, sizeof(GridSync));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_bar, sizeof(GridBar));
  if (e != cudaSuccess) {
    topo_destroy(c);
    return TOPO_ERR_OOM;
  }
  cudaMemcpy(c->d_stencil_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_stencil_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(c->d_sync, 0, sizeof(GridSync));
  cudaMemset(c->d_bar, 0, sizeof(GridBar));
  topo_status s = filter_launch(c, nullptr, c->d_Hsinv, 0);
  if (s == TOPO_OK) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = TOPO_ERR_CUDA;
  }
  if (s != TOPO_OK) {
    topo_destroy(c);
    return s;
  }
  *out = c;
  return TOPO_OK;
}

extern "C" topo_status topo_destroy(topo_ctx* c) {
  if (!c) return TOPO_OK;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  cudaFree(c->d_fixed_bits);
  cudaFree(c->d_fixed_list);
  cudaFree(c->d_stencil_off);
  cudaFree(c->d_stencil_w);
  cudaFree(c->d_Hsinv);
  cudaFree(c->d_sync);
  cudaFree(c->d_bar);
  cudaFree(c->d_scratch);
  cudaFree(c->d_red);
  cudaFree(c->d_helm);
  free(c);
  return TOPO_OK;
}

extern "C" const char* topo_last_error(const topo_ctx* c) { return c ? c->err : "null context"; }

extern "C" topo_status topo_set_param(topo_ctx* c, topo_param which, double v) {
  if (!c) return TOPO_ERR_INVALID;
  switch (which) {
    case TOPO_PARAM_INNER_RTOL:
      if (!(v > 0 && v < 1)) return fail(c, TOPO_ERR_INVALID, "inner rtol must be in (0,1)");
      c->inner_rtol = v;
      return TOPO_OK;
    case TOPO_PARAM_MAX_OUTER:
      if (!(v >= 1 && v <= 1000)) return fail(c, TOPO_ERR_INVALID, "max outer must be in [1,1000]");
      c->max_outer = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_WAIT_CYCLES:
      if (!(v >= 1e3 && v <= 1e11)) return fail(c, TOPO_ERR_INVALID, "wait cycles out of range");
      c->wait_cycles = (long long)v;
      return TOPO_OK;
    case TOPO_PARAM_ROM_REFINE:
      if (!(v >= 0 && v <= 100)) return fail(c, TOPO_ERR_INVALID, "rom refine out of range");
      c->rom_refine = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_TILE_X:
      if (!(v >= 0 && v <= 1e6)) return fail(c, TOPO_ERR_INVALID, "apply columns per CTA must be in [0,1e6]");
      c->apply_cols = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_INNER_CAP:
      if (!(v >= 1 && v <= 1e7)) return fail(c, TOPO_ERR_INVALID, "inner cap must be in [1,1e7]");
      c->inner_cap = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_PCG_MAX_CTAS:
      if (!(v >= 0 && v <= 1e6)) return fail(c, TOPO_ERR_INVALID, "max CTAs must be in [0,1e6]");
      c->pcg_max_ctas = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_HDM_KERNEL:
      if (!(v == 0 || v == 1)) return fail(c, TOPO_ERR_INVALID, "hdm kernel must be 0 or 1");
      c->hdm_kernel = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_ROM_TENSOR:
      if (!(v == 0 || v == 1)) return fail(c, TOPO_ERR_INVALID, "rom tensor must be 0 or 1");
      c->rom_tensor = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_ROM_ASSEMBLY:
      if (!(v == 0 || v == 1)) return fail(c, TOPO_ERR_INVALID, "rom assembly must be 0 or 1");
      c->rom_asm_tensor = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_APPLY_STAGES:
      if (!(v == 0 || v == 2 || v == 3 || v == 4)) return fail(c, TOPO_ERR_INVALID, "apply stages must be 0, 2, 3 or 4");
      c->apply_stages = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_PCG_POLY:
      if (!(v >= 0 && v <= 8 && v == (int)v)) return fail(c, TOPO_ERR_INVALID, "pcg poly must be an integer in [0,8]");
      c->pcg_poly = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_PCG_MG:
      if (!(v == 0 || v == 1)) return fail(c, TOPO_ERR_INVALID, "pcg mg must be 0 or 1");
      c->pcg_mg = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_MG_DEGREE:
      if (!(v >= 1 && v <= 4 && v == (int)v)) return fail(c, TOPO_ERR_INVALID, "mg degree must be an integer in [1,4]");
      c->mg_deg = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_MG_SINGLE_NODES:
      if (!(v >= -1 && v <= 1e9 && v == (long long)v))
        return fail(c, TOPO_ERR_INVALID, "mg single-CTA node count must be an integer in [-1,1e9]");
      c->mg_single_nodes = (long long)v;
      return TOPO_OK;
    case TOPO_PARAM_FILTER:
      if (!(v == 0 || v == 1)) return fail(c, TOPO_ERR_INVALID, "filter must be 0 (cone) or 1 (Helmholtz)");
      c->filter_kind = (int)v;
      return TOPO_OK;
    case TOPO_PARAM_HELMHOLTZ_R:
      if (!(v >= 0 && v <= 1e4)) return fail(c, TOPO_ERR_INVALID, "Helmholtz length must be in [0,1e4]");
      c->helm_r = v;
      return TOPO_OK;
    case TOPO_PARAM_PCG_BLOCKS_PER_SM:
      if (!(v >= 0 && v <= 8)) return fail(c, TOPO_ERR_INVALID, "blocks per SM must be in [0,8]");
      c->pcg_blocks_per_sm = (int)v;
      return TOPO_OK;
  }
  return fail(c, TOPO_ERR_INVALID, "unknown parameter %d", (int)which);
}

extern "C" topo_status topo_check(topo_ctx* c) {
  if (!c) return TOPO_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "topo_check: stream");
  int st = 0;
  e = cudaMemcpy(&st, &c->d_sync->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "topo_check: status");
  if (st != 0) {
    int zero = 0;
    cudaMemcpy(&c->d_sync->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return fail(c, (topo_status)st, "device status %d", st);
  }
  return TOPO_OK;
}

extern "C" topo_status topo_sizes(const topo_ctx* c, long long* ndof, long long* nel, long long* nnodes) {
  if (!c) return TOPO_ERR_INVALID;
  if (ndof) *ndof = c->g.ndof;
  if (nel) *nel = c->g.nel;
  if (nnodes) *nnodes = c->g.nnodes;
  return TOPO_OK;
}

extern "C" topo_status topo_filter(topo_ctx* c, const double* in, double* out, int adjoint) {
  if (!c) return TOPO_ERR_INVALID;
  if (!dev_ptr_ok(in) || !dev_ptr_ok(out) || in == out)
    return fail(c, TOPO_ERR_INVALID, "topo_filter: null, misaligned or aliased pointers");
  return filter_launch(c, in, out, adjoint ? 2 : 1);
}

// J = sum_c l_c^T u_c, dc_rho_e = -E'(rho_e) sum_c w_{c,e}^T K_e u_{c,e} with w = Lam (a general
// output) or w = u (compliance, Lam null), and the filter adjoint of dc_rho.
static topo_status output_grad_impl(topo_ctx* c, const double* rho, const double* U, const double* Lam, int m,
                                    int ld, const double* L, double* J, double* dc_rho, double* dc_psi,
                                    const char* what) {
  const Grid& g = c->g;
  if (m < 1 || (long long)ld < g.ndof) return fail(c, TOPO_ERR_INVALID, "%s: m >= 1 and ld >= N required", what);
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(U) || !dev_ptr_ok(L) || !dev_ptr_ok(J) || !dev_ptr_ok(dc_rho) ||
      (dc_psi && !dev_ptr_ok(dc_psi)) || (Lam && !dev_ptr_ok(Lam)))
    return fail(c, TOPO_ERR_INVALID, "%s: null or misaligned pointer", what);
  // J = sum_c l_c^T u_c (fixed order)
  int G = red_blocks(c, g.ndof);
  topo_status s = ensure_red(c, sizeof(double) * (size_t)(G * m + 64));
  if (s) return s;
  dot_cols_partial_kernel<<<dim3(G, m), 256, 0, c->stream>>>(L, U, g.ndof, ld, m, c->d_red);
  note_launch();
  sum_final_kernel<<<1, 256, 0, c->stream>>>(c->d_red, G * m, J, 0);
  note_launch();
  long long blocks = (g.nel + 127) / 128;
  if (blocks > 16LL * c->num_sms) blocks = 16LL * c->num_sms;
  if (g.dim == 2) {
    GradArgs<2> a;
    a.g = g;
    a.ke = c->q4_64;
    a.rho = rho;
    a.U = U;
    a.ld = ld;
    a.m = m;
    a.dc = dc_rho;
    a.ldr = a.ldu = a.ldd = 0;
    a.Lam = Lam;
    grad_kernel<2><<<(int)blocks, 128, 0, c->stream>>>(a);
    note_launch();
  } else {
    GradArgs<3> a;
    a.g = g;
    a.ke = c->h8_64;
    a.rho = rho;
    a.U = U;
    a.ld = ld;
    a.m = m;
    a.dc = dc_rho;
    a.ldr = a.ldu = a.ldd = 0;
    a.Lam = Lam;
    grad_kernel<3><<<(int)blocks, 128, 0, c->stream>>>(a);
    note_launch();
  }
  TOPO_CUDA_TRY(c, cudaGetLastError());
  if (dc_psi) return filter_launch(c, dc_rho, dc_psi, 2);
  return TOPO_OK;
}

extern "C" topo_status topo_compliance_grad(topo_ctx* c, const double* rho, const double* U, int m, int ld,
                                            const double* F, double* J, double* dc_rho, double* dc_psi) {
  if (!c) return TOPO_ERR_INVALID;
  return output_grad_impl(c, rho, U, nullptr, m, ld, F, J, dc_rho, dc_psi, "compliance_grad");
}

extern "C" topo_status topo_output_grad(topo_ctx* c, const double* rho, const double* U, const double* Lam, int m,
                                        int ld, const double* L, double* J, double* dc_rho, double* dc_psi) {
  if (!c) return TOPO_ERR_INVALID;
  if (!Lam) return fail(c, TOPO_ERR_INVALID, "topo_output_grad: null adjoint states");
  return output_grad_impl(c, rho, U, Lam, m, ld, L, J, dc_rho, dc_psi, "topo_output_grad");
}

extern "C" topo_status topo_launch_count(long long* out) {
  if (!out) return TOPO_ERR_INVALID;
  *out = topo::g_launches.load(std::memory_order_relaxed);
  return TOPO_OK;
}
