// Reduced stiffness from per-element reduced matrices.
//
// Eq. hatkbm writes the reduced stiffness as H(rho) = sum_e E(rho_e) (P_e^T Phi)^T K_e (P_e^T Phi)
// and Remark rom_assemble notes that each term is a dense k x k product. The paper forms the
// sum anew for every density (2 ndof_e k^2 N_e flops, Section 3.4). Here the rho-independent
// factors Hel_e = (P_e^T Phi)^T K_e (P_e^T Phi) are computed once per basis and kept in HBM;
// every new density then costs one streaming weighted reduction over the elements,
// H(rho) = sum_e E(rho_e) Hel_e (k(k+1)/2 FMAs and as many stored words per element).
//
// Layout: Hel is (N_e + 1) rows of npair = k(k+1)/2 FP64 words (upper triangle, row-major
// packed). Row N_e holds Phi_D^T Phi_D over the Dirichlet DOFs: the identity rows/columns of
// the operator convention, so that H matches Phi^T K(rho) Phi exactly for any Phi.
#include <algorithm>

#include "common.cuh"

namespace topo {

template <int DIM>
struct ElemArgs {
  Grid g;
  typename KeOf<DIM, double>::type ke;
  const double* Phi;
  long long ld;
  int k, npair, EB;
  double* Hel;
};

// One CTA per EB elements: gather Phi_e (ndof_e x k) into shared memory (Dirichlet rows as
// zero), W_e = K_e Phi_e, then every upper-triangle entry Phi_e^T W_e, stored coalesced.
template <int DIM>
__global__ void __launch_bounds__(256) rom_elem_kernel(const __grid_constant__ ElemArgs<DIM> a) {
  constexpr int NN = DIM == 2 ? 4 : 8, ND = DIM * NN;
  extern __shared__ double sm[];
  const int k = a.k, npair = a.npair;
  double* P = sm;                       // [EB][ND][k]
  double* W = sm + (size_t)a.EB * ND * k;  // [EB][ND][k]
  unsigned char* pi = reinterpret_cast<unsigned char*>(W + (size_t)a.EB * ND * k);
  unsigned char* pj = pi + npair;
  const Grid& g = a.g;
  const long long e0 = (long long)blockIdx.x * a.EB;
  const int nE = (int)min((long long)a.EB, g.nel - e0);
  // pair table (i <= j), row-major upper triangle
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int base = i * k - i * (i - 1) / 2;
    for (int j = i; j < k; ++j) {
      pi[base + j - i] = (unsigned char)i;
      pj[base + j - i] = (unsigned char)j;
    }
  }
  const int cxa[8] = {0, 1, 1, 0, 0, 1, 1, 0}, cya[8] = {0, 0, 1, 1, 0, 0, 1, 1}, cza[8] = {0, 0, 0, 0, 1, 1, 1, 1};
  for (int idx = threadIdx.x; idx < nE * ND * k; idx += blockDim.x) {
    const int j = idx / (nE * ND);
    const int r = idx % (nE * ND);
    const int el = r / ND, ad = r % ND;
    const int L = ad / DIM, comp = ad % DIM;
    const long long e = e0 + el;
    const int i = (int)(e % g.nx);
    const long long rest = e / g.nx;
    const int jj = (int)(rest % g.ny), kk = (int)(rest / g.ny);
    const long long n = (i + cxa[L]) + (long long)g.nnx * ((jj + cya[L]) + (long long)g.nny * (DIM == 3 ? kk + cza[L] : 0));
    const long long dof = DIM * n + comp;
    P[((size_t)el * ND + ad) * k + j] = is_fixed(g, dof) ? 0.0 : a.Phi[(long long)j * a.ld + dof];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nE * ND * k; idx += blockDim.x) {
    const int el = idx / (ND * k), rem = idx % (ND * k), r = rem / k, j = rem % k;
    const double* pc = P + (size_t)el * ND * k + j;
    double acc = 0.0;
#pragma unroll 8
    for (int b = 0; b < ND; ++b) acc = fma(a.ke.k[r * ND + b], pc[(size_t)b * k], acc);
    W[((size_t)el * ND + r) * k + j] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nE * npair; idx += blockDim.x) {
    const int el = idx / npair, p = idx % npair;
    const int i = pi[p], j = pj[p];
    const double* pe = P + (size_t)el * ND * k;
    const double* we = W + (size_t)el * ND * k;
    double acc = 0.0;
#pragma unroll 8
    for (int r = 0; r < ND; ++r) acc = fma(pe[r * k + i], we[r * k + j], acc);
    a.Hel[(size_t)(e0 + el) * npair + p] = acc;
  }
}

// Row N_e: Phi_D^T Phi_D over the Dirichlet DOFs (fixed order, one thread per entry).
__global__ void rom_elem_dirichlet_kernel(const double* Phi, long long ld, int k, const int* fixed_list, int nfixed,
                                          double* row) {
  const int npair = k * (k + 1) / 2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npair; p += gridDim.x * blockDim.x) {
    int i = 0, rem = p;
    while (rem >= k - i) {
      rem -= k - i;
      ++i;
    }
    const int j = i + rem;
    double acc = 0.0;
    for (int t = 0; t < nfixed; ++t) {
      const long long d = fixed_list[t];
      acc = fma(Phi[(long long)i * ld + d], Phi[(long long)j * ld + d], acc);
    }
    row[p] = acc;
  }
}

// E(rho_e) for all elements, plus weight 1 for the Dirichlet row.
__global__ void elem_moduli_kernel(Grid g, const double* rho, double* E) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e <= g.nel; e += (long long)gridDim.x * blockDim.x)
    E[e] = e < g.nel ? young<double>(rho[e], g.E0, g.Emin, g.ipenal) : 1.0;
}

// partial[blockIdx.x][p] = sum over the CTA's element rows of E_e Hel[e][p]; grid.y covers p.
__global__ void __launch_bounds__(256) rom_assemble_partial_kernel(const double* __restrict__ Hel,
                                                                   const double* __restrict__ E, long long rows,
                                                                   int npair, long long rows_per_cta,
                                                                   double* partial) {
  const int p = blockIdx.y * blockDim.x + threadIdx.x;
  const long long r0 = blockIdx.x * rows_per_cta;
  const long long r1 = min(rows, r0 + rows_per_cta);
  if (p >= npair) return;
  // eight interleaved accumulators (fixed order) keep eight streaming loads in flight
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  long long r = r0;
  for (; r + 7 < r1; r += 8) {
    double h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = __ldcs(Hel + (r + q) * npair + p);
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = fma(__ldg(E + r + q), h[q], acc[q]);
  }
  for (; r < r1; ++r) acc[0] = fma(__ldg(E + r), __ldcs(Hel + r * npair + p), acc[0]);
  partial[(size_t)blockIdx.x * npair + p] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// H (k x k row-major, symmetric) from the G partial packed sums in a fixed order: a CTA takes
// 32 consecutive packed entries (lane = entry); warp w sums partials g in [G w / 8, G (w + 1) / 8)
// in order and the 8 warp sums are added in warp order (the G-long FP64 sums spread over SMs).
__global__ void __launch_bounds__(256) rom_assemble_final_kernel(const double* __restrict__ partial, int G, int k,
                                                                 double* H) {
  __shared__ double red[8][33];
  const int npair = k * (k + 1) / 2;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int p = blockIdx.x * 32 + l;
  const int g0 = (int)((long long)G * w / 8), g1 = (int)((long long)G * (w + 1) / 8);
  double s = 0.0;
  if (p < npair)
    for (int g = g0; g < g1; ++g) s += __ldcg(partial + (size_t)g * npair + p);
  red[w][l] = s;
  __syncthreads();
  if (w == 0 && p < npair) {
    double t = red[0][l];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][l];
    int i = 0, rem = p;
    while (rem >= k - i) {
      rem -= k - i;
      ++i;
    }
    const int j = i + rem;
    H[i * k + j] = t;
    H[j * k + i] = t;
  }
}

void launch_rom_assemble_final(cudaStream_t stream, const double* partial, int G, int k, double* H) {
  const int npair = k * (k + 1) / 2;
  rom_assemble_final_kernel<<<(npair + 31) / 32, 256, 0, stream>>>(partial, G, k, H);
  note_launch();
}

// Kernels of the k x k reduced solve live in rom.cu.
topo_status reduced_solve(topo_ctx* c, int k, const double* b, double* H_work, double* yhat, double* Jk);

template <int DIM>
static topo_status elem_impl(topo_ctx* c, const double* Phi, int k, long long ld, double* Hel,
                             const typename KeOf<DIM, double>::type& ke) {
  constexpr int ND = DIM == 2 ? 8 : 24;
  const int npair = k * (k + 1) / 2;
  const size_t budget = 96 * 1024;
  int EB = (int)std::max<size_t>(1, std::min<size_t>(64, (budget - 2 * npair) / (2 * (size_t)ND * k * sizeof(double))));
  const size_t smem = 2 * (size_t)EB * ND * k * sizeof(double) + 2 * (size_t)npair + 16;
  // smem <= budget + 16 for every k; the attribute takes that bound, one value for every call, so
  // host threads that launch concurrently never lower it under one another's launch
  TOPO_CUDA_TRY(c, cudaFuncSetAttribute(rom_elem_kernel<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(budget + 16)));
  ElemArgs<DIM> a;
  a.g = c->g;
  a.ke = ke;
  a.Phi = Phi;
  a.ld = ld;
  a.k = k;
  a.npair = npair;
  a.EB = EB;
  a.Hel = Hel;
  const long long blocks = (c->g.nel + EB - 1) / EB;
  rom_elem_kernel<DIM><<<(unsigned)blocks, 256, smem, c->stream>>>(a);
  note_launch();
  rom_elem_dirichlet_kernel<<<(npair + 127) / 128, 128, 0, c->stream>>>(Phi, ld, k, c->d_fixed_list, c->nfixed,
                                                                      Hel + (size_t)c->g.nel * npair);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_rom_elem(topo_ctx* c, const double* Phi, int k, int ld, double* Hel) {
  if (!c) return TOPO_ERR_INVALID;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_elem: 1 <= k <= 128");
  if ((long long)ld < c->g.ndof) return fail(c, TOPO_ERR_INVALID, "topo_rom_elem: ld < N");
  if (!dev_ptr_ok(Phi) || !dev_ptr_ok(Hel)) return fail(c, TOPO_ERR_INVALID, "topo_rom_elem: null or misaligned pointer");
  if (c->g.dim == 2) return elem_impl<2>(c, Phi, k, ld, Hel, c->q4_64);
  return elem_impl<3>(c, Phi, k, ld, Hel, c->h8_64);
}

extern "C" topo_status topo_rom_solve_elem(topo_ctx* c, const double* rho, const double* Hel, int k, const double* b,
                                           double* H_work, double* yhat, double* Jk) {
  if (!c) return TOPO_ERR_INVALID;
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_rom_solve_elem: 1 <= k <= 128");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(Hel) || !dev_ptr_ok(b) || !dev_ptr_ok(H_work) || !dev_ptr_ok(yhat) ||
      !dev_ptr_ok(Jk))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_solve_elem: null or misaligned pointer");
  const int npair = k * (k + 1) / 2;
  const long long rows = c->g.nel + 1;
  long long G = 4LL * c->num_sms;  // enough streaming loads in flight for HBM
  long long per = (rows + G - 1) / G;
  G = (rows + per - 1) / per;
  const size_t eoff = ((size_t)rows * sizeof(double) + 255) & ~(size_t)255;
  topo_status s = ensure_scratch(c, eoff + (size_t)G * npair * sizeof(double) + 4096);
  if (s) return s;
  double* E = (double*)c->d_scratch;
  double* partial = (double*)((char*)c->d_scratch + eoff);
  elem_moduli_kernel<<<(int)std::min<long long>(8LL * c->num_sms, (rows + 255) / 256), 256, 0, c->stream>>>(c->g, rho, E);
  note_launch();
  const int by = (npair + 255) / 256;
  rom_assemble_partial_kernel<<<dim3((unsigned)G, by), std::min(256, ((npair + 31) / 32) * 32), 0, c->stream>>>(
      Hel, E, rows, npair, per, partial);
  note_launch();
  launch_rom_assemble_final(c->stream, partial, (int)G, k, H_work);
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return reduced_solve(c, k, b, H_work, yhat, Jk);
}
