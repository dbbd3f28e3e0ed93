// topo_rom_solve_elem_noalloc: the element-path reduced solve without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a reduced solve: a
// serving loop whose memory budget is owned by an outside allocator, code that runs while
// another component holds the whole device pool, or a latency-critical loop that cannot
// afford the implicit device synchronisation of cudaMalloc/cudaFree. topo_rom_solve_elem may
// grow the context's scratch on first use; this variant never does. Its scratch is the
// file-scope device array below, which every GPU that loads the library keeps until exit.
#include <mutex>

#include "common.cuh"

namespace topo {

// Kernels of the element path (romelem.cu) and of the k x k solve (rom.cu), reused unchanged.
__global__ void elem_moduli_kernel(Grid g, const double* rho, double* E);
__global__ void __launch_bounds__(256) rom_assemble_partial_kernel(const double* __restrict__ Hel,
                                                                   const double* __restrict__ E, long long rows,
                                                                   int npair, long long rows_per_cta,
                                                                   double* partial);
void launch_rom_assemble_final(cudaStream_t stream, const double* partial, int G, int k, double* H);
// k x k reduced solve (rom.cu): Cholesky of H_work into L, yhat, Jk; *ok = factorisation succeeded.
topo_status launch_reduced_solve(topo_ctx* c, int k, const double* b, double* H_work, double* yhat, double* Jk,
                                 int* ok);

// 8 MiB shared by all calls in the process: a 256-byte flag block, E(rho) for N_e + 1 rows,
// and the per-CTA partial sums of the reduced matrix.
static constexpr size_t kNoAllocBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, resolved once per device with that device current. In host
// code the symbol itself is only a host-side stand-in, never a device address.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

static topo_status noalloc_scratch(topo_ctx* c, unsigned char** out) {
  const int dev = c->device;
  if (dev < 0 || dev >= 64) return fail(c, TOPO_ERR_INVALID, "no-alloc scratch: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "no-alloc scratch: cudaGetDevice");
    if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(c, e, "no-alloc scratch: cudaSetDevice");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "no-alloc scratch: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return TOPO_OK;
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_rom_solve_elem_noalloc(topo_ctx* c, const double* rho, const double* Hel, int k,
                                                   const double* b, double* H_work, double* yhat, double* Jk) {
  if (!c) return TOPO_ERR_INVALID;
  if (k < 1 || k > 64) return fail(c, TOPO_ERR_INVALID, "topo_rom_solve_elem_noalloc: 1 <= k <= 64");
  if (!dev_ptr_ok(rho) || !dev_ptr_ok(Hel) || !dev_ptr_ok(b) || !dev_ptr_ok(H_work) || !dev_ptr_ok(yhat) ||
      !dev_ptr_ok(Jk))
    return fail(c, TOPO_ERR_INVALID, "topo_rom_solve_elem_noalloc: null or misaligned pointer");
  const int npair = k * (k + 1) / 2;
  const long long rows = c->g.nel + 1;
  long long G = 2LL * c->num_sms;
  const long long per = (rows + G - 1) / G;
  G = (rows + per - 1) / per;
  const size_t flags_bytes = 256;
  const size_t e_bytes = ((size_t)rows * sizeof(double) + 255) & ~(size_t)255;
  const size_t need = flags_bytes + e_bytes + (size_t)G * npair * sizeof(double);
  if (need > kNoAllocBytes)
    return fail(c, TOPO_ERR_INVALID,
                "topo_rom_solve_elem_noalloc: needs %zu bytes of scratch for N_e = %lld, k = %d; the fixed "
                "array holds %zu",
                need, c->g.nel, k, kNoAllocBytes);
  unsigned char* base = nullptr;
  topo_status s = noalloc_scratch(c, &base);
  if (s) return s;
  int* ok = reinterpret_cast<int*>(base);
  double* E = reinterpret_cast<double*>(base + flags_bytes);
  double* partial = reinterpret_cast<double*>(base + flags_bytes + e_bytes);
  // The array keeps the previous call's contents: the factorisation flag must start at zero.
  TOPO_CUDA_TRY(c, cudaMemsetAsync(ok, 0, flags_bytes, c->stream));
  elem_moduli_kernel<<<(int)std::min<long long>(8LL * c->num_sms, (rows + 255) / 256), 256, 0, c->stream>>>(c->g, rho,
                                                                                                           E);
  note_launch();
  rom_assemble_partial_kernel<<<dim3((unsigned)G, (npair + 255) / 256), std::min(256, ((npair + 31) / 32) * 32), 0,
                                c->stream>>>(Hel, E, rows, npair, per, partial);
  note_launch();
  launch_rom_assemble_final(c->stream, partial, (int)G, k, H_work);
  // k <= 64: the factor (32 KB) fits the default shared-memory window, no attribute change
  return launch_reduced_solve(c, k, b, H_work, yhat, Jk, ok);
}
