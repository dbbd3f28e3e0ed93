// Batched form: many independent design problems of uneven size solved in one persistent
// cooperative launch (plus batched filter, gradient and reduced solves).
//
// Each instance keeps its own context (Dirichlet mask, element matrices, filter, scratch,
// barrier state); all contexts share the batch's stream. The state solves run in one of two
// forms, chosen by the instance contexts' TOPO_PARAM_PCG_MG:
//
// Multigrid (the default). Each instance runs topo_solve_hdm's multigrid-preconditioned solve,
// one persistent cooperative launch with a fixed share of the SMs (SMs / S CTAs), on one of S
// internal streams; the instances are assigned largest first to the least loaded stream, the
// streams fork from and join back to the batch's stream with events. Instances run at their own
// pace: one whose V-cycle stalls and finishes with the polynomial preconditioner (hundreds of
// iterations where the others take tens) holds only its share. (A single persistent launch over
// all instances with multigrid groups was measured at 39 s for the 256-instance batch, against
// 5.5 s for the same solves run one after another: the CTAs of a group are fixed before the
// solve, and the group of an instance that falls back to the polynomial finishes last.)
//
// Jacobi (TOPO_PARAM_PCG_MG = 0). ONE launch of pcg2_batch_kernel: every instance gets a group
// of co-resident CTAs sized by its estimated work (nodes x load cases x mesh width, the last a
// proxy for the iteration count), has its own arrival counter and its own CG scalars, and
// converges on its own. When the instances need more CTAs than can be co-resident the batch runs
// in waves.
//
// Autotuning: the number of streams S (multigrid form) or of CTAs per SM of the batched launch
// (Jacobi form) is chosen on the first solve of a batch by timing each candidate on a short run
// of the same instances, and cached in the batch.
//
// Graph capture: a solve whose arguments equal the previous solve's (same pointers, sizes,
// tolerance, iteration cap, form and tuning, every instance's scratch unchanged) and asks for no
// host info reuses that solve's staged launches: it issues only the per-instance state resets,
// the launches and (multigrid form) the fork and join events, with no host synchronisation, so
// it can be captured in a CUDA graph after one eager call.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pcg2.cuh"

struct topo_batch {
  int count;
  std::vector<topo_ctx*> ctx;
  cudaStream_t stream;
  int num_sms;
  topo::GridSync* d_sync;  // batch-wide sticky status
  // launch tables (device) and their pinned host staging
  void* d_args;
  size_t args_bytes;
  int* d_tab;
  size_t tab_ints;
  void* h_stage;
  size_t stage_bytes;
  int tuned_bps;  // autotuned CTAs per SM (0 = not tuned yet)
  // the previous solve's launch, reused by an identical call (see the file comment)
  std::vector<unsigned long long> sig;
  std::vector<size_t> c_wave_off, c_wave_ctas;
  size_t c_grp_off;
  std::vector<int> c_grp;
  std::vector<void*> c_zflag, c_info;
  // multigrid form: internal streams, their fork and join events, and the staged solves
  std::vector<cudaStream_t> ms;
  std::vector<cudaEvent_t> ms_done;
  cudaEvent_t ms_fork;
  int tuned_streams;  // autotuned S (0 = not tuned yet)
  std::vector<unsigned long long> sig_mg;
  std::vector<topo::SoloLaunch2> c_solo;
  std::vector<int> c_stream_of;  // per instance, launch order is c_order
  std::vector<int> c_order;
  // batched reduced solves: device tables, partial sums, flags and their signature
  void* d_rom;
  size_t rom_bytes;
  std::vector<unsigned long long> sig_rom;
  int rom_items, rom_ypairs;
  size_t rom_inst_off, rom_item_off, rom_red_off, rom_part_off;
  char err[512];
};

namespace topo {

static topo_status bfail(topo_batch* b, topo_status s, const char* msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
  return s;
}

// Work weight of an instance for CTA allocation.
static double work_weight(const topo_ctx* c, int m) {
  return (double)c->g.nnodes * std::max(1, m) * (double)std::max(c->g.nx, c->g.ny);
}

struct Plan {
  std::vector<int> wave_of;   // per instance
  std::vector<int> grp;       // CTAs per instance
  int waves;
};

// Split instances into waves of at most cap CTAs; inside a wave, CTAs proportional to work.
static Plan make_plan(topo_batch* b, const int* m, int cap) {
  Plan p;
  const int n = b->count;
  p.wave_of.assign(n, 0);
  p.grp.assign(n, 1);
  std::vector<double> w(n);
  double total = 0;
  for (int i = 0; i < n; ++i) total += (w[i] = work_weight(b->ctx[i], m[i]));
  // number of waves: enough that every instance can have at least one CTA
  p.waves = std::max(1, (n + cap - 1) / cap);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  // round-robin the heaviest instances over waves, then size groups inside each wave
  for (int r = 0; r < n; ++r) p.wave_of[order[r]] = r % p.waves;
  for (int wv = 0; wv < p.waves; ++wv) {
    std::vector<int> ids;
    double tw = 0;
    for (int i = 0; i < n; ++i)
      if (p.wave_of[i] == wv) {
        ids.push_back(i);
        tw += w[i];
      }
    int left = cap - (int)ids.size();  // one CTA each is guaranteed
    for (int i : ids) {
      const long long units = (long long)((b->ctx[i]->g.nnx + 31) / 32) * b->ctx[i]->g.nny * b->ctx[i]->g.nnz;
      const int maxg = (int)std::max(1LL, units / 8);
      int extra = (int)std::floor(left * (w[i] / tw) * 0.999);
      p.grp[i] = std::min(maxg, 1 + std::max(0, extra));
    }
  }
  return p;
}

// The multigrid form's internal streams and events (created on first use).
static topo_status ensure_streams(topo_batch* b, int S) {
  if (!b->ms_fork && cudaEventCreateWithFlags(&b->ms_fork, cudaEventDisableTiming) != cudaSuccess)
    return bfail(b, TOPO_ERR_CUDA, "batched solve: event creation");
  while ((int)b->ms.size() < S) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return bfail(b, TOPO_ERR_CUDA, "batched solve: stream creation");
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(st);
      return bfail(b, TOPO_ERR_CUDA, "batched solve: event creation");
    }
    b->ms.push_back(st);
    b->ms_done.push_back(ev);
  }
  return TOPO_OK;
}

// Fork S streams from the batch's stream, launch every staged solve on its stream (largest
// first), join the streams back.
static topo_status launch_mg_streams(topo_batch* b, int S) {
  TOPO_CUDA_TRY(b->ctx[0], cudaEventRecord(b->ms_fork, b->stream));
  for (int q = 0; q < S; ++q) TOPO_CUDA_TRY(b->ctx[0], cudaStreamWaitEvent(b->ms[q], b->ms_fork, 0));
  for (int i : b->c_order) {
    cudaError_t e = launch_solo2(b->ctx[i], b->c_solo[i], b->ms[b->c_stream_of[i]]);
    if (e != cudaSuccess) return bfail(b, cuda_fail(b->ctx[i], e, "batched multigrid solve launch"), b->ctx[i]->err);
  }
  for (int q = 0; q < S; ++q) {
    TOPO_CUDA_TRY(b->ctx[0], cudaEventRecord(b->ms_done[q], b->ms[q]));
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamWaitEvent(b->stream, b->ms_done[q], 0));
  }
  return TOPO_OK;
}

static topo_status batch_solve_mg(topo_batch* b, const double* const* rho, const double* const* F, double* const* U,
                                  const int* m, const int* ld, double rtol, int maxit, int S,
                                  topo_solve_info* info_host) {
  const int n = b->count;
  S = std::max(1, std::min(S, n));
  std::vector<unsigned long long> sig;
  sig.reserve(6 * (size_t)n + 4);
  for (int i = 0; i < n; ++i) {
    sig.push_back((unsigned long long)(uintptr_t)rho[i]);
    sig.push_back((unsigned long long)(uintptr_t)F[i]);
    sig.push_back((unsigned long long)(uintptr_t)U[i]);
    sig.push_back((unsigned long long)m[i]);
    sig.push_back((unsigned long long)ld[i]);
    sig.push_back(b->ctx[i]->scratch_gen);
  }
  unsigned long long rbits = 0;
  memcpy(&rbits, &rtol, sizeof(rbits));
  sig.push_back(rbits);
  sig.push_back((unsigned long long)maxit);
  sig.push_back((unsigned long long)S);
  topo_status s = ensure_streams(b, S);
  if (s) return s;
  if (!info_host && sig == b->sig_mg) return launch_mg_streams(b, S);
  b->sig_mg.clear();
  // stage every instance for its share, then assign largest first to the least loaded stream
  const int share = std::max(1, b->num_sms / S);
  b->c_solo.resize(n);
  for (int i = 0; i < n; ++i) {
    s = stage_solo2(b->ctx[i], rho[i], F[i], U[i], m[i], ld[i], rtol, maxit, share, &b->c_solo[i]);
    if (s) return bfail(b, s, b->ctx[i]->err);
  }
  std::vector<double> w(n);
  for (int i = 0; i < n; ++i) w[i] = (double)b->ctx[i]->g.nnodes * std::max(1, m[i]);
  b->c_order.resize(n);
  for (int i = 0; i < n; ++i) b->c_order[i] = i;
  std::sort(b->c_order.begin(), b->c_order.end(), [&](int x, int y) { return w[x] > w[y] || (w[x] == w[y] && x < y); });
  std::vector<double> load(S, 0.0);
  b->c_stream_of.assign(n, 0);
  for (int i : b->c_order) {
    const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->c_stream_of[i] = q;
    load[q] += w[i];
  }
  // staging may have grown a context's scratch (a synchronising reallocation): the signature
  // records the scratch generation after it
  for (int i = 0; i < n; ++i) sig[6 * (size_t)i + 5] = b->ctx[i]->scratch_gen;
  s = launch_mg_streams(b, S);
  if (s) return s;
  b->sig_mg = sig;
  if (info_host) {
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    topo_status worst = TOPO_OK;
    for (int i = 0; i < n; ++i) {
      const SoloLaunch2& L = b->c_solo[i];
      int hi[4];
      double hr[2];
      TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(hi, L.a.info, 16, cudaMemcpyDeviceToHost));
      TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(hr, L.a.info_rr, 16, cudaMemcpyDeviceToHost));
      int dev_status = 0;
      TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(&dev_status, &b->ctx[i]->d_sync->status, sizeof(int),
                                          cudaMemcpyDeviceToHost));
      info_host[i].iters = hi[0];
      info_host[i].outer = 0;
      info_host[i].relres = std::sqrt(hr[0]);
      info_host[i].floor = std::sqrt(hr[1]);
      info_host[i].poly = L.mg ? (hi[3] ? L.a.poly : 0) : L.a.poly;
      info_host[i].mg_levels = L.mg ? L.a.mg.L : 0;
      info_host[i].fallback = L.mg ? hi[3] : 0;
      info_host[i].status = dev_status ? dev_status : hi[2];
      if (dev_status) {
        int zero = 0;
        cudaMemcpy(&b->ctx[i]->d_sync->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
      }
      if (info_host[i].status && worst == TOPO_OK) worst = (topo_status)info_host[i].status;
    }
    if (worst) return bfail(b, worst, "batched solve: some instance did not converge");
  }
  return TOPO_OK;
}

template <int DIM>
static topo_status batch_solve_dim(topo_batch* b, const double* const* rho, const double* const* F,
                                   double* const* U, const int* m, const int* ld, double rtol, int maxit,
                                   int bps, topo_solve_info* info_host) {
  const int n = b->count;
  std::vector<unsigned long long> sig;
  sig.reserve(6 * (size_t)n + 3);
  for (int i = 0; i < n; ++i) {
    sig.push_back((unsigned long long)(uintptr_t)rho[i]);
    sig.push_back((unsigned long long)(uintptr_t)F[i]);
    sig.push_back((unsigned long long)(uintptr_t)U[i]);
    sig.push_back((unsigned long long)m[i]);
    sig.push_back((unsigned long long)ld[i]);
    sig.push_back(b->ctx[i]->scratch_gen);
  }
  unsigned long long rbits = 0;
  memcpy(&rbits, &rtol, sizeof(rbits));
  sig.push_back(rbits);
  sig.push_back((unsigned long long)maxit);
  sig.push_back((unsigned long long)bps);
  if (!info_host && sig == b->sig) {
    // identical call: reset each instance's barrier, halo flags and info, then launch the
    // already staged waves (no host synchronisation)
    for (int i = 0; i < n; ++i) {
      TOPO_CUDA_TRY(b->ctx[0], cudaMemsetAsync(b->ctx[i]->d_bar, 0, sizeof(GridBar), b->stream));
      TOPO_CUDA_TRY(b->ctx[0],
                    cudaMemsetAsync(b->c_zflag[i], 0, sizeof(unsigned long long) * b->c_grp[i], b->stream));
      TOPO_CUDA_TRY(b->ctx[0], cudaMemsetAsync(b->c_info[i], 0, 32, b->stream));
    }
    for (size_t wv = 0; wv < b->c_wave_off.size(); ++wv) {
      const int* d_inst = b->d_tab + b->c_wave_off[wv];
      const int* d_rank = d_inst + b->c_wave_ctas[wv];
      TOPO_CUDA_TRY(b->ctx[0], launch_pcg2_batch2((unsigned)b->c_wave_ctas[wv], b->stream,
                                                  (const Pcg2Args<2>*)b->d_args, d_inst, d_rank,
                                                  b->d_tab + b->c_grp_off));
      note_launch();
    }
    return TOPO_OK;
  }
  b->sig.clear();  // the staging below replaces the cached launch
  const int occ = pcg2_occupancy();
  const int per_sm = std::max(1, std::min(bps, occ));
  const int cap = per_sm * b->num_sms;
  Plan plan = make_plan(b, m, cap);
  std::vector<Pcg2Args<DIM>> args(n);
  for (int i = 0; i < n; ++i) {
    topo_status s = build_pcg2_args<DIM>(b->ctx[i], rho[i], F[i], U[i], m[i], ld[i], rtol, maxit, plan.grp[i],
                                         &args[i], b->d_sync);
    if (s) return bfail(b, s, b->ctx[i]->err);
  }
  // device tables: args, then per wave the CTA -> (instance, rank) maps and group sizes
  const size_t abytes = sizeof(Pcg2Args<DIM>) * n;
  std::vector<int> tab;
  std::vector<size_t> wave_off, wave_ctas;
  for (int wv = 0; wv < plan.waves; ++wv) {
    wave_off.push_back(tab.size());
    size_t start = tab.size();
    std::vector<int> inst, rank;
    for (int i = 0; i < n; ++i)
      if (plan.wave_of[i] == wv)
        for (int r = 0; r < plan.grp[i]; ++r) {
          inst.push_back(i);
          rank.push_back(r);
        }
    wave_ctas.push_back(inst.size());
    tab.insert(tab.end(), inst.begin(), inst.end());
    tab.insert(tab.end(), rank.begin(), rank.end());
    (void)start;
  }
  const size_t grp_off = tab.size();
  tab.insert(tab.end(), plan.grp.begin(), plan.grp.end());
  const size_t need_stage = abytes + tab.size() * sizeof(int);
  if (need_stage > b->stage_bytes) {
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    if (b->h_stage) cudaFreeHost(b->h_stage);
    b->h_stage = nullptr;
    TOPO_CUDA_TRY(b->ctx[0], cudaMallocHost(&b->h_stage, need_stage));
    b->stage_bytes = need_stage;
  }
  if (abytes > b->args_bytes) {
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    if (b->d_args) cudaFree(b->d_args);
    b->d_args = nullptr;
    TOPO_CUDA_TRY(b->ctx[0], cudaMalloc(&b->d_args, abytes));
    b->args_bytes = abytes;
  }
  if (tab.size() > b->tab_ints) {
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    if (b->d_tab) cudaFree(b->d_tab);
    b->d_tab = nullptr;
    TOPO_CUDA_TRY(b->ctx[0], cudaMalloc(&b->d_tab, tab.size() * sizeof(int)));
    b->tab_ints = tab.size();
  }
  // the pinned staging may still feed a previous call's copies: wait for them
  TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
  memcpy(b->h_stage, args.data(), abytes);
  memcpy((char*)b->h_stage + abytes, tab.data(), tab.size() * sizeof(int));
  TOPO_CUDA_TRY(b->ctx[0], cudaMemcpyAsync(b->d_args, b->h_stage, abytes, cudaMemcpyHostToDevice, b->stream));
  TOPO_CUDA_TRY(b->ctx[0], cudaMemcpyAsync(b->d_tab, (char*)b->h_stage + abytes, tab.size() * sizeof(int),
                                           cudaMemcpyHostToDevice, b->stream));
  for (int i = 0; i < n; ++i) {
    TOPO_CUDA_TRY(b->ctx[0], cudaMemsetAsync(b->ctx[i]->d_bar, 0, sizeof(GridBar), b->stream));
    TOPO_CUDA_TRY(b->ctx[0],
                  cudaMemsetAsync(args[i].zflag, 0, sizeof(unsigned long long) * plan.grp[i], b->stream));
    TOPO_CUDA_TRY(b->ctx[0], cudaMemsetAsync(args[i].info, 0, 32, b->stream));
  }
  for (int wv = 0; wv < plan.waves; ++wv) {
    const int* d_inst = b->d_tab + wave_off[wv];
    const int* d_rank = d_inst + wave_ctas[wv];
    const int* d_grp = b->d_tab + grp_off;
    TOPO_CUDA_TRY(b->ctx[0], launch_pcg2_batch2((unsigned)wave_ctas[wv], b->stream, (const Pcg2Args<2>*)b->d_args,
                                                d_inst, d_rank, d_grp));
    note_launch();
  }
  b->c_wave_off = wave_off;
  b->c_wave_ctas = wave_ctas;
  b->c_grp_off = grp_off;
  b->c_grp = plan.grp;
  b->c_zflag.assign(n, nullptr);
  b->c_info.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    b->c_zflag[i] = args[i].zflag;
    b->c_info[i] = args[i].info;
  }
  b->sig = sig;
  if (info_host) {
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    topo_status worst = TOPO_OK;
    for (int i = 0; i < n; ++i) {
      int hi[4];
      double hr[2];
      TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(hi, args[i].info, 16, cudaMemcpyDeviceToHost));
      TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(hr, args[i].info_rr, 16, cudaMemcpyDeviceToHost));
      info_host[i].iters = hi[0];
      info_host[i].outer = 0;
      info_host[i].relres = std::sqrt(hr[0]);
      info_host[i].floor = std::sqrt(hr[1]);
      info_host[i].status = hi[2];
      info_host[i].poly = 1;
      info_host[i].mg_levels = 0;
      if (hi[2] && worst == TOPO_OK) worst = (topo_status)hi[2];
    }
    int st = 0;
    TOPO_CUDA_TRY(b->ctx[0], cudaMemcpy(&st, &b->d_sync->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
      int zero = 0;
      cudaMemcpy(&b->d_sync->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return bfail(b, (topo_status)st, "batched solve: device status set");
    }
    if (worst) return bfail(b, worst, "batched solve: some instance did not converge");
  }
  return TOPO_OK;
}

// ---------------------------------------------------------------------------------------
// Batched reduced solves (element path): H_i = sum_e E(rho_i,e) Hel_i[e] + Hel_i[N_e,i], then
// y_i = H_i^-1 b_i, J_i = b_i^T y_i, for every instance in three launches.
// ---------------------------------------------------------------------------------------
struct BromInst {
  const double* Hel;
  const double* rho;
  double* H;
  long long nel;     // element rows; row nel (weight 1) holds the Dirichlet term
  long long part0;   // offset of the instance's first item partial (doubles)
  int npair, k, item0, nitems;
  double E0, Emin;
  int ipenal, pad;
};
struct BromItem {
  long long r0, r1;  // rows [r0, r1) of instance inst
  int inst, local;   // local: index of the item within its instance
};
constexpr int BROM_CHUNK = 256;  // rows whose moduli a CTA stages at a time

// partial[part0 + local * npair + p] = sum over the item's rows e of E_e Hel[e][p] (thread = p;
// grid.y covers the pairs). The item's moduli are computed once per row into shared memory.
__global__ void __launch_bounds__(256) brom_partial_kernel(const BromInst* __restrict__ insts,
                                                           const BromItem* __restrict__ items, double* partial) {
  __shared__ double Es[BROM_CHUNK];
  const BromItem it = items[blockIdx.x];
  const BromInst& I = insts[it.inst];
  const int p = blockIdx.y * blockDim.x + threadIdx.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long c0 = it.r0; c0 < it.r1; c0 += BROM_CHUNK) {
    const int n = (int)min((long long)BROM_CHUNK, it.r1 - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const long long e = c0 + t;
      Es[t] = e < I.nel ? young<double>(__ldg(I.rho + e), I.E0, I.Emin, I.ipenal) : 1.0;
    }
    __syncthreads();
    if (p < I.npair) {
      int t = 0;
      for (; t + 3 < n; t += 4) {
        double h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __ldcs(I.Hel + (c0 + t + q) * I.npair + p);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(Es[t + q], h[q], acc[q]);
      }
      for (; t < n; ++t) acc[0] = fma(Es[t], __ldcs(I.Hel + (c0 + t) * I.npair + p), acc[0]);
    }
  }
  if (p < I.npair) partial[I.part0 + (long long)it.local * I.npair + p] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// H_i from its items' partials, summed in item order (block = instance, thread = pair).
__global__ void __launch_bounds__(256) brom_final_kernel(const BromInst* __restrict__ insts, const double* partial) {
  const BromInst& I = insts[blockIdx.x];
  for (int p = threadIdx.x; p < I.npair; p += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < I.nitems; ++q) s += __ldcg(partial + I.part0 + (long long)q * I.npair + p);
    int i = 0, rem = p;
    while (rem >= I.k - i) {
      rem -= I.k - i;
      ++i;
    }
    const int j = i + rem;
    I.H[i * I.k + j] = s;
    I.H[j * I.k + i] = s;
  }
}

static topo_status batch_rom_solve_multi(topo_batch* b, const double* const* rho, const double* const* Hel,
                                         const int* k, const double* const* bvec, double* const* H_work,
                                         double* const* yhat, double* Jk) {
  const int n = b->count;
  std::vector<unsigned long long> sig;
  sig.reserve(6 * (size_t)n + 1);
  for (int i = 0; i < n; ++i) {
    sig.push_back((unsigned long long)(uintptr_t)rho[i]);
    sig.push_back((unsigned long long)(uintptr_t)Hel[i]);
    sig.push_back((unsigned long long)k[i]);
    sig.push_back((unsigned long long)(uintptr_t)bvec[i]);
    sig.push_back((unsigned long long)(uintptr_t)H_work[i]);
    sig.push_back((unsigned long long)(uintptr_t)yhat[i]);
  }
  sig.push_back((unsigned long long)(uintptr_t)Jk);
  if (sig != b->sig_rom) {
    // items: about eight per SM over the whole batch, each at least one chunk of rows
    long long total = 0;
    for (int i = 0; i < n; ++i) total += b->ctx[i]->g.nel + 1;
    long long per = std::max<long long>(BROM_CHUNK, (total + 8LL * b->num_sms - 1) / (8LL * b->num_sms));
    per = (per + BROM_CHUNK - 1) / BROM_CHUNK * BROM_CHUNK;
    std::vector<BromInst> insts(n);
    std::vector<BromItem> items;
    std::vector<RedSolve> red(n);
    long long part = 0;
    int maxpair = 1;
    for (int i = 0; i < n; ++i) {
      const topo_ctx* c = b->ctx[i];
      BromInst& I = insts[i];
      I.Hel = Hel[i];
      I.rho = rho[i];
      I.H = H_work[i];
      I.nel = c->g.nel;
      I.npair = k[i] * (k[i] + 1) / 2;
      I.k = k[i];
      I.E0 = c->g.E0;
      I.Emin = c->g.Emin;
      I.ipenal = c->g.ipenal;
      I.pad = 0;
      I.item0 = (int)items.size();
      const long long rows = c->g.nel + 1;
      int local = 0;
      for (long long r0 = 0; r0 < rows; r0 += per, ++local) items.push_back({r0, std::min(rows, r0 + per), i, local});
      I.nitems = local;
      I.part0 = part;
      part += (long long)local * I.npair;
      maxpair = std::max(maxpair, I.npair);
    }
    const size_t oi = 0, oit = (sizeof(BromInst) * n + 255) & ~(size_t)255;
    const size_t ored = oit + ((sizeof(BromItem) * items.size() + 255) & ~(size_t)255);
    const size_t ook = ored + ((sizeof(RedSolve) * n + 255) & ~(size_t)255);
    const size_t opart = ook + ((sizeof(int) * n + 255) & ~(size_t)255);
    const size_t need = opart + sizeof(double) * (size_t)part;
    if (need > b->rom_bytes) {
      TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
      if (b->d_rom) cudaFree(b->d_rom);
      b->d_rom = nullptr;
      b->rom_bytes = 0;
      TOPO_CUDA_TRY(b->ctx[0], cudaMalloc(&b->d_rom, need));
      b->rom_bytes = need;
    }
    char* base = (char*)b->d_rom;
    for (int i = 0; i < n; ++i)
      red[i] = {H_work[i], bvec[i], yhat[i], Jk + i, &b->ctx[i]->d_sync->status, (int*)(base + ook) + i, k[i], 0};
    const size_t tbytes = opart;
    if (tbytes > b->stage_bytes) {
      TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
      if (b->h_stage) cudaFreeHost(b->h_stage);
      b->h_stage = nullptr;
      TOPO_CUDA_TRY(b->ctx[0], cudaMallocHost(&b->h_stage, tbytes));
      b->stage_bytes = tbytes;
    }
    // the pinned staging may still feed a previous call's copies: wait for them
    TOPO_CUDA_TRY(b->ctx[0], cudaStreamSynchronize(b->stream));
    char* h = (char*)b->h_stage;
    memcpy(h + oi, insts.data(), sizeof(BromInst) * n);
    memcpy(h + oit, items.data(), sizeof(BromItem) * items.size());
    memcpy(h + ored, red.data(), sizeof(RedSolve) * n);
    TOPO_CUDA_TRY(b->ctx[0], cudaMemcpyAsync(base, h, ook, cudaMemcpyHostToDevice, b->stream));
    b->rom_items = (int)items.size();
    b->rom_ypairs = (maxpair + 255) / 256;
    b->rom_inst_off = oi;
    b->rom_item_off = oit;
    b->rom_red_off = ored;
    b->rom_part_off = opart;
    b->sig_rom = sig;
  }
  char* base = (char*)b->d_rom;
  const BromInst* d_inst = (const BromInst*)(base + b->rom_inst_off);
  brom_partial_kernel<<<dim3((unsigned)b->rom_items, (unsigned)b->rom_ypairs), 256, 0, b->stream>>>(
      d_inst, (const BromItem*)(base + b->rom_item_off), (double*)(base + b->rom_part_off));
  note_launch();
  brom_final_kernel<<<n, 256, 0, b->stream>>>(d_inst, (const double*)(base + b->rom_part_off));
  note_launch();
  TOPO_CUDA_TRY(b->ctx[0], launch_chol_small_multi((const RedSolve*)(base + b->rom_red_off), n, b->stream));
  return TOPO_OK;
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_batch_create(const topo_problem* probs, int count, void* cuda_stream, topo_batch** out) {
  if (!out) return TOPO_ERR_INVALID;
  *out = nullptr;
  if (!probs || count < 1) return TOPO_ERR_INVALID;
  for (int i = 1; i < count; ++i)
    if (probs[i].dim != probs[0].dim) return TOPO_ERR_INVALID;
  if (probs[0].dim != 2) return TOPO_ERR_INVALID;  // batched solves are 2D Q4 only
  topo_batch* b = new topo_batch();
  b->count = count;
  b->stream = (cudaStream_t)cuda_stream;
  b->ctx.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    topo_status s = topo_create(&probs[i], cuda_stream, &b->ctx[i]);
    if (s) {
      topo_batch_destroy(b);
      return s;
    }
  }
  b->num_sms = b->ctx[0]->num_sms;
  if (cudaMalloc(&b->d_sync, sizeof(GridSync)) != cudaSuccess) {
    topo_batch_destroy(b);
    return TOPO_ERR_OOM;
  }
  cudaMemset(b->d_sync, 0, sizeof(GridSync));
  *out = b;
  return TOPO_OK;
}

extern "C" topo_status topo_batch_destroy(topo_batch* b) {
  if (!b) return TOPO_OK;
  cudaStreamSynchronize(b->stream);
  for (cudaStream_t st : b->ms) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t ev : b->ms_done) cudaEventDestroy(ev);
  if (b->ms_fork) cudaEventDestroy(b->ms_fork);
  for (topo_ctx* c : b->ctx)
    if (c) topo_destroy(c);
  cudaFree(b->d_sync);
  cudaFree(b->d_args);
  cudaFree(b->d_tab);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  cudaFree(b->d_rom);
  delete b;
  return TOPO_OK;
}

extern "C" const char* topo_batch_last_error(const topo_batch* b) { return b ? b->err : "null batch"; }

extern "C" topo_status topo_batch_context(topo_batch* b, int i, topo_ctx** out) {
  if (!b || !out || i < 0 || i >= b->count) return TOPO_ERR_INVALID;
  *out = b->ctx[i];
  return TOPO_OK;
}

extern "C" topo_status topo_batch_solve_hdm(topo_batch* b, const double* const* rho, const double* const* F,
                                            double* const* U, const int* m, const int* ld, double rtol, int maxit,
                                            topo_solve_info* info_host) {
  if (!b) return TOPO_ERR_INVALID;
  if (!rho || !F || !U || !m || !ld) return bfail(b, TOPO_ERR_INVALID, "batched solve: null argument array");
  if (!(rtol > 0.0) || maxit < 0) return bfail(b, TOPO_ERR_INVALID, "batched solve: rtol > 0, maxit >= 0");
  for (int i = 0; i < b->count; ++i) {
    if (m[i] < 1 || m[i] > 32 || (long long)ld[i] < b->ctx[i]->g.ndof || !dev_ptr_ok(rho[i]) || !dev_ptr_ok(F[i]) ||
        !dev_ptr_ok(U[i]) || F[i] == U[i])
      return bfail(b, TOPO_ERR_INVALID, "batched solve: bad instance arguments (m in [1,32], ld >= N, pointers)");
  }
  bool mg = true;
  for (const topo_ctx* c : b->ctx) mg = mg && c->pcg_mg != 0;
  int bps = mg ? b->tuned_streams : b->tuned_bps;
  if (bps == 0) {
    // autotune the CTAs per SM on short runs of these instances; the caller's initial guesses
    // are saved first and restored afterwards
    std::vector<double*> saved(b->count, nullptr);
    for (int i = 0; i < b->count; ++i) {
      const size_t bytes = sizeof(double) * (size_t)ld[i] * m[i];
      if (cudaMalloc(&saved[i], bytes) != cudaSuccess) {
        for (double* q : saved) cudaFree(q);
        return bfail(b, TOPO_ERR_OOM, "batched solve: autotuning copy");
      }
      cudaMemcpyAsync(saved[i], U[i], bytes, cudaMemcpyDeviceToDevice, b->stream);
    }
    float best = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // candidates: streams of the multigrid form, CTAs per SM of the Jacobi launch
    const int cands_mg[3] = {4, 8, 16}, cands_j[4] = {1, 2, 3, 4};
    bps = mg ? 8 : 2;
    for (int ci = 0; ci < (mg ? 3 : 4); ++ci) {
      const int cand = mg ? cands_mg[ci] : cands_j[ci];
      cudaEventRecord(e0, b->stream);
      topo_status s = mg ? batch_solve_mg(b, rho, F, U, m, ld, rtol, 30, cand, nullptr)
                         : batch_solve_dim<2>(b, rho, F, U, m, ld, rtol, 30, cand, nullptr);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      if (s) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bps = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < b->count; ++i) {
      cudaMemcpyAsync(U[i], saved[i], sizeof(double) * (size_t)ld[i] * m[i], cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    for (double* q : saved) cudaFree(q);
    if (mg)
      b->tuned_streams = bps;
    else
      b->tuned_bps = bps;
  }
  if (mg) return batch_solve_mg(b, rho, F, U, m, ld, rtol, maxit, bps, info_host);
  return batch_solve_dim<2>(b, rho, F, U, m, ld, rtol, maxit, bps, info_host);
}

extern "C" topo_status topo_batch_filter(topo_batch* b, const double* const* in, double* const* out, int adjoint) {
  if (!b || !in || !out) return TOPO_ERR_INVALID;
  for (int i = 0; i < b->count; ++i) {
    topo_status s = topo_filter(b->ctx[i], in[i], out[i], adjoint);
    if (s) return bfail(b, s, b->ctx[i]->err);
  }
  return TOPO_OK;
}

extern "C" topo_status topo_batch_compliance_grad(topo_batch* b, const double* const* rho, const double* const* U,
                                                  const int* m, const int* ld, const double* const* F, double* J,
                                                  double* const* dc_rho, double* const* dc_psi) {
  if (!b || !rho || !U || !m || !ld || !F || !J || !dc_rho) return TOPO_ERR_INVALID;
  for (int i = 0; i < b->count; ++i) {
    topo_status s = topo_compliance_grad(b->ctx[i], rho[i], U[i], m[i], ld[i], F[i], J + i, dc_rho[i],
                                         dc_psi ? dc_psi[i] : nullptr);
    if (s) return bfail(b, s, b->ctx[i]->err);
  }
  return TOPO_OK;
}

extern "C" topo_status topo_batch_rom_solve_elem(topo_batch* b, const double* const* rho, const double* const* Hel,
                                                 const int* k, const double* const* bvec, double* const* H_work,
                                                 double* const* yhat, double* Jk) {
  if (!b || !rho || !Hel || !k || !bvec || !H_work || !yhat || !Jk) return TOPO_ERR_INVALID;
  bool small = true;
  for (int i = 0; i < b->count; ++i) {
    if (k[i] < 1 || k[i] > 128 || !dev_ptr_ok(rho[i]) || !dev_ptr_ok(Hel[i]) || !dev_ptr_ok(bvec[i]) ||
        !dev_ptr_ok(H_work[i]) || !dev_ptr_ok(yhat[i]) || !dev_ptr_ok(Jk))
      return bfail(b, TOPO_ERR_INVALID, "batched reduced solve: 1 <= k <= 128 and device pointers required");
    small = small && k[i] <= 32;
  }
  if (small) {
    topo_status s = batch_rom_solve_multi(b, rho, Hel, k, bvec, H_work, yhat, Jk);
    return s ? bfail(b, s, b->ctx[0]->err) : TOPO_OK;
  }
  // a basis above 32 vectors: one call per instance (the CTA-wide Cholesky of topo_rom_solve_elem)
  for (int i = 0; i < b->count; ++i) {
    topo_status s = topo_rom_solve_elem(b->ctx[i], rho[i], Hel[i], k[i], bvec[i], H_work[i], yhat[i], Jk + i);
    if (s) return bfail(b, s, b->ctx[i]->err);
  }
  return TOPO_OK;
}
