// The trust-region step of one major iteration (Algorithm 2, Section 4.2) on the device:
//   topo_tr_init     the run's state: Delta_0 = tau ||r(0, rho)|| = tau ||f|| on the free DOFs
//                    (Eq. trrad0), Delta_max = factor Delta_0, J at the first centre
//   topo_tr_project  P_C(psi - t g), the Euclidean projection onto the feasible set
//                    C = [0,1]^Ne with sum psi <= vmax (Eq. feaset-topopt, unit element volumes)
//   topo_tr_trials   trial designs psi_c + s (psi_x - psi_c), s = 0, 1, 1/2, 1/4, ...
//   topo_tr_select   the longest trial inside the error-aware trust region (Eq. trcon-topopt)
//                    that passes the Armijo decrease test on the model, and its reduced state
//   topo_tr_update   varrho_k, step acceptance and the radius rule (Algorithm 2, steps 4-6)
// Every decision is taken on the device from device values, so a run advances without the
// host reading anything back until it reports.
//
// The projection. By the KKT conditions P_C(z) = clip(z - mu, 0, 1) with mu >= 0 the root of
// v(mu) = sum_e clip(z_e - mu, 0, 1) - vmax (mu = 0 when clip(z) already fits). v is
// continuous, nonincreasing and piecewise linear with breakpoints {z_e, z_e - 1}. Each round
// evaluates v at 32 points of the current bracket [lo, hi] (v(lo) > 0 >= v(hi)) and keeps the
// section holding the root. Elements whose breakpoints lie outside the bracket contribute a
// constant (1 or 0) or a linear term z_e - mu on all of it and are summed once per round
// (n_sat, n_lin, S_lin); only the others ("straddlers") are evaluated at the 32 points. When a
// round's bracket holds no breakpoint, v is linear on it and the root is exact:
// mu = (n_sat + S_lin - vmax) / n_lin. Sums run per tile of 2048 elements and then over the
// tiles in a fixed order, so the result does not depend on the launch and is deterministic.
#include <cmath>

#include "common.cuh"

namespace topo {

constexpr int PJ_THREADS = 256;
constexpr int PJ_PER = 8;
constexpr int PJ_TILE = PJ_THREADS * PJ_PER;
constexpr int PJ_PTS = 32;            // section points per round
constexpr int PJ_SLOTS = PJ_PTS + 4;  // straddler sums per point, then n_sat, n_lin, S_lin, n_str
constexpr int PJ_ROUNDS = 12;         // 5 bits of the bracket per round: 60 bits in all

struct ProjState {
  double lo, hi, mu, tau;
  int done;
  int pad[7];
};

struct ProjArgs {
  const double* psi;
  const double* g;  // null: z = psi
  double t;
  int scaled;
  double vmax;
  long long n;
  int tiles;
  double* part;   // 2 x PJ_SLOTS x tiles, slot-major (the buffer of round r is r & 1)
  double* maxes;  // 2 x tiles: max |psi|, max |g| of each tile
  ProjState* st;  // PJ_ROUNDS + 1 states: st[r] is the bracket round r evaluated
  double* out;
  double* spart;  // 3 x tiles
  double* stats;
};

// z_e = psi_e - tau g_e, rounded as two operations (the product, then the difference).
__device__ __forceinline__ double pj_z(const ProjArgs& a, double tau, long long e) {
  return a.g ? __dsub_rn(a.psi[e], __dmul_rn(tau, a.g[e])) : a.psi[e];
}

// mu_j = lo + (hi - lo) j / 32, with the same rounding wherever it is formed.
__device__ __forceinline__ double pj_mu(double lo, double hi, int j) {
  return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), (double)j * (1.0 / PJ_PTS)));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__device__ inline double block_max(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    t = warp_max(t);
  }
  __syncthreads();
  return t;
}

// From the sums of the round that evaluated bracket S (round index r), the next bracket, or the
// root. Invariant: v(S.lo) > 0 (except at round 0, whose lo = 0 is tested), v(S.hi) <= 0.
__device__ void pj_decide(ProjState& S, const double* sum, int r, double vmax) {
  const double n_sat = sum[PJ_PTS], n_lin = sum[PJ_PTS + 1], s_lin = sum[PJ_PTS + 2], n_str = sum[PJ_PTS + 3];
  auto v = [&](int j) {
    const double mu = pj_mu(S.lo, S.hi, j);
    return __dsub_rn(__dadd_rn(__dadd_rn(n_sat, __dsub_rn(s_lin, __dmul_rn(n_lin, mu))), sum[j]), vmax);
  };
  if (r == 0 && v(0) <= 0.0) {  // the box projection already fits the volume
    S.mu = 0.0;
    S.done = 1;
    return;
  }
  if (n_str == 0.0) {  // no breakpoint inside: v is linear on the bracket
    const double mu = n_lin > 0.0 ? __ddiv_rn(__dsub_rn(__dadd_rn(n_sat, s_lin), vmax), n_lin) : S.hi;
    S.mu = fmin(fmax(mu, S.lo), S.hi);
    S.done = 1;
    return;
  }
  int j = 1;
  while (j < PJ_PTS && v(j) > 0.0) ++j;
  const double lo = pj_mu(S.lo, S.hi, j - 1);
  const double hi = j < PJ_PTS ? pj_mu(S.lo, S.hi, j) : S.hi;
  S.lo = lo;
  S.hi = hi;
}

__global__ void __launch_bounds__(PJ_THREADS) proj_max_kernel(ProjArgs a) {
  __shared__ double red[PJ_THREADS / 32];
  double pm = 0.0, gm = 0.0;
  const long long base = (long long)blockIdx.x * PJ_TILE;
  for (int i = 0; i < PJ_PER; ++i) {
    const long long e = base + i * PJ_THREADS + threadIdx.x;
    if (e < a.n) {
      pm = fmax(pm, fabs(a.psi[e]));
      if (a.g) gm = fmax(gm, fabs(a.g[e]));
    }
  }
  pm = block_max(pm, red);
  gm = block_max(gm, red);
  if (threadIdx.x == 0) {
    a.maxes[blockIdx.x] = pm;
    a.maxes[a.tiles + blockIdx.x] = gm;
  }
}

// Sums of PJ_SLOTS values over the block (fixed order), written to part[slot * tiles + tile].
__device__ inline void pj_write_slots(double* vals, double* part, int tiles, double (*wred)[PJ_SLOTS]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < PJ_SLOTS; ++s) {
    const double t = warp_sum(vals[s]);
    if (l == 0) wred[w][s] = t;
  }
  __syncthreads();
  if (threadIdx.x < PJ_SLOTS) {
    double t = 0.0;
    for (int q = 0; q < PJ_THREADS / 32; ++q) t += wred[q][threadIdx.x];
    part[(size_t)threadIdx.x * tiles + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(PJ_THREADS) proj_round_kernel(ProjArgs a, int r) {
  __shared__ double s_sum[PJ_SLOTS];
  __shared__ double s_mu[PJ_PTS];
  __shared__ double wred[PJ_THREADS / 32][PJ_SLOTS];
  __shared__ double red[PJ_THREADS / 32];
  __shared__ ProjState S;
  if (r == 0) {
    // tau and the first bracket [0, max|psi| + tau max|g|] (maxima are exact in any order; the
    // margin keeps every z_e below hi after rounding)
    double pm = 0.0, gm = 0.0;
    for (int i = threadIdx.x; i < a.tiles; i += blockDim.x) {
      pm = fmax(pm, a.maxes[i]);
      gm = fmax(gm, a.maxes[a.tiles + i]);
    }
    pm = block_max(pm, red);
    gm = block_max(gm, red);
    if (threadIdx.x == 0) {
      S.tau = a.g ? (a.scaled ? (gm > 0.0 ? __ddiv_rn(a.t, gm) : 0.0) : a.t) : 0.0;
      S.lo = 0.0;
      S.hi = (pm + S.tau * gm) * (1.0 + 1e-12) + 1e-300;
      S.mu = 0.0;
      S.done = 0;
      if (blockIdx.x == 0) a.st[0] = S;
    }
    __syncthreads();
  } else {
    if (threadIdx.x == 0) S = a.st[r - 1];
    __syncthreads();
    if (!S.done) {
      reduce_slots(a.part + (size_t)((r - 1) & 1) * PJ_SLOTS * a.tiles, (unsigned)a.tiles, PJ_SLOTS, s_sum);
      if (threadIdx.x == 0) pj_decide(S, s_sum, r - 1, a.vmax);
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) a.st[r] = S;
    __syncthreads();
    if (S.done) return;
  }
  const double lo = S.lo, hi = S.hi, tau = S.tau;
  if (threadIdx.x < PJ_PTS) s_mu[threadIdx.x] = pj_mu(lo, hi, threadIdx.x);
  __syncthreads();
  double vals[PJ_SLOTS];
#pragma unroll
  for (int s = 0; s < PJ_SLOTS; ++s) vals[s] = 0.0;
  const long long base = (long long)blockIdx.x * PJ_TILE;
  for (int i = 0; i < PJ_PER; ++i) {
    const long long e = base + i * PJ_THREADS + threadIdx.x;
    if (e >= a.n) break;
    const double z = pj_z(a, tau, e);
    const double zh = z - hi, zl = z - lo;
    if (zh >= 1.0) {
      vals[PJ_PTS] += 1.0;
    } else if (zl <= 0.0) {
    } else if (zl <= 1.0 && zh >= 0.0) {
      vals[PJ_PTS + 1] += 1.0;
      vals[PJ_PTS + 2] += z;
    } else {
      vals[PJ_PTS + 3] += 1.0;
#pragma unroll
      for (int j = 0; j < PJ_PTS; ++j) vals[j] += fmin(fmax(z - s_mu[j], 0.0), 1.0);
    }
  }
  pj_write_slots(vals, a.part + (size_t)(r & 1) * PJ_SLOTS * a.tiles, a.tiles, wred);
}

__global__ void __launch_bounds__(PJ_THREADS) proj_final_kernel(ProjArgs a) {
  __shared__ double s_sum[PJ_SLOTS];
  __shared__ double red[3 * 32];
  __shared__ ProjState S;
  if (threadIdx.x == 0) S = a.st[PJ_ROUNDS - 1];
  __syncthreads();
  if (!S.done) {
    reduce_slots(a.part + (size_t)((PJ_ROUNDS - 1) & 1) * PJ_SLOTS * a.tiles, (unsigned)a.tiles, PJ_SLOTS, s_sum);
    if (threadIdx.x == 0) {
      pj_decide(S, s_sum, PJ_ROUNDS - 1, a.vmax);
      if (!S.done) {  // the bracket is at rounding width: its upper end fits the volume
        S.mu = S.hi;
        S.done = 1;
      }
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == 0) a.st[PJ_ROUNDS] = S;
  __syncthreads();
  const double mu = S.mu, tau = S.tau;
  double gd = 0.0, dd = 0.0, vol = 0.0;
  const long long base = (long long)blockIdx.x * PJ_TILE;
  for (int i = 0; i < PJ_PER; ++i) {
    const long long e = base + i * PJ_THREADS + threadIdx.x;
    if (e >= a.n) break;
    const double p0 = a.psi[e];
    const double x = fmin(fmax(pj_z(a, tau, e) - mu, 0.0), 1.0);
    a.out[e] = x;  // after every read of psi[e] (out may alias psi)
    const double d = x - p0;
    if (a.g) gd = fma(a.g[e], d, gd);
    dd = fma(d, d, dd);
    vol += x;
  }
  block_sum3(gd, dd, vol, red);
  if (threadIdx.x == 0) {
    a.spart[blockIdx.x] = gd;
    a.spart[a.tiles + blockIdx.x] = dd;
    a.spart[2 * a.tiles + blockIdx.x] = vol;
  }
}

__global__ void proj_stats_kernel(ProjArgs a) {
  __shared__ double s[3];
  reduce_slots(a.spart, (unsigned)a.tiles, 3, s);
  if (threadIdx.x == 0) {
    a.stats[0] = s[0];
    a.stats[1] = sqrt(s[1]);
    a.stats[2] = a.st[PJ_ROUNDS].mu;
    a.stats[3] = s[2];
  }
}

// ---------------------------------------------------------------------------------------
// Trial steps, selection, update.
// ---------------------------------------------------------------------------------------
__global__ void tr_trials_kernel(int R, const double* psi_c, const double* psi_x, double* trials, long long ldt,
                                 long long ne) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ne * R;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / ne);
    const long long e = t - (long long)r * ne;
    const double pc = psi_c[e];
    // s = 2^-(r-1) is exact, so s (psi_x - psi_c) is exact and the sum is rounded once
    trials[(long long)r * ldt + e] = r == 0 ? pc : fma(ldexp(1.0, 1 - r), __dsub_rn(psi_x[e], pc), pc);
  }
}

__global__ void tr_select_kernel(topo_tr_state* st, int R, const double* Jk, const double* resnorm,
                                 const double* gtd, double c1) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double Jkc = Jk[0], delta = st->delta, gd = *gtd;
  int sel = R - 1, inside = 0;
  for (int r = 1; r < R; ++r) {
    const double s = ldexp(1.0, 1 - r);
    // m_k(psi_s) <= m_k(psi_c) + c1 s g.(psi_x - psi_c), the product formed left to right
    if (resnorm[2 * r] <= delta && Jk[r] <= __dadd_rn(Jkc, __dmul_rn(__dmul_rn(c1, s), gd))) {
      sel = r;
      inside = 1;
      break;
    }
  }
  st->sel = sel;
  st->inside = inside;
  st->step = ldexp(1.0, 1 - sel);
  st->Jk_c = Jkc;
  st->Jk_hat = Jk[sel];
  st->theta_hat = resnorm[2 * sel];
  st->gtd = gd;
}

// psi_hat = trials[sel], u_hat = Phi y_sel (the reduced state, the full-order solve's start).
__global__ void tr_gather_kernel(const topo_tr_state* st, const double* trials, long long ldt, long long ne,
                                 const double* Phi, long long ld, int k, const double* yhat, double* psi_hat,
                                 double* u_hat, long long N) {
  extern __shared__ double sy[];
  const int sel = st->sel;
  for (int j = threadIdx.x; j < k; j += blockDim.x) sy[j] = yhat[(long long)sel * k + j];
  __syncthreads();
  const long long n = N > ne ? N : ne;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (i < ne) psi_hat[i] = trials[(long long)sel * ldt + i];
    if (i < N) {
      double acc = 0.0;
      for (int j = 0; j < k; ++j) acc = fma(Phi[(long long)j * ld + i], sy[j], acc);
      u_hat[i] = acc;
    }
  }
}

__global__ void tr_update_kernel(topo_tr_state* st, topo_tr_params p, const double* J_hat) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double Jh = *J_hat;
  const double pred = st->Jk_c - st->Jk_hat;
  const double ratio = pred > 0.0 ? (st->J_c - Jh) / pred : -INFINITY;
  const bool acc = ratio >= p.eta1;  // false for NaN as well
  const double d = st->delta;
  double dn;
  if (!acc)
    dn = p.gamma1 * d;
  else if (ratio < p.eta2)
    dn = p.gamma2 * d;
  else
    dn = fmin(p.grow * d, st->delta_max);
  st->J_hat = Jh;
  st->ratio = ratio;
  st->accepted = acc ? 1 : 0;
  st->delta_prev = d;
  st->delta = dn;
  if (acc) st->J_c = Jh;
  st->iter += 1;
}

// On acceptance the candidate becomes the centre (and its state a snapshot of the window).
__global__ void tr_move_kernel(const topo_tr_state* st, long long ne, long long N, double* psi_c,
                               const double* psi_hat, double* u_c, const double* u_hat, double* g_c,
                               const double* g_hat, double* u_slot) {
  if (!st->accepted) return;
  const long long n = N > ne ? N : ne;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (i < ne) {
      psi_c[i] = psi_hat[i];
      g_c[i] = g_hat[i];
    }
    if (i < N) {
      const double u = u_hat[i];
      u_c[i] = u;
      if (u_slot) u_slot[i] = u;
    }
  }
}

__global__ void tr_init_kernel(Grid g, const double* f, double tau, double dmax_factor, const double* J_c,
                               topo_tr_state* st) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < g.ndof; i += blockDim.x)
    if (!is_fixed(g, i)) s = fma(f[i], f[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double d0 = tau * sqrt(s);
    topo_tr_state z = {};
    z.delta = d0;
    z.delta_max = dmax_factor * d0;
    z.delta_prev = d0;
    z.J_c = *J_c;
    z.ratio = 0.0;
    *st = z;
  }
}

static long long grid_for(topo_ctx* c, long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 8LL * c->num_sms;
  return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_tr_init(topo_ctx* c, topo_tr_state* st, const double* f, double tau, double dmax_factor,
                                    const double* J_c) {
  if (!c) return TOPO_ERR_INVALID;
  if (!dev_ptr_ok(st) || !dev_ptr_ok(f) || !dev_ptr_ok(J_c))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_init: null or misaligned pointer");
  if (!(tau > 0.0) || !(dmax_factor >= 1.0))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_init: tau > 0 and dmax_factor >= 1 required");
  tr_init_kernel<<<1, 1024, 0, c->stream>>>(c->g, f, tau, dmax_factor, J_c, st);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_tr_project(topo_ctx* c, const double* psi, const double* g, double t, int scaled,
                                       double vmax, double* out, double* stats) {
  if (!c) return TOPO_ERR_INVALID;
  if (!dev_ptr_ok(psi) || !dev_ptr_ok(out) || !dev_ptr_ok(stats) || (g && !dev_ptr_ok(g)))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_project: null or misaligned pointer");
  if (g && (g == out)) return fail(c, TOPO_ERR_INVALID, "topo_tr_project: out must not alias g");
  if (!(vmax >= 0.0) || !std::isfinite(t))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_project: vmax >= 0 and a finite t required");
  if (scaled && !(t >= 0.0)) return fail(c, TOPO_ERR_INVALID, "topo_tr_project: a scaled step needs t >= 0");
  const long long n = c->g.nel;
  const int tiles = (int)((n + PJ_TILE - 1) / PJ_TILE);
  const size_t bytes = sizeof(double) * ((size_t)2 * PJ_SLOTS * tiles + 2 * tiles + 3 * tiles + 8) +
                       sizeof(ProjState) * (PJ_ROUNDS + 1) + 256;
  topo_status s = ensure_red(c, bytes);
  if (s) return s;
  ProjArgs a;
  a.psi = psi;
  a.g = g;
  a.t = t;
  a.scaled = scaled;
  a.vmax = vmax;
  a.n = n;
  a.tiles = tiles;
  char* base = (char*)c->d_red;
  a.st = (ProjState*)base;
  base += sizeof(ProjState) * (PJ_ROUNDS + 1);
  a.part = (double*)base;
  a.maxes = a.part + (size_t)2 * PJ_SLOTS * tiles;
  a.spart = a.maxes + 2 * tiles;
  a.out = out;
  a.stats = stats;
  proj_max_kernel<<<tiles, PJ_THREADS, 0, c->stream>>>(a);
  note_launch();
  for (int r = 0; r < PJ_ROUNDS; ++r) {
    proj_round_kernel<<<tiles, PJ_THREADS, 0, c->stream>>>(a, r);
    note_launch();
  }
  proj_final_kernel<<<tiles, PJ_THREADS, 0, c->stream>>>(a);
  note_launch();
  proj_stats_kernel<<<1, 128, 0, c->stream>>>(a);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_tr_trials(topo_ctx* c, int R, const double* psi_c, const double* psi_x, double* trials,
                                      int ldt) {
  if (!c) return TOPO_ERR_INVALID;
  const long long ne = c->g.nel;
  if (R < 2 || R > 64) return fail(c, TOPO_ERR_INVALID, "topo_tr_trials: 2 <= R <= 64");
  if ((long long)ldt < ne) return fail(c, TOPO_ERR_INVALID, "topo_tr_trials: ldt < N_e");
  if (!dev_ptr_ok(psi_c) || !dev_ptr_ok(psi_x) || !dev_ptr_ok(trials))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_trials: null or misaligned pointer");
  tr_trials_kernel<<<(int)grid_for(c, ne * R), 256, 0, c->stream>>>(R, psi_c, psi_x, trials, ldt, ne);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_tr_select(topo_ctx* c, topo_tr_state* st, const topo_tr_params* prm, int R,
                                      const double* Jk, const double* resnorm, const double* gtd,
                                      const double* trials, int ldt, const double* Phi, int k, int ld,
                                      const double* yhat, double* psi_hat, double* u_hat) {
  if (!c) return TOPO_ERR_INVALID;
  const long long ne = c->g.nel, N = c->g.ndof;
  if (!prm) return fail(c, TOPO_ERR_INVALID, "topo_tr_select: null parameters");
  if (R < 2 || R > 64) return fail(c, TOPO_ERR_INVALID, "topo_tr_select: 2 <= R <= 64");
  if (k < 1 || k > 128) return fail(c, TOPO_ERR_INVALID, "topo_tr_select: 1 <= k <= 128");
  if ((long long)ldt < ne || (long long)ld < N) return fail(c, TOPO_ERR_INVALID, "topo_tr_select: ldt < N_e or ld < N");
  if (!(prm->c1 >= 0.0 && prm->c1 < 1.0)) return fail(c, TOPO_ERR_INVALID, "topo_tr_select: 0 <= c1 < 1 required");
  if (!dev_ptr_ok(st) || !dev_ptr_ok(Jk) || !dev_ptr_ok(resnorm) || !dev_ptr_ok(gtd) || !dev_ptr_ok(trials) ||
      !dev_ptr_ok(Phi) || !dev_ptr_ok(yhat) || !dev_ptr_ok(psi_hat) || !dev_ptr_ok(u_hat))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_select: null or misaligned pointer");
  tr_select_kernel<<<1, 32, 0, c->stream>>>(st, R, Jk, resnorm, gtd, prm->c1);
  note_launch();
  tr_gather_kernel<<<(int)grid_for(c, N > ne ? N : ne), 256, k * sizeof(double), c->stream>>>(
      st, trials, ldt, ne, Phi, ld, k, yhat, psi_hat, u_hat, N);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}

extern "C" topo_status topo_tr_update(topo_ctx* c, topo_tr_state* st, const topo_tr_params* prm, const double* J_hat,
                                      double* psi_c, const double* psi_hat, double* u_c, const double* u_hat,
                                      double* g_c, const double* g_hat, double* u_slot) {
  if (!c) return TOPO_ERR_INVALID;
  const long long ne = c->g.nel, N = c->g.ndof;
  if (!prm) return fail(c, TOPO_ERR_INVALID, "topo_tr_update: null parameters");
  if (!(prm->gamma1 > 0.0 && prm->gamma1 <= prm->gamma2 && prm->gamma2 <= 1.0 && prm->eta1 > 0.0 &&
        prm->eta1 < prm->eta2 && prm->eta2 < 1.0 && prm->grow >= 1.0))
    return fail(c, TOPO_ERR_INVALID,
                "topo_tr_update: 0 < gamma1 <= gamma2 <= 1, 0 < eta1 < eta2 < 1 and grow >= 1 required");
  if (!dev_ptr_ok(st) || !dev_ptr_ok(J_hat) || !dev_ptr_ok(psi_c) || !dev_ptr_ok(psi_hat) || !dev_ptr_ok(u_c) ||
      !dev_ptr_ok(u_hat) || !dev_ptr_ok(g_c) || !dev_ptr_ok(g_hat) || (u_slot && !dev_ptr_ok(u_slot)))
    return fail(c, TOPO_ERR_INVALID, "topo_tr_update: null or misaligned pointer");
  tr_update_kernel<<<1, 32, 0, c->stream>>>(st, *prm, J_hat);
  note_launch();
  tr_move_kernel<<<(int)grid_for(c, N > ne ? N : ne), 256, 0, c->stream>>>(st, ne, N, psi_c, psi_hat, u_c, u_hat,
                                                                           g_c, g_hat, u_slot);
  note_launch();
  TOPO_CUDA_TRY(c, cudaGetLastError());
  return TOPO_OK;
}
