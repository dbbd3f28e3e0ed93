// Shared by pcg2.cu (the stencil PCG) and batch.cu (its batched launch).
#pragma once

#include "common.cuh"
#include "mg.cuh"

namespace topo {

constexpr int P2_MAX_COLS = 32;
constexpr int P2_MAX_POLY = 8;        // highest degree of the polynomial preconditioner
constexpr int P2_SLOTS = 8;           // reduced values per column and barrier (5 used at most)
constexpr int P2_THREADS = 256;       // batched kernel: up to 4 CTAs per SM
constexpr int P2_THREADS_SOLO = 512;  // single solve: one CTA per SM (half the barrier arrivals)

template <int DIM>
struct Pcg2Args {
  Grid g;
  typename KeOf<DIM, double>::type ke;
  const double* rho;
  const double* F;
  double* U;
  long long ld;
  int m;
  long long N;       // scratch leading dimension (= ndof)
  long long nunits;  // ceil(nnx / 32) * nny * nnz
  double* C;         // [NB*DIM*DIM][nnodes]
  double* dinv;      // [N]
  double* r;         // N x m each
  double* z;
  double* w;
  double* p;
  double* s;
  // polynomial preconditioner (poly > 1 only), all FP32:
  float* C32;        //   the stencil [NB*DIM*DIM][nnodes] and D^-1 [N]
  float* dinv32;
  float* t0;         //   direction vectors, alternating, whose halo its applies read; N x m each
  float* t1;
  float* res;        //   residual of its Chebyshev iteration; N x m
  float* z32;        //   the accumulated result; N x m
  int poly;          // degree of the preconditioner polynomial in D^-1 K (1 = Jacobi)
  double cheb_ratio; // its Chebyshev interval: [lambda_max / cheb_ratio, lambda_max]
  MgArgs mg;         // multigrid preconditioner (the multigrid kernel only)
  double* partial;   // [2 barrier parities][P2_SLOTS slots][m][G]
  unsigned long long* zflag;  // [G]: phase-U completions of each CTA (z published), reset per launch
  GridSync* gs;      // sticky status
  GridBar* gb;
  double rtol;
  int maxit;
  long long wait_cycles;
  int* info;
  double* info_rr;
};

template <int DIM>
struct StencilGeom {
  static constexpr int NB = DIM == 2 ? 9 : 27;
  static constexpr int NC = NB * DIM * DIM;  // coefficients per node
};

// Launch the batched 2D solve kernel: ctas CTAs (co-resident, cooperative) on stream.
cudaError_t launch_pcg2_batch2(unsigned ctas, cudaStream_t stream, const Pcg2Args<2>* args, const int* cta_inst,
                               const int* cta_rank, const int* grp_size);

// Prepare one instance's solve for a group of G CTAs: scratch, stencil and vector pointers,
// barrier state, info words. status is the sticky status word the solve reports into.
// poly > 1 selects the Chebyshev polynomial preconditioner of that degree (three more scratch
// vectors); the batched solve uses 1.
template <int DIM>
topo_status build_pcg2_args(topo_ctx* c, const double* rho, const double* F, double* U, int m, int ld, double rtol,
                            int maxit, int G, Pcg2Args<DIM>* out, GridSync* status, int poly = 1, bool mg = false);

// Resident CTAs per SM of the batched kernel.
int pcg2_occupancy();

// A single 2D solve (topo_solve_hdm's preconditioner choice and arguments) staged for a share of
// at most max_ctas CTAs and launched on a given stream: the batched multigrid form runs many
// concurrently. The solve's info words are a.info (iters, -, status, fallback) and a.info_rr.
struct SoloLaunch2 {
  Pcg2Args<2> a;
  unsigned G;
  size_t dyn;
  int mg;
};
topo_status stage_solo2(topo_ctx* c, const double* rho, const double* F, double* U, int m, int ld, double rtol,
                        int maxit, int max_ctas, SoloLaunch2* out);
cudaError_t launch_solo2(topo_ctx* c, const SoloLaunch2& s, cudaStream_t stream);

}  // namespace topo
