/*
 * libtopo: C ABI of the GB300 (sm_103a) hot path of the ROM-accelerated minimum-compliance
 * SIMP method of Yano, Huang and Zahr (arXiv 2004.05756).
 *
 * The operator behind every call is the penalised linear-elasticity stiffness
 *     K(rho) = sum_e E(rho_e) P_e K_e P_e^T,   E(rho) = Emin + rho^p (E0 - Emin)
 * (Section 2.1, Eq. linelast-res1, with the material law written as Emin/E0; the paper's
 * alpha(rho) = rho_l + (1 - rho_l) rho^p is Emin = rho_l E0), applied matrix-free on a
 * structured grid of unit Q4 (2D, plane stress) or H8 (3D) elements.
 *
 * Conventions shared by all calls:
 *   - Node n = i + (nx+1)(j + (ny+1)k), x fastest. DOF = dim*n + c (interleaved).
 *     Element e = i + nx(j + ny k). N = dim * nodes, N_e = elements.
 *   - Vector blocks are column-major N x m with leading dimension ld >= N (in elements).
 *   - Homogeneous Dirichlet DOFs stay in the vectors: their rows and columns of K act as the
 *     identity and the loads must be zero there. On the free DOFs this is exactly the
 *     paper's elimination of Dirichlet DOFs (the remark after Eq. linelastU).
 *   - Every array argument is a DEVICE pointer owned by the caller, 8-byte aligned, unless a
 *     comment says "host". The context owns only its own scratch.
 *   - Calls are asynchronous and ordered on the CUDA stream given to topo_create. Scalar
 *     outputs are device pointers. A call that must return host data (noted below)
 *     synchronises the stream.
 *   - Every call returns a topo_status and never aborts or traps. Invalid arguments return
 *     TOPO_ERR_INVALID before anything is launched; topo_last_error() gives a message.
 *     Errors found on the device (non-SPD reduced matrix, timeouts in device-side waits,
 *     breakdown) are recorded in a sticky device status word read by topo_check().
 *   - A context must not be used from two host threads at once.
 */
#ifndef TOPO_H
#define TOPO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct topo_ctx topo_ctx;

typedef enum {
  TOPO_OK = 0,
  TOPO_ERR_INVALID = 1,       /* bad argument, shape, pointer or problem description */
  TOPO_ERR_OOM = 2,           /* scratch allocation failed */
  TOPO_ERR_NOT_CONVERGED = 3, /* PCG reached maxit before rtol */
  TOPO_ERR_NOT_SPD = 4,       /* non-positive pivot in the k x k Cholesky or p^T K p <= 0 */
  TOPO_ERR_TIMEOUT = 5,       /* a device-side wait gave up (bounded spin) */
  TOPO_ERR_CUDA = 6           /* a CUDA runtime call failed */
} topo_status;

/* Arithmetic of the operator applications inside a call.
 *   TOPO_FP64               every step in FP64.
 *   TOPO_FP32_REFINED       K(rho)V with FP32 vectors, FP32 E(rho) and FP32 K_e, wrapped in
 *                           FP64-residual iterative refinement where the call has a fixed
 *                           point (topo_solve_hdm, topo_rom_solve).
 *   TOPO_FP32_BF16KE_REFINED as above but K_e entries rounded to BF16 (scaled per element by
 *                           E(rho_e), FP32 accumulation). */
typedef enum { TOPO_FP64 = 0, TOPO_FP32_REFINED = 1, TOPO_FP32_BF16KE_REFINED = 2 } topo_prec;

/* Problem description. dim = 2 (Q4, nz ignored) or 3 (H8). 1 <= nx, ny, nz; N < 2^31.
 * E0 > Emin >= 0; 0 <= nu < 0.5; penal an integer in [1, 6]; rmin in (0, 6] is the radius
 * of the linear density filter in element lengths. fixed_dof_mask is a HOST array of N bytes
 * (non-zero = homogeneous Dirichlet DOF), copied at creation. */
typedef struct {
  int dim, nx, ny, nz;
  double E0, Emin, nu, penal, rmin;
  const unsigned char* fixed_dof_mask;
} topo_problem;

/* Host-side report of topo_solve_hdm (max over load cases). */
typedef struct {
  int iters;      /* total PCG iterations (inner FP32 iterations for refined forms) */
  int outer;      /* FP64 refinement steps (0 for TOPO_FP64) */
  double relres;  /* final ||f - K u||_2 / ||f||_2 over free DOFs, FP64 */
  int status;     /* topo_status of the solve */
  double floor;   /* 2 eps || |K| |u| ||_2 / ||f||_2: the FP64 rounding floor of any residual of
                     u. The FP64 solves accept relres <= max(rtol, floor): designs that put loads
                     on near-void material cannot go below it (0 when not computed) */
  int poly;       /* degree of the polynomial preconditioner of the FP64 stencil solve (1 =
                     Jacobi; each iteration then applies K poly times); 0 for the other solvers
                     and for the multigrid preconditioner */
  int mg_levels;  /* levels of the multigrid preconditioner of the FP64 stencil solve (0 when the
                     solve used another preconditioner) */
  int fallback;   /* 1 when the multigrid solve continued with the polynomial preconditioner from
                     its true residual: the FP32 V-cycle stopped being positive definite, or the
                     residual stopped halving within 64 iterations (conditioning beyond FP32) */
} topo_solve_info;

/* Tunable parameters (topo_set_param). */
typedef enum {
  TOPO_PARAM_INNER_RTOL = 0,   /* relative tolerance of each FP32 inner PCG solve (default 1e-5) */
  TOPO_PARAM_MAX_OUTER = 1,    /* max FP64 refinement steps (default 30) */
  TOPO_PARAM_WAIT_CYCLES = 2,  /* spin limit of device-side waits, in SM clock cycles (default 2e9) */
  TOPO_PARAM_ROM_REFINE = 3,   /* max FP64 refinement steps of the reduced solve (default 8) */
  TOPO_PARAM_TILE_X = 4,       /* columns per CTA of the 2D node-centric block apply (the
                                  autotuned split of a K(rho) V launch; 0 = default) */
  TOPO_PARAM_PCG_BLOCKS_PER_SM = 5, /* CTAs per SM of the persistent PCG (0 = occupancy) */
  TOPO_PARAM_INNER_CAP = 6,        /* max FP32 inner iterations per refinement step (default 2000) */
  TOPO_PARAM_HDM_KERNEL = 7,       /* FP64 solve: 0 = K(rho) assembled once per solve as a per-node
                                      stencil, Chronopoulos-Gear PCG (default); 1 = element-form PCG */
  TOPO_PARAM_PCG_MAX_CTAS = 8,     /* cap on the CTAs of one persistent FP64 solve (0 = whole GPU);
                                      lets solves of several contexts share the GPU concurrently and
                                      fixes their reduction order independently of load */
  TOPO_PARAM_ROM_TENSOR = 9,       /* contraction Phi^T W of the FP32 projection forms of
                                      topo_rom_solve: 1 = tensor cores (tcgen05 kind::tf32 on an exact
                                      hi/lo split of each FP32 operand, FP32 accumulate per 256 rows,
                                      FP64 beyond; default), 0 = SIMT FP32 */
  TOPO_PARAM_APPLY_STAGES = 10,    /* 2D FP32 block apply with ld % 4 == 0 and V 16-byte aligned:
                                      2, 3 (default) or 4 = halo rows staged by TMA (one box per
                                      halo row and 8 columns) with that many tile-column units in
                                      flight per CTA of a persistent grid; 0 = per-thread cp.async
                                      staging (the form used for other leading dimensions) */
  TOPO_PARAM_PCG_POLY = 11,        /* FP64 solve (TOPO_PARAM_HDM_KERNEL 0): preconditioner
                                      z = p(D^-1 K) D^-1 r, p from d steps of the Chebyshev
                                      iteration on [lambda_max/100, lambda_max], lambda_max the
                                      Gershgorin bound of D^-1 K, evaluated in FP32 on an FP32 copy
                                      of the stencil (the CG, its residuals and the stopping test
                                      stay FP64). d = 1 is Jacobi; 2-8 trade d - 1 more operator
                                      applies (halo exchanges, no grid barrier) per iteration for
                                      fewer iterations and reductions; 0 = automatic (default: 8 in
                                      2D, 4 in 3D). Used when TOPO_PARAM_PCG_MG is 0 */
  TOPO_PARAM_PCG_MG = 12,          /* FP64 solve (TOPO_PARAM_HDM_KERNEL 0): 1 (default) = geometric
                                      multigrid V-cycle preconditioner: Galerkin coarse operators
                                      P^T K P of linear interpolation, formed in FP64 once per
                                      solve, Chebyshev smoothing on [lambda_max/30, lambda_max]
                                      per level, the coarsest level (<= 160 DOFs) solved with its
                                      dense inverse; the V-cycle runs in FP32 and the CG, its
                                      residuals and stopping test in FP64. 0 = the polynomial /
                                      Jacobi preconditioner of TOPO_PARAM_PCG_POLY. Meshes too small
                                      to coarsen use the polynomial */
  TOPO_PARAM_MG_DEGREE = 13,       /* multigrid: Chebyshev smoothing steps before and after the
                                      coarse correction, 1 .. 4 (default 2) */
  TOPO_PARAM_MG_SINGLE_NODES = 14, /* multigrid: coarse levels with at most this many nodes run on
                                      one CTA, their vectors in its shared memory, with block
                                      barriers instead of halo exchanges between CTAs (default
                                      -1: 1024 in 2D, 0 in 3D; levels whose vectors do not fit
                                      96 KB with those of
                                      the coarser levels stay on all CTAs; the coarsest level
                                      always runs on one CTA and level 0 never does) */
  TOPO_PARAM_FILTER = 15,          /* density filter of topo_filter and of every call that filters
                                      (topo_rom_eval_batch, topo_compliance_grad's dc_psi): 0 = the
                                      linear cone filter of radius rmin (default); 1 = the Helmholtz
                                      filter of Section 2.2 (Eq. helm-soln .. cdens-star): nodal
                                      phi = H^-1 b(psi) with the Q1 Helmholtz operator
                                      -r^2 Lap + 1 under Neumann conditions, rho_e = the average of
                                      phi over the element's nodes. Solved exactly by the cosine
                                      eigenvectors of the 1D Q1 Neumann matrices (two transforms of
                                      FP64 mode products and a diagonal scaling); self-adjoint, so
                                      adjoint = 1 gives the same map */
  TOPO_PARAM_HELMHOLTZ_R = 16,     /* the Helmholtz length r in element lengths (0 = default:
                                      rmin / (2 sqrt 3), the length the filter's cited reference
                                      relates to a cone radius rmin; the paper prints
                                      r = 2 sqrt(3) R) */
  TOPO_PARAM_ROM_ASSEMBLY = 17     /* contraction H_r = sum_e E(rho_r,e) Hel[e] of
                                      topo_rom_eval_batch and topo_rom_assemble_batch: 1 (default) =
                                      tensor cores (tcgen05 kind::f16) on the Ozaki scheme's exact
                                      split of each FP64 operand into 8 BF16 digits, with exact
                                      FP32 sums over 512 element rows and FP64 beyond: each entry
                                      within about 2^-51 of sum_e |E_e| |Hel[e]| of the exact sum,
                                      up to 128 candidates per pass over Hel; 0 = FP64 SIMT (the
                                      rounding of FP64 sums), 32 candidates per pass */
} topo_param;

/* Create a context for one problem; computes K_e (2x2(x2) Gauss quadrature), the filter
 * weights and normalisers, and uploads the Dirichlet mask. cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) that the context borrows. The current CUDA device at
 * creation is the context's device. Allocates device scratch. */
topo_status topo_create(const topo_problem* prob, void* cuda_stream, topo_ctx** out);
topo_status topo_destroy(topo_ctx* ctx);
const char* topo_last_error(const topo_ctx* ctx);
topo_status topo_set_param(topo_ctx* ctx, topo_param which, double value);

/* Synchronise the context's stream and return (and clear) the sticky device status. */
topo_status topo_check(topo_ctx* ctx);

/* Diagnostics: total number of CUDA kernel launches issued by the library in this process,
 * over all contexts (host output). */
topo_status topo_launch_count(long long* out);

/* Sizes of the context's problem (host outputs; any may be NULL). */
topo_status topo_sizes(const topo_ctx* ctx, long long* ndof, long long* nel, long long* nnodes);

/* Linear density filter (the benchmark's replacement of the Helmholtz filter of
 * Section 2.2, Eq. cdens-star): w_ei = max(0, rmin - |c_e - c_i|), Hs_e = sum_i w_ei.
 * adjoint == 0: out_e = sum_i w_ei in_i / Hs_e           (rho = filter(psi))
 * adjoint != 0: out_i = sum_e w_ei in_e / Hs_e           ((d rho/d psi)^T v, used by
 *                                                          Eq. pap_sensitivity)
 * in, out: FP64[N_e], must not alias. */
topo_status topo_filter(topo_ctx* ctx, const double* in, double* out, int adjoint);

/* Y = K(rho) V for m columns (Eq. linelast-res1, matrix-free). rho: FP64[N_e] in [0, 1].
 * V, Y: N x m with leading dimension ld, FP64 for TOPO_FP64, FP32 otherwise. Dirichlet rows
 * give Y = V. V and Y must not alias. m = 0 is a no-op. */
topo_status topo_apply_K(topo_ctx* ctx, const double* rho, const void* V, void* Y, int m, int ld,
                         topo_prec prec);

/* State solve K(rho) u = f (Eq. linelastsoln) for m load cases by Jacobi-preconditioned CG
 * in one persistent cooperative launch, to ||f - K u||_2 <= rtol ||f||_2 over free DOFs
 * (each column separately; the reported residual is the true FP64 one). The FP32 forms run
 * FP32 inner PCG inside FP64 iterative refinement; a refinement step that fails to halve the
 * FP64 residual norm (eps_32 * cond(K) too large for the design) stops the refinement and
 * the call finishes with FP64 PCG from the current iterate, so those forms synchronise. F, U: FP64 N x m, ld; U holds the initial guess on entry and
 * the solution on exit (Dirichlet DOFs set to 0). maxit bounds the (inner) iterations.
 * info_host (host, may be NULL): if non-NULL the call synchronises and fills it, and
 * returns TOPO_ERR_NOT_CONVERGED when rtol was not reached. */
topo_status topo_solve_hdm(topo_ctx* ctx, const double* rho, const double* F, double* U, int m,
                           int ld, double rtol, int maxit, topo_prec prec,
                           topo_solve_info* info_host);

/* Reduced basis from snapshots (Eq. rob-optim; for compliance the adjoint snapshots equal
 * the primal ones): classical Gram-Schmidt applied twice to the columns of Usnap (FP64
 * N x m, ld) in order, dropping a column whose orthogonalised norm is < 1e-10 times the
 * largest snapshot norm. Writes the k kept orthonormal columns to Phi (FP64, capacity
 * N x m, same ld), then H = Phi^T K(rho) Phi (FP64 k x k, row-major, leading dimension k,
 * capacity m*m) and b = Phi^T f (FP64[k]; f FP64[N]) (Eq. hatkbm). H may be NULL: then only
 * Phi and b are formed (the element path forms H(rho) per density from topo_rom_elem). k_out
 * is a HOST int; the call synchronises to return it. Usnap and Phi may be the same buffer. */
topo_status topo_rom_build(topo_ctx* ctx, const double* rho, const double* Usnap, int m, int ld,
                           double* Phi, int* k_out, double* H, double* b, const double* f);

/* POD of a snapshot block (Section 4.2, Eq. rob-optim: POD_n, the first n left singular vectors,
 * of the previous trust-region centres' states): U is N x m at ld (1 <= m <= 64); column skip
 * (-1 = none) is left out; Pod (N x (n + 1 if append else n), ldp) receives the n leading left
 * singular vectors of the remaining m' columns, orthonormal, followed by a copy of append
 * (FP64[N], may be NULL): the block whose Gram-Schmidt orthonormalisation (topo_rom_build) is the
 * basis of Eq. rob-optim. sigma (device FP64[m']) receives the singular values in descending
 * order when n >= 1. 0 <= n <= m'. Method: the Gram matrix U^T U in FP64 and its cyclic Jacobi
 * eigen-decomposition on one CTA: a singular value carries an error of about
 * eps sigma_max^2 / sigma_i and its vector a loss of orthogonality of about eps sigma_max^2 /
 * sigma_i^2; one below about 1.2e-7 of the largest is rounding noise of the Gram matrix, and its
 * vector is returned as zero (topo_rom_build then drops it). */
topo_status topo_rom_pod(topo_ctx* ctx, const double* U, int m, int ld, int skip, int n, const double* append,
                         double* Pod, int ldp, double* sigma);

/* Reduced solve at a new density (Section 3.1 and the cost analysis of Section 3.4):
 * H(rho) = Phi^T K(rho) Phi, Cholesky H = L L^T in FP64, yhat = H^{-1} b, Jk = b^T yhat.
 * Phi: FP64 N x k, ld; b FP64[k]; H_work FP64 k*k (on exit: L in the lower triangle,
 * row-major); yhat FP64[k]; Jk device FP64 scalar. 1 <= k <= 128.
 * prec TOPO_FP64: H with FP64 applies and contraction.
 * prec FP32 forms: H from FP32 applies and contraction, then yhat is refined with FP64
 * reduced residuals b - Phi^T K(rho) Phi yhat (at most TOPO_PARAM_ROM_REFINE steps).
 * A non-positive pivot sets TOPO_ERR_NOT_SPD in the device status and yhat = NaN. */
topo_status topo_rom_solve(topo_ctx* ctx, const double* rho, const double* Phi, int k, int ld,
                           const double* b, double* H_work, double* yhat, double* Jk,
                           topo_prec prec);

/* Element reduced matrices of a basis (Eq. hatkbm written per element, Remark rom_assemble):
 * Hel[e] = (P_e^T Phi)^T K_e (P_e^T Phi) at unit density, independent of rho. Stored as
 * (N_e + 1) rows of npair = k(k+1)/2 FP64 words (upper triangle, row-major packed); row N_e
 * is Phi_D^T Phi_D over the Dirichlet DOFs (the identity part of the operator convention).
 * Phi: FP64 N x k, ld. Hel: caller-owned, (N_e + 1) * npair FP64. 1 <= k <= 128. Compute once
 * per basis; every later density needs only topo_rom_solve_elem. */
topo_status topo_rom_elem(topo_ctx* ctx, const double* Phi, int k, int ld, double* Hel);

/* Reduced solve from element reduced matrices: H(rho) = sum_e E(rho_e) Hel[e] + Hel[N_e] (a
 * streaming, deterministic reduction over the elements), then the FP64 Cholesky solve of
 * topo_rom_solve: H_work (k*k, on exit L), yhat[k], Jk (device scalar). */
topo_status topo_rom_solve_elem(topo_ctx* ctx, const double* rho, const double* Hel, int k, const double* b,
                                double* H_work, double* yhat, double* Jk);

/* topo_rom_solve_elem without any device allocation. The paper has no counterpart: this
 * entry exists for callers that cannot allocate device memory when they need a reduced solve
 * (a serving loop whose memory budget belongs to an outside allocator, code running while
 * another component holds the device pool, or a latency-critical loop that cannot accept the
 * implicit device synchronisation of cudaMalloc/cudaFree). Same arguments and results as
 * topo_rom_solve_elem, with 1 <= k <= 64. Its scratch is one fixed 8 MiB device array inside the
 * library (kept by every GPU that loads the library until the process exits); a problem that
 * needs more (about N_e + 1 + 2 * SMs * k(k+1)/2 doubles) is rejected with TOPO_ERR_INVALID and
 * a message. The first call on each device looks up the array's device address; make that
 * first call before any stream capture. All calls share the array, so calls that overlap on
 * the GPU (other streams, other contexts, other host threads) race: serialise them. */
topo_status topo_rom_solve_elem_noalloc(topo_ctx* ctx, const double* rho, const double* Hel, int k,
                                        const double* b, double* H_work, double* yhat, double* Jk);

/* ROM design evaluations of R candidate designs on one resident basis, in one call (the
 * candidates of a trust-region step, Algorithm 2; each evaluation as Section 3.1 Eq. rom_soln,
 * Section 3.3 and Remark topopt_compl):
 *   rho_r = filter(psi_r) (filtered != 0; else psi_r is the density),
 *   H_r = sum_e E(rho_r,e) Hel[e] + Hel[N_e] (element reduced matrices of topo_rom_elem),
 *   y_r = H_r^-1 b by FP64 Cholesky, Jk[r] = b^T y_r,
 *   u_r = Phi y_r, resnorm[2r] = ||f - K(rho_r) u_r||_2 and resnorm[2r+1] = that / ||f||_2
 *   (free DOFs, FP64),
 *   dpsi_r = filter^T(-E'(rho_r) u_r,e^T K_e u_r,e) (or the unfiltered gradient when filtered
 *   is 0), when dpsi is not NULL.
 * psi: R fields of N_e doubles at stride ldp >= N_e; Phi: N x k at leading dimension ld;
 * Hel: (N_e + 1) x k(k+1)/2 from topo_rom_elem for this Phi; b = Phi^T f (FP64[k]); f FP64[N].
 * Outputs (device): Jk[R], resnorm[2R], yhat[R*k] (may be NULL), dpsi (R fields at stride ldp,
 * may be NULL; must not alias psi). 1 <= k <= 128. Every candidate's results equal those of the
 * one-candidate calls (topo_filter, topo_rom_solve_elem, topo_rom_error,
 * topo_compliance_grad) up to the rounding order of their sums, and do not depend on the other
 * candidates of the batch. A non-positive pivot sets TOPO_ERR_NOT_SPD in the device status and
 * NaN for that candidate. Asynchronous on the context's stream. */
topo_status topo_rom_eval_batch(topo_ctx* ctx, int R, const double* psi, int ldp, int filtered,
                                const double* Hel, const double* Phi, int k, int ld, const double* b,
                                const double* f, double* Jk, double* resnorm, double* yhat, double* dpsi);

/* Reduced matrices of R densities on one basis from their moduli (Section 3.4, Remark
 * rom_assemble): H[r] = sum_{e < N_e} E[r][e] Hel[e] + E[r][N_e] Hel[N_e], unpacked to k x k
 * row-major. E: R rows of N_e + 1 doubles at stride ldE >= N_e + 1 (E[r][e] = E(rho_e) for
 * e < N_e and E[r][N_e] = 1 give the H of topo_rom_solve_elem); Hel from topo_rom_elem; H:
 * device FP64[R * k * k]. R >= 0, 1 <= k <= 128. The contraction is the one
 * TOPO_PARAM_ROM_ASSEMBLY selects; each H[r] depends only on row r of E. Asynchronous on the
 * context's stream. */
topo_status topo_rom_assemble_batch(topo_ctx* ctx, int R, const double* E, long long ldE, const double* Hel, int k,
                                    double* H);

/* A posteriori residual (Section 3.3; the trust-region constraint of Eq. trcon-topopt):
 * u_k = Phi yhat, r = f - K(rho) u_k on the free DOFs, resnorm[0] = ||r||_2,
 * resnorm[1] = ||r||_2 / ||f||_2 (device FP64[2]). uk_opt (FP64[N], may be NULL) receives
 * u_k. Always FP64. */
topo_status topo_rom_error(topo_ctx* ctx, const double* rho, const double* Phi, int k, int ld,
                           const double* yhat, const double* f, double* resnorm, double* uk_opt);

/* Compliance and its gradient (Section 2.3 and Eq. pap_sensitivity with lambda = u,
 * Remark topopt_compl): J = sum_c f_c^T u_c (device scalar), ce_e = sum_c u_{c,e}^T K_e
 * u_{c,e}, dc_rho_e = -p (E0 - Emin) rho_e^(p-1) ce_e (FP64[N_e]), and, if dc_psi is non-NULL,
 * dc_psi = filter adjoint of dc_rho (FP64[N_e]). U, F: FP64 N x m, ld. Works for HDM states
 * and ROM reconstructions alike. */
topo_status topo_compliance_grad(topo_ctx* ctx, const double* rho, const double* U, int m, int ld,
                                 const double* F, double* J, double* dc_rho, double* dc_psi);

/* General linear output j(u) = sum_c l_c^T u_c (Section 2.3-2.4; Eq. pap_sensitivity with
 * dj/drho = 0): J = sum_c l_c^T u_c (device scalar), dc_rho_e = -p (E0 - Emin) rho_e^(p-1)
 * sum_c lambda_{c,e}^T K_e u_{c,e} with the adjoint states Lam (K lambda_c = l_c, Eq.
 * linelast-adj1: topo_solve_hdm with the output vectors as loads, K being symmetric), and, when
 * dc_psi is not NULL, its filter adjoint. U, Lam, L: FP64 N x m at ld; Dirichlet rows of Lam
 * are ignored. With Lam = U and L = F this is topo_compliance_grad. Works for full-order states
 * and for ROM reconstructions u_k = Phi y, lambda_k = Phi z (Section 3.2) alike. */
topo_status topo_output_grad(topo_ctx* ctx, const double* rho, const double* U, const double* Lam, int m, int ld,
                             const double* L, double* J, double* dc_rho, double* dc_psi);

/* sigma_min(K(rho)) over the free DOFs, the constant of the a posteriori bounds of Section 3.3
 * (Theorem rom_primal_error: ||u - u_k||_K <= sigma_min^-1/2 ||r||; for compliance
 * |J - J_k| <= sigma_min^-1 ||r||^2), by shift-invert Lanczos: steps Lanczos steps on K^-1 (each one
 * topo_solve_hdm at rtol, FP64, from a start vector that is zero on Dirichlet DOFs, with full
 * CGS2 reorthogonalisation), then the largest eigenvalue theta of the tridiagonal matrix and its
 * Ritz residual res = beta_m |s_m|. out (device FP64[4]): 1 / theta (the estimate; never below
 * sigma_min in exact arithmetic), 1 / (theta + res) (below sigma_min when the Ritz value belongs
 * to K^-1's largest eigenvalue: the lower bound to use in the error bounds), theta, res.
 * 2 <= steps <= 64, 0 < rtol <= 1e-2. Allocates its Lanczos vectors ((steps + 1) N doubles) and
 * synchronises the stream; a solve that does not converge returns TOPO_ERR_NOT_CONVERGED. */
topo_status topo_sigma_min(topo_ctx* ctx, const double* rho, int steps, double rtol, double* out);

/* Reduced load of a vector (Section 3.1 Eq. hatkbm's f_k = Phi^T f; Section 3.2's adjoint load
 * Phi^T dj/du^T): out = Phi^T v (device FP64[k]); Phi N x k at ld, v FP64[N]. 1 <= k <= 128. */
topo_status topo_rom_rhs(topo_ctx* ctx, const double* Phi, int k, int ld, const double* v, double* out);

/* ---------------------------------------------------------------------------------------
 * Trust-region step of one major iteration of the error-aware trust-region method
 * (Algorithm 2, Section 4.2; Algorithm 1 for the acceptance and radius rule) for compliance.
 * A run's state lives in device memory and every decision (trial selection, acceptance,
 * radius) is taken on the device, so a major iteration needs no host read-back:
 *   topo_tr_project  target psi_x = P_C(psi_c - (move / ||g||_inf) g)   (step 3, subproblem)
 *   topo_tr_trials   psi_s = psi_c + s (psi_x - psi_c), s = 0, 1, 1/2, ...
 *   topo_rom_eval_batch on the trials                            (m_k and theta_k, step 3)
 *   topo_tr_select   the candidate psi_hat and its reduced state
 *   topo_filter, topo_solve_hdm, topo_compliance_grad at psi_hat      (J(psi_hat), step 4)
 *   topo_tr_update   varrho_k, acceptance, Delta_{k+1}                (steps 4-6)
 * The subproblem (step 3) is solved approximately by one projected-gradient step with
 * backtracking, the Armijo rule along a feasible direction (Bertsekas, Nonlinear Programming,
 * Section 2.3), stopped at the trust-region constraint as the paper stops its MMA iterations
 * (end of Section 4.2); the feasible set is convex, so every trial is feasible.
 * --------------------------------------------------------------------------------------- */

/* Device-resident state of one run (128 bytes, caller-owned device memory, 8-byte aligned). */
typedef struct {
  double delta;      /* Delta_k, the current radius (after topo_tr_update: Delta_{k+1}) */
  double delta_max;  /* Delta_max */
  double delta_prev; /* the radius the last update started from */
  double J_c;        /* J(psi^(k)), full-order compliance at the centre */
  double Jk_c;       /* m_k(psi^(k)), reduced compliance at the centre (trial 0) */
  double Jk_hat;     /* m_k(psi_hat) */
  double J_hat;      /* J(psi_hat) */
  double theta_hat;  /* theta_k(psi_hat) = ||f - K(rho(psi_hat)) u_k(psi_hat)||_2 (Eq. trcon-topopt) */
  double step;       /* s of the candidate: psi_hat = psi^(k) + s (psi_x - psi^(k)) */
  double ratio;      /* varrho_k; -inf when the predicted reduction is not positive */
  double gtd;        /* g . (psi_x - psi^(k)), the slope the decrease test uses */
  double pad0;
  int sel;           /* trial index of the candidate (1 .. R-1) */
  int inside;        /* 1 when the candidate passed both tests of topo_tr_select */
  int accepted;      /* 1 when psi^(k+1) = psi_hat */
  int iter;          /* major iterations completed */
  int pad1[4];
} topo_tr_state;

/* Host parameters of the acceptance and radius rule (Algorithm 2, steps 5-6) and of the
 * decrease test. Section 5 uses gamma1 = 0.5, gamma2 = 1, eta1 = 0.1, eta2 = 0.75. */
typedef struct {
  double gamma1, gamma2; /* radius factors below eta1 and on [eta1, eta2) */
  double eta1, eta2;     /* acceptance and very-successful thresholds */
  double grow;           /* radius factor from eta2 on, capped at delta_max (the paper leaves it open) */
  double c1;             /* Armijo constant of the decrease test, 0 <= c1 < 1 */
} topo_tr_params;

/* State of a new run at its first centre: delta = tau ||r(0, rho)||_2 = tau ||f||_2 over the free
 * DOFs (Eq. trrad0), delta_max = dmax_factor * delta (Section 5: 100), J_c = *J_c (device
 * scalar, from topo_compliance_grad), every other field zero. f: FP64[N] (device). tau > 0,
 * dmax_factor >= 1. */
topo_status topo_tr_init(topo_ctx* ctx, topo_tr_state* st, const double* f, double tau, double dmax_factor,
                         const double* J_c);

/* out = P_C(psi - tau g), the Euclidean projection onto C = {x in [0,1]^Ne : sum_e x_e <= vmax}
 * (Eq. feaset-topopt with unit element volumes): out = clip(psi - tau g - mu, 0, 1) with the
 * volume multiplier mu >= 0 found as the root of a piecewise-linear function, exactly on its
 * last linear piece. tau = t, or t / max_e |g_e| when scaled != 0 (t is then a move limit in
 * design units). g may be NULL (a plain projection of psi: the feasibility restoration of a
 * starting design). With t = 1, scaled = 0 and g = grad J, stats[1] is the criticality measure
 * ||psi - P_C(psi - grad J)|| of Section 4.1. All FP64[N_e] device arrays; out may alias psi
 * but not g. stats (device FP64[4]): g.(out - psi) (0 without g), ||out - psi||_2, mu,
 * sum_e out_e. vmax >= 0 (+inf: box only). Deterministic: the sums run in a fixed order. */
topo_status topo_tr_project(topo_ctx* ctx, const double* psi, const double* g, double t, int scaled, double vmax,
                            double* out, double* stats);

/* Trial designs: row r of trials (stride ldt >= N_e) = psi_c + s_r (psi_x - psi_c) with s_0 = 0
 * and s_r = 2^-(r-1), r = 1 .. R-1 (each rounded once: s_r (psi_x - psi_c) is exact). 2 <= R <= 64. */
topo_status topo_tr_trials(topo_ctx* ctx, int R, const double* psi_c, const double* psi_x, double* trials, int ldt);

/* The candidate of a trust-region step from the reduced evaluations of the trials (Jk[R] and
 * resnorm[2R] of topo_rom_eval_batch, yhat[R*k]): the smallest r >= 1 with
 *   resnorm[2r] <= st->delta  and  Jk[r] <= Jk[0] + (c1 s_r) * gtd,
 * or r = R - 1 when none passes. Writes st->sel, inside, step, Jk_c = Jk[0], Jk_hat, theta_hat,
 * gtd (= *gtd, device scalar: stats[0] of the topo_tr_project that formed psi_x), and
 * psi_hat = trials[sel] (FP64[N_e]), u_hat = Phi y_sel (FP64[N], Phi N x k at ld), the
 * reduced state at the candidate (the start of its full-order solve). */
topo_status topo_tr_select(topo_ctx* ctx, topo_tr_state* st, const topo_tr_params* prm, int R, const double* Jk,
                           const double* resnorm, const double* gtd, const double* trials, int ldt, const double* Phi,
                           int k, int ld, const double* yhat, double* psi_hat, double* u_hat);

/* Algorithm 2, steps 4-6, after the full-order evaluation of the candidate (J_hat: device
 * scalar): varrho_k = (J_c - J_hat) / (Jk_c - Jk_hat) (-inf when the denominator is not
 * positive); accepted = varrho_k >= eta1; delta <- gamma1 delta when not accepted, gamma2 delta
 * when varrho_k < eta2, else min(grow delta, delta_max). On acceptance J_c <- J_hat and the
 * candidate's design, state and gradient are copied over the centre's (psi_c, u_c: FP64[N_e],
 * FP64[N]; g_c <- g_hat, FP64[N_e]) and, when u_slot is not NULL, its state into u_slot (a
 * column of the snapshot window). Nothing is copied on rejection. */
topo_status topo_tr_update(topo_ctx* ctx, topo_tr_state* st, const topo_tr_params* prm, const double* J_hat,
                           double* psi_c, const double* psi_hat, double* u_c, const double* u_hat, double* g_c,
                           const double* g_hat, double* u_slot);

/* ---------------------------------------------------------------------------------------
 * Batched form: many independent 2D problems (uneven sizes, 1..32 load cases each) behind one
 * handle. Each instance owns a context (topo_batch_context) on the batch's stream, so every
 * single-instance call above also works on it. Argument arrays are HOST arrays of count entries
 * (device pointers inside).
 * --------------------------------------------------------------------------------------- */
typedef struct topo_batch topo_batch;

/* Create count contexts (dim must be 2 for all) on one stream. */
topo_status topo_batch_create(const topo_problem* probs, int count, void* cuda_stream, topo_batch** out);
topo_status topo_batch_destroy(topo_batch* batch);
const char* topo_batch_last_error(const topo_batch* batch);
/* The context of instance i (owned by the batch). */
topo_status topo_batch_context(topo_batch* batch, int i, topo_ctx** out);

/* All state solves (Eq. linelastsoln) of the batch, in one of two forms chosen by the instance
 * contexts' TOPO_PARAM_PCG_MG (set it on every instance through topo_batch_context):
 *  - 1 on every instance (the default): each instance runs topo_solve_hdm's multigrid-
 *    preconditioned FP64 solve as its own persistent cooperative launch with a fixed share of
 *    the SMs (SMs / S CTAs), on one of S internal streams (instances assigned largest first to
 *    the least loaded stream; the streams fork from and join back to the batch's stream). The
 *    first call tunes S over 4, 8 and 16 on short runs.
 *  - otherwise: ONE persistent cooperative launch in which each instance runs the Jacobi-
 *    preconditioned FP64 stencil PCG on its own group of co-resident CTAs (sized by nodes x load
 *    cases x mesh width) with its own barrier and convergence; instances that do not fit the
 *    co-resident capacity run in further waves. The first call tunes the CTAs per SM.
 * Tuning runs save and restore the initial guesses. U[i] holds the initial guess and receives
 * the solution. A call identical to the previous one (same arguments, no info) replays its staged
 * launches without host synchronisation. info_host (host array of count, may be NULL) makes the
 * call synchronise and report per instance (iterations, relative residual, FP64 floor, status,
 * preconditioner fields as topo_solve_hdm). */
topo_status topo_batch_solve_hdm(topo_batch* batch, const double* const* rho, const double* const* F,
                                 double* const* U, const int* m, const int* ld, double rtol, int maxit,
                                 topo_solve_info* info_host);
/* topo_filter on every instance. */
topo_status topo_batch_filter(topo_batch* batch, const double* const* in, double* const* out, int adjoint);
/* topo_compliance_grad on every instance; J is a DEVICE array of count compliances. */
topo_status topo_batch_compliance_grad(topo_batch* batch, const double* const* rho, const double* const* U,
                                       const int* m, const int* ld, const double* const* F, double* J,
                                       double* const* dc_rho, double* const* dc_psi);
/* topo_rom_solve_elem on every instance (Section 3.1 Eq. rom_soln with the element reduced
 * matrices of topo_rom_elem); k is a HOST array, Jk a DEVICE array of count. When every k <= 32
 * all instances run in three launches: one assembly of every H_i over a table of (instance, row
 * range) items, one fixed-order reduction per instance, one warp per Cholesky; the tables are
 * staged once and reused while the arguments are unchanged (no host synchronisation then).
 * Otherwise each instance runs topo_rom_solve_elem. A non-positive pivot sets NOT_SPD in that
 * instance's context status and NaN in its y and Jk. */
topo_status topo_batch_rom_solve_elem(topo_batch* batch, const double* const* rho, const double* const* Hel,
                                      const int* k, const double* const* b, double* const* H_work,
                                      double* const* yhat, double* Jk);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_H */
