"""One optimisation run of the error-aware trust-region method (Algorithm 2, Section 4.2) for
compliance on one libtopo context.

A major iteration is the sequence of library calls

  model update (step 2)   topo_rom_build (Phi, b from the snapshot window), topo_rom_elem
  step (step 3)           topo_tr_project (psi_x = P_C(psi_c - move g / ||g||_inf)),
                          topo_tr_trials (psi_c + s (psi_x - psi_c), s = 0, 1, 1/2, ...),
                          topo_rom_eval_batch (m_k and theta_k of every trial in one call),
                          topo_tr_select (the candidate and its reduced state)
  ratio (step 4)          topo_filter, topo_solve_hdm (started from the reduced state),
                          topo_compliance_grad at the candidate
  acceptance, radius      topo_tr_update (steps 5-6), then topo_tr_project once more for the
                          criticality measure of the new centre (Section 4.1)

The run's state (centre design, its gradient, the snapshot window whose newest column is the
centre's state, the trust-region radius and the compliances) stays in device memory; every
decision is taken by the library's kernels, and the host reads one small buffer at the end of
the iteration to report it. This module only allocates buffers and sequences calls.
"""
from __future__ import annotations

import numpy as np

from . import native


class TrustRegionRun:
    """State and buffers of one run. psi0 is the starting design (projected onto the feasible
    set first: the closest feasible design). L is the snapshot window (the basis is the
    orthonormalisation of the L most recent centre states)."""

    def __init__(self, T, p, psi0, *, tau: float = 0.1, dmax_factor: float = 100.0, move: float = 0.2,
                 trials: int = 7, volfrac: float = 0.5, L: int = 8, rtol: float = 1e-8, maxit: int = 400000,
                 params: native.topo_tr_params | None = None, alloc_stream=None, pod_nmax: int | None = None):
        import torch
        self.torch = torch
        self.alloc_stream = alloc_stream  # allocate the buffers on this stream's pool (None: current)
        self.T, self.p = T, p
        self.move, self.R, self.L = float(move), int(trials) + 1, int(L)
        # POD truncation (Eq. rob-optim): basis = GramSchmidt([POD_n(previous centres), u_c]) with
        # n = min(previous - 1, pod_nmax); the ring then holds L previous centres and the current
        self.pod_nmax = pod_nmax
        self.ring = self.L + (1 if pod_nmax is not None else 0)
        self.vmax = float(volfrac) * p.nel
        self.rtol, self.maxit = float(rtol), int(maxit)
        self.prm = params if params is not None else native.tr_params()
        self.nwin = 0
        self.hdm_iters = 0
        self.alloc()
        self._start(psi0, tau, dmax_factor)

    # device tensors that carry the run from one major iteration to the next; everything else
    # is rebuilt by each iteration
    CARRIED = ("psi_c", "g_c", "window", "out")

    def alloc(self):
        """Allocate every device buffer of the run (from alloc_stream's pool when one is given;
        the current stream then waits for it)."""
        torch = self.torch
        if self.alloc_stream is None:
            self._alloc()
            return
        with torch.cuda.stream(self.alloc_stream):
            self._alloc()
        torch.cuda.current_stream().wait_stream(self.alloc_stream)

    def _alloc(self):
        torch, p = self.torch, self.p
        f64 = dict(dtype=torch.float64, device="cuda")
        ne, N, R, L = p.nel, p.ndof, self.R, self.ring
        self.F = torch.as_tensor(np.ascontiguousarray(p.F[:, :1].T)).to(**f64)
        self.f = self.F[0]
        self.psi_c = torch.empty(ne, **f64)
        self.g_c = torch.empty(ne, **f64)
        self.window = torch.zeros((L, N), **f64)
        self.Phi = torch.zeros((L, N), **f64)
        self.Hel = torch.zeros((ne + 1) * L * (L + 1) // 2, **f64)
        self.b = torch.zeros(L, **f64)
        self.trials = torch.empty((R, ne), **f64)
        self.Jk = torch.empty(R, **f64)
        self.resnorm = torch.empty((R, 2), **f64)
        self.yhat = torch.empty(R * L, **f64)
        self.psi_x = torch.empty(ne, **f64)
        self.psi_hat = torch.empty(ne, **f64)
        self.u_hat = torch.zeros((1, N), **f64)
        self.g_hat = torch.empty(ne, **f64)
        self.rho = torch.empty(ne, **f64)
        self.dc = torch.empty(ne, **f64)
        self.scratch = torch.empty(ne, **f64)
        self.J = torch.zeros(1, **f64)
        # one buffer read back per iteration: the state (16 doubles) and two projection stats
        self.out = torch.zeros(native.TR_STATE_BYTES // 8 + 8, **f64)
        self.st = self.out[:native.TR_STATE_BYTES // 8]
        self.stats_dir = self.out[16:20]
        self.stats_crit = self.out[20:24]
        if self.pod_nmax is not None:
            self.pbuf = torch.zeros((L, N), **f64)   # the POD vectors followed by u_c
            self.sigma = torch.zeros(L, **f64)

    def free(self):
        """Drop every device buffer (after the carried ones were copied out)."""
        for name in list(vars(self)):
            if isinstance(getattr(self, name), self.torch.Tensor):
                setattr(self, name, None)

    @staticmethod
    def device_words(p, L: int, trials: int = 7) -> int:
        """FP64 words of the run's own buffers (the context's solver scratch not included)."""
        ne, N, R = p.nel, p.ndof, trials + 1
        return 2 * L * N + (ne + 1) * L * (L + 1) // 2 + R * ne + 2 * R + R * L + L + 9 * ne + 2 * N + 32

    def _start(self, psi0, tau, dmax_factor):
        torch, T = self.torch, self.T
        psi0 = torch.as_tensor(np.asarray(psi0, dtype=np.float64)).to(device="cuda")
        T.topo_tr_project(psi0, None, 0.0, False, self.vmax, self.psi_c, self.stats_crit)  # feasibility
        T.topo_filter(self.psi_c, self.rho)
        u0 = self.window[0:1]
        info = T.topo_solve_hdm(self.rho, self.F, u0, rtol=self.rtol, maxit=self.maxit, prec="fp64")
        self.hdm_iters += info["iters"]
        T.topo_compliance_grad(self.rho, u0, self.F, self.J, self.dc, self.g_c)
        T.topo_tr_init(self.st, self.f, tau, dmax_factor, self.J)
        self.nwin = 1

    def state(self) -> dict:
        return native.tr_state_read(self.st)

    def iterate(self) -> dict:
        """One major iteration; returns the state after it with the iteration's quantities."""
        T = self.T
        m = min(self.nwin, self.ring)
        if self.pod_nmax is None:
            k = T.topo_rom_build(self.rho, self.window[:m], self.Phi, None, self.b, self.f)
        else:
            cur = (self.nwin - 1) % self.ring
            n = max(0, min(m - 2, self.pod_nmax))
            T.topo_rom_pod(self.window[:m], n, self.pbuf[:n + 1], self.sigma, skip=cur, append=self.window[cur])
            k = T.topo_rom_build(self.rho, self.pbuf[:n + 1], self.Phi, None, self.b, self.f)
        T.topo_rom_elem(self.Phi[:k], k, self.Hel)
        T.topo_tr_project(self.psi_c, self.g_c, self.move, True, self.vmax, self.psi_x, self.stats_dir)
        T.topo_tr_trials(self.psi_c, self.psi_x, self.trials)
        yhat = self.yhat[:self.R * k]
        T.topo_rom_eval_batch(self.trials, self.Hel, self.Phi[:k], k, self.b[:k], self.f, self.Jk, self.resnorm,
                              yhat, None)
        T.topo_tr_select(self.st, self.prm, self.Jk, self.resnorm, self.stats_dir[0:1], self.trials, self.Phi[:k],
                         k, yhat, self.psi_hat, self.u_hat[0])
        T.topo_filter(self.psi_hat, self.rho)
        info = T.topo_solve_hdm(self.rho, self.F, self.u_hat, rtol=self.rtol, maxit=self.maxit, prec="fp64")
        T.topo_compliance_grad(self.rho, self.u_hat, self.F, self.J, self.dc, self.g_hat)
        # the centre's state is the newest window column; an accepted candidate's goes to the next slot
        slot = self.window[self.nwin % self.ring]
        T.topo_tr_update(self.st, self.prm, self.J, self.psi_c, self.psi_hat, slot, self.u_hat[0], self.g_c,
                         self.g_hat, None)
        T.topo_tr_project(self.psi_c, self.g_c, 1.0, False, self.vmax, self.scratch, self.stats_crit)
        T.topo_check()
        host = self.out.cpu().numpy()
        s = native.topo_tr_state.from_buffer_copy(host[:native.TR_STATE_BYTES // 8].tobytes())
        out = {n: getattr(s, n) for n, _ in native.topo_tr_state._fields_ if not n.startswith("pad")}
        if out["accepted"]:
            self.nwin += 1
        self.hdm_iters += info["iters"]
        out.update(k=k, mu=float(host[18]), chi=float(host[21]), hdm_iters=info["iters"],
                   hdm_status=info["status"])
        return out
