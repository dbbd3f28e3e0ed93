"""Serving form: continuous batching of design-evaluation requests on one GPU.

A request is one trust-region design evaluation in the shape of one major iteration of the
paper's Algorithm 2, for one problem (2D Q4 MBB or 3D H8 cantilever) and one seeded design:

  1. filter the centre design and solve the full-order model there (the new snapshot);
  2. build the reduced basis from the snapshot window (here the centre state) and the
     element reduced matrices of the basis;
  3. evaluate the candidate design with the reduced model: reduced solve, residual estimate
     theta = ||f - K(rho) Phi y|| (the error-aware trust-region constraint, Eq. trcon-topopt);
  4. if theta > Delta = tau ||f|| (tau = 0.1: the scaling of the initial radius, Eq. trrad0,
     since r(0, rho) = -f), fall back to a full-order solve at the candidate;
  5. compliance and filtered gradient at the candidate (from u_k, or from the HDM state).

The server keeps `slots` workers. Each owns a CUDA stream; a request admitted to a slot keeps
its densities, basis, element reduced matrices and CG state resident in device memory until it
completes. Requests are admitted in arrival order as soon as a slot is free AND the request's
estimated device memory fits the free budget (admission by free HBM), so requests that arrive
while others run start as capacity frees up and their kernels overlap on the GPU. Every
persistent solve of a request uses a fixed share of the GPU (total CTAs / slots), which also
fixes its reduction order: a request's results are bitwise the same alone and in a mix.

All arithmetic runs in libtopo's kernels; this module only schedules and marshals.
"""
from __future__ import annotations

import dataclasses
import math
import threading
import time

import numpy as np

from . import workloads as w


@dataclasses.dataclass
class Request:
    rid: int
    dim: int
    shape: tuple
    seed: int
    arrival: float = 0.0  # seconds after the stream starts


@dataclasses.dataclass
class Result:
    rid: int
    J: float
    theta: float
    delta: float
    used_hdm: bool
    Jk: float
    grad_norm: float
    hdm_iters: int
    t_arrival: float
    t_start: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def estimate_bytes(dim: int, shape, k: int = 1) -> int:
    """Device memory a request keeps resident (FP64): the assembled stencil of the solve
    (3^d d^2 words per node), PCG vectors and scratch, densities, the basis, the element
    reduced matrices and a few vectors of the request itself."""
    if dim == 2:
        nx, ny = shape
        nodes, nel = (nx + 1) * (ny + 1), nx * ny
    else:
        nx, ny, nz = shape
        nodes, nel = (nx + 1) * (ny + 1) * (nz + 1), nx * ny * nz
    ndof = dim * nodes
    nc = (9 if dim == 2 else 27) * dim * dim
    words = nc * nodes + 8 * ndof + 6 * nel + k * ndof + (k * (k + 1) // 2) * (nel + 1) + 6 * ndof
    return 8 * words + (4 << 20)


class Server:
    """Continuous-batching server over libtopo contexts (one per admitted request)."""

    def __init__(self, slots: int = 4, budget_bytes: int | None = None, tau: float = 0.1, rtol: float = 1e-8,
                 maxit: int = 400000):
        import torch
        from . import build, native
        build.build()
        self.torch = torch
        self.native = native
        self.slots = slots
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(0.8 * free) if budget_bytes is None else int(budget_bytes)
        self.tau = tau
        self.rtol = rtol
        self.maxit = maxit
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        # every persistent solve of a request uses this many CTAs (the SMs split over the slots;
        # one solve CTA fills an SM)
        self.ctas = max(1, props.multi_processor_count // slots)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.lock = threading.Condition()
        self.in_use = 0
        self.free_slots = list(range(slots))
        self.max_concurrency = 0
        self.concurrency = 0

    # -- one request ------------------------------------------------------------------------
    def _evaluate(self, req: Request, stream) -> dict:
        torch, native = self.torch, self.native
        p = w.build_problem(req.dim, req.shape)
        f64 = dict(dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            T = native.Topo(p, stream=stream)
            T.topo_set_param(native.TOPO_PARAM_PCG_MAX_CTAS, self.ctas)
            psi_c = w.design_field(p, req.seed)
            psi_x = w.perturbed_designs(p, psi_c, 1, amplitude=0.05, first_seed=req.seed % 100000 + 1)[:, 0]
            rho = torch.empty(p.nel, **f64)
            T.topo_filter(torch.as_tensor(psi_c).to(**f64), rho)
            F = torch.as_tensor(p.F[:, :1].T.copy()).to(**f64)
            f = F[0]
            U = torch.zeros((1, p.ndof), **f64)
            info = T.topo_solve_hdm(rho, F, U, rtol=self.rtol, maxit=self.maxit, prec="fp64")
            iters = info["iters"]
            Phi = torch.zeros_like(U)
            H = torch.zeros(1, **f64)
            b = torch.zeros(1, **f64)
            k = T.topo_rom_build(rho, U, Phi, H, b, f)
            Hel = torch.zeros((p.nel + 1) * k * (k + 1) // 2, **f64)
            T.topo_rom_elem(Phi[:k], k, Hel)
            rho_x = torch.empty(p.nel, **f64)
            T.topo_filter(torch.as_tensor(psi_x).to(**f64), rho_x)
            Hw = torch.zeros(k * k, **f64)
            y = torch.zeros(k, **f64)
            Jk = torch.zeros(1, **f64)
            T.topo_rom_solve_elem(rho_x, Hel, k, b[:k], Hw, y, Jk)
            rn = torch.zeros(2, **f64)
            uk = torch.zeros(p.ndof, **f64)
            T.topo_rom_error(rho_x, Phi[:k], k, y, f, rn, uk)
            theta = rn[0].item()
            fnorm = float(np.linalg.norm(p.F[:, 0]))
            delta = self.tau * fnorm
            used_hdm = theta > delta
            Ux = uk.reshape(1, -1)
            if used_hdm:
                Ux = torch.zeros((1, p.ndof), **f64)
                info2 = T.topo_solve_hdm(rho_x, F, Ux, rtol=self.rtol, maxit=self.maxit, prec="fp64")
                iters += info2["iters"]
            J = torch.zeros(1, **f64)
            dc = torch.empty(p.nel, **f64)
            dpsi = torch.empty(p.nel, **f64)
            T.topo_compliance_grad(rho_x, Ux, F, J, dc, dpsi)
            T.topo_check()
            out = dict(J=J.item(), theta=theta, delta=delta, used_hdm=bool(used_hdm), Jk=Jk.item(),
                       grad_norm=float(torch.linalg.vector_norm(dpsi).item()), hdm_iters=iters)
            T.close()
        return out

    # -- the stream -----------------------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve the requests; arrival times are honoured when realtime is true (requests are
        then admitted no earlier than their arrival), otherwise all arrive at t = 0."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        results: list[Result | None] = [None] * len(reqs)
        errors = []
        t0 = time.perf_counter()
        threads = []

        def worker(idx: int, req: Request, slot: int, need: int, t_arr: float):
            t_start = time.perf_counter() - t0
            try:
                out = self._evaluate(req, self.streams[slot])
                results[idx] = Result(rid=req.rid, t_arrival=t_arr, t_start=t_start,
                                      t_done=time.perf_counter() - t0, **out)
            except Exception as e:  # surfaced after the stream
                errors.append((req.rid, e))
            finally:
                with self.lock:
                    self.in_use -= need
                    self.free_slots.append(slot)
                    self.concurrency -= 1
                    self.lock.notify_all()

        for idx, req in enumerate(reqs):
            t_arr = req.arrival if realtime else 0.0
            if realtime:
                wait = t0 + req.arrival - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            need = estimate_bytes(req.dim, req.shape)
            if need > self.budget:
                errors.append((req.rid, MemoryError(f"request needs {need} B > budget {self.budget} B")))
                continue
            with self.lock:
                while not self.free_slots or self.in_use + need > self.budget:
                    self.lock.wait()
                slot = self.free_slots.pop(0)
                self.in_use += need
                self.concurrency += 1
                self.max_concurrency = max(self.max_concurrency, self.concurrency)
            th = threading.Thread(target=worker, args=(idx, req, slot, need, t_arr), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        if errors:
            rid, e = errors[0]
            raise RuntimeError(f"request {rid} failed: {e}") from e
        return [r for r in results if r is not None]


def poisson_requests(count: int, rate_per_s: float, seed: int = 7, q4=((100, 50), (800, 400)),
                     h8=((32, 32, 32), (96, 48, 48))) -> list[Request]:
    """The seeded serving stream: Poisson arrivals, half 2D Q4, half 3D H8, sizes log-uniform
    between the given corners."""
    raw = w.serving_stream(count, rate_per_s=rate_per_s, seed=seed, q4_range=q4, h8_range=h8)
    return [Request(rid=i, dim=r["dim"], shape=tuple(r["shape"]), seed=r["seed"] % (2 ** 31), arrival=r["arrival"])
            for i, r in enumerate(raw)]


def summarize(results: list[Result], wall: float) -> dict:
    lat = sorted(r.latency for r in results)
    pick = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)] if lat else None
    return dict(requests=len(results), evals_per_s=len(results) / wall if wall > 0 else None,
                p50_ms=1e3 * pick(0.50), p99_ms=1e3 * pick(0.99),
                hdm_fallbacks=sum(r.used_hdm for r in results))
