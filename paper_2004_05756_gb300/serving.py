"""Serving form: continuous batching of design-evaluation requests on one GPU.

A request is one trust-region design evaluation in the shape of one major iteration of the
paper's Algorithm 2, for one problem (2D Q4 MBB or 3D H8 cantilever):

  1. filter the centre design and solve the full-order model there (the new snapshot);
  2. build the reduced basis from the snapshot window and the element reduced matrices of the
     basis;
  3. evaluate the proposed candidate with the reduced model: reduced solve, residual estimate
     theta = ||f - K(rho) Phi y|| (the error-aware trust-region constraint, Eq. trcon-topopt);
  4. the trust-region constraint theta <= Delta = tau ||f|| (tau = 0.1: the scaling of the
     initial radius, Eq. trrad0, since r(0, rho) = -f) decides the candidate the way the
     subproblem's constraint does: the largest step from the centre toward the proposal,
     s = 1, 1/2, ..., 2^-tr_halvings, whose reduced evaluation satisfies it is taken; if none
     does, the proposal (s = 1) is evaluated with a full-order solve started from its reduced
     state u_k;
  5. compliance and filtered gradient at the candidate (from u_k, or from the HDM state).

Requests either stand alone (their window is the one centre snapshot) or belong to a session:
the consecutive evaluations of one optimisation run. A session keeps its context, snapshot
window (the last kmax centre states), basis, element reduced matrices and last centre state
resident in device memory between its requests, so its basis grows with the run and its centre
solves start from the previous centre's state (a warm start of the iterative solve; the
converged result is the same fixed point). The designs of a session follow a seeded random
walk: the centre of step t is the previous centre plus a smoothed perturbation of amplitude
0.02, the candidate the centre plus one of amplitude 0.05.

The server keeps `slots` request slots. Requests start in arrival order as soon as a slot is
free and, for a standalone request or the first request of a session, its estimated device
memory fits the free budget (admission by free HBM). Requests of one session run in order;
requests of different sessions and standalone requests overlap on the GPU. A session's memory
is released after its last request. When a request does not fit, the least recently used idle
session (resident, between two of its requests) is evicted: its window, basis, element
reduced matrices and last centre state are copied to pinned host memory and its device memory
is freed. Its next request admits the memory again and copies the state back, so an evicted
session's results are the same as if it had stayed resident. Every persistent solve uses a fixed share of the GPU (its
SMs divided by the slots), which also fixes its reduction order: a request's results are
bitwise the same alone and in a mix.

All arithmetic runs in libtopo's kernels; this module only schedules and marshals.
"""
from __future__ import annotations

import dataclasses
import heapq
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
    session: int | None = None  # optimisation run this request belongs to (None: standalone)
    step: int = 0  # index of the request within its session
    last: bool = True  # the session's last request (its state is released afterwards)


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
    k: int
    step: float  # trust-region step taken toward the proposed candidate (1 on fallback)
    rom_evals: int
    t_arrival: float
    t_start: float
    t_done: float
    session: int | None = None
    index: int = 0  # position of the request within its session

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def _sizes(dim: int, shape):
    if dim == 2:
        nx, ny = shape
        return (nx + 1) * (ny + 1), nx * ny
    nx, ny, nz = shape
    return (nx + 1) * (ny + 1) * (nz + 1), nx * ny * nz


def estimate_bytes(dim: int, shape, k: int = 1) -> int:
    """Device memory a request (or a session with a window of k snapshots) keeps resident
    (FP64): the assembled stencil of the solve (3^d d^2 words per node), PCG vectors and
    scratch, densities, the window and the basis, the element reduced matrices and a few
    vectors of the request itself."""
    nodes, nel = _sizes(dim, shape)
    ndof = dim * nodes
    nc = (9 if dim == 2 else 27) * dim * dim
    words = nc * nodes + 8 * ndof + 6 * nel + 2 * k * ndof + (k * (k + 1) // 2) * (nel + 1) + 6 * ndof
    return 8 * words + (4 << 20)


class _Session:
    """Resident state of one optimisation run (device tensors on the session's own stream)."""

    STATE = ("window", "Phi", "Hel", "u_prev")  # device tensors that carry the run

    def __init__(self, srv: "Server", req: Request, held: int):
        torch = srv.torch
        self.srv = srv
        self.p = w.build_problem(req.dim, req.shape)
        self.stream = torch.cuda.Stream()
        self.kmax = srv.kmax
        p = self.p
        f64 = dict(dtype=torch.float64, device="cuda")
        # The tensors come from the server's one allocation stream: blocks a spilled session
        # frees go back to that stream's pool, where the next session's allocations reuse them
        # without emptying the allocator's cache (which would synchronise the device).
        with torch.cuda.stream(srv.alloc_stream):
            self.window = torch.zeros((self.kmax, p.ndof), **f64)
            self.Phi = torch.zeros((self.kmax, p.ndof), **f64)
            self.Hel = torch.zeros((p.nel + 1) * self.kmax * (self.kmax + 1) // 2, **f64)
            self.u_prev = torch.zeros((1, p.ndof), **f64)
        self.stream.wait_stream(srv.alloc_stream)
        with torch.cuda.stream(self.stream):
            self._open_context()
        self.nwin = 0
        self.seed = req.seed
        self.psi = w.design_field(p, req.seed)  # centre of step 0
        # admission state, guarded by the server's lock
        self.held = held          # device bytes admitted for the session
        self.counted = True       # held is part of the server's in-use total
        self.resident = True      # state on the device (False: spilled to host)
        self.busy = True          # a request of the session holds a slot
        self.evicting = False
        self.last_use = time.perf_counter()
        self._host = None

    def _open_context(self):
        native = self.srv.native
        self.T = native.Topo(self.p, stream=self.stream)
        self.T.topo_set_param(native.TOPO_PARAM_PCG_MAX_CTAS, self.srv.ctas)

    def evict(self):
        """Copy the state to pinned host memory, then free the context and device tensors."""
        torch = self.srv.torch
        with torch.cuda.stream(self.stream):
            host = {}
            for name in self.STATE:
                t = getattr(self, name)
                host[name] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                host[name].copy_(t, non_blocking=True)
        self.stream.synchronize()
        self.T.close()
        self.T = None
        for name in self.STATE:
            setattr(self, name, None)
        self._host = host
        self.resident = False

    def restore(self):
        """Recreate the context and copy the spilled state back (bitwise the same)."""
        torch = self.srv.torch
        with torch.cuda.stream(self.srv.alloc_stream):
            for name in self.STATE:
                h = self._host[name]
                setattr(self, name, torch.empty(h.shape, dtype=h.dtype, device="cuda"))
        self.stream.wait_stream(self.srv.alloc_stream)
        with torch.cuda.stream(self.stream):
            self._open_context()
            for name in self.STATE:
                getattr(self, name).copy_(self._host[name], non_blocking=True)
        self.stream.synchronize()
        self._host = None
        self.resident = True

    def designs(self, step: int):
        """Centre and candidate of the given step (the steps of a session arrive in order)."""
        if step > 0:
            self.psi = w.perturbed_designs(self.p, self.psi, 1, amplitude=0.02,
                                           first_seed=w.seed_for(f"walk{self.seed}", 2 * step))[:, 0]
        psi_x = w.perturbed_designs(self.p, self.psi, 1, amplitude=0.05,
                                    first_seed=w.seed_for(f"walk{self.seed}", 2 * step + 1))[:, 0]
        return self.psi, psi_x

    def close(self):
        self.stream.synchronize()
        if self.T is not None:
            self.T.close()
            self.T = None


class Server:
    """Continuous-batching server over libtopo contexts."""

    def __init__(self, slots: int = 4, budget_bytes: int | None = None, tau: float = 0.1, rtol: float = 1e-8,
                 maxit: int = 400000, kmax: int = 8, tr_halvings: int = 6):
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
        self.kmax = kmax
        self.tr_halvings = tr_halvings
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        # every persistent solve of a request uses this many CTAs (the SMs split over the slots;
        # one solve CTA fills an SM)
        self.ctas = max(1, props.multi_processor_count // slots)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.alloc_stream = torch.cuda.Stream()  # allocation stream of every session's tensors
        self.evict_ms: list[float] = []    # wall time of each spill (copy out, context teardown)
        self.restore_ms: list[float] = []  # wall time of each restore
        self.lock = threading.Condition()
        self.in_use = 0
        self.free_slots = list(range(slots))
        self.max_concurrency = 0
        self.concurrency = 0
        self.sessions: dict[int, _Session] = {}  # live sessions, resident or spilled
        self.waiting: list[tuple] = []  # (arrival, request id) of the requests waiting to start
        self.evictions = 0
        self.restores = 0

    # -- one evaluation -----------------------------------------------------------------------
    def _evaluate(self, T, p, psi_c, psi_x, window, nwin, Phi, Hel, U0, stream) -> dict:
        """Steps 1-5 on context T. The new centre state goes to slot (nwin - 1) % kmax of the
        window (kmax x N); U0 is the centre solve's initial guess and receives its solution."""
        torch = self.torch
        f64 = dict(dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            rho = torch.empty(p.nel, **f64)
            T.topo_filter(torch.as_tensor(psi_c).to(**f64), rho)
            F = torch.as_tensor(p.F[:, :1].T.copy()).to(**f64)
            f = F[0]
            info = T.topo_solve_hdm(rho, F, U0, rtol=self.rtol, maxit=self.maxit, prec="fp64")
            iters = info["iters"]
            kmax = window.shape[0]
            window[(nwin - 1) % kmax].copy_(U0[0])
            m = min(nwin, kmax)
            H = torch.zeros(m * m, **f64)
            b = torch.zeros(m, **f64)
            k = T.topo_rom_build(rho, window[:m], Phi, H, b, f)
            T.topo_rom_elem(Phi[:k], k, Hel)
            fnorm = float(np.linalg.norm(p.F[:, 0]))
            delta = self.tau * fnorm
            Hw = torch.zeros(k * k, **f64)

            def rom_at(psi):
                rho_s = torch.empty(p.nel, **f64)
                T.topo_filter(torch.as_tensor(psi).to(**f64), rho_s)
                y = torch.zeros(k, **f64)
                Jk = torch.zeros(1, **f64)
                T.topo_rom_solve_elem(rho_s, Hel, k, b[:k], Hw, y, Jk)
                rn = torch.zeros(2, **f64)
                uk = torch.zeros(p.ndof, **f64)
                T.topo_rom_error(rho_s, Phi[:k], k, y, f, rn, uk)
                return rho_s, uk, Jk.item(), rn[0].item()

            # the largest step toward the proposal that the trust-region constraint admits
            first = None
            s, nrom, acc = 1.0, 0, None
            for h in range(self.tr_halvings + 1):
                ev = rom_at(psi_x if h == 0 else psi_c + s * (psi_x - psi_c))
                nrom += 1
                if first is None:
                    first = ev
                if ev[3] <= delta:
                    acc = ev
                    break
                s *= 0.5
            used_hdm = acc is None
            if used_hdm:  # full-order solve at the proposal, from its reduced state
                rho_x, uk, Jk, theta = first
                s = 1.0
                Ux = uk.reshape(1, -1).clone()
                info2 = T.topo_solve_hdm(rho_x, F, Ux, rtol=self.rtol, maxit=self.maxit, prec="fp64")
                iters += info2["iters"]
            else:
                rho_x, uk, Jk, theta = acc
                Ux = uk.reshape(1, -1)
            J = torch.zeros(1, **f64)
            dc = torch.empty(p.nel, **f64)
            dpsi = torch.empty(p.nel, **f64)
            T.topo_compliance_grad(rho_x, Ux, F, J, dc, dpsi)
            T.topo_check()
            return dict(J=J.item(), theta=theta, delta=delta, used_hdm=bool(used_hdm), Jk=Jk,
                        grad_norm=float(torch.linalg.vector_norm(dpsi).item()), hdm_iters=iters, k=k, step=s,
                        rom_evals=nrom)

    def _standalone(self, req: Request, stream) -> dict:
        torch, native = self.torch, self.native
        p = w.build_problem(req.dim, req.shape)
        f64 = dict(dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            T = native.Topo(p, stream=stream)
            T.topo_set_param(native.TOPO_PARAM_PCG_MAX_CTAS, self.ctas)
            psi_c = w.design_field(p, req.seed)
            psi_x = w.perturbed_designs(p, psi_c, 1, amplitude=0.05, first_seed=req.seed % 100000 + 1)[:, 0]
            window = torch.zeros((1, p.ndof), **f64)
            Phi = torch.zeros((1, p.ndof), **f64)
            Hel = torch.zeros(p.nel + 1, **f64)
            U0 = torch.zeros((1, p.ndof), **f64)
            out = self._evaluate(T, p, psi_c, psi_x, window, 1, Phi, Hel, U0, stream)
            T.close()
        return out

    def _in_session(self, S: _Session, req: Request) -> dict:
        psi_c, psi_x = S.designs(req.step)
        S.nwin += 1
        return self._evaluate(S.T, S.p, psi_c, psi_x, S.window, S.nwin, S.Phi, S.Hel, S.u_prev, S.stream)

    # -- the stream -----------------------------------------------------------------------------
    def _evict_one(self, keep) -> bool:
        """With the lock held: spill the least recently used idle session other than `keep`.
        The copy runs with the lock released; returns False when no session is idle."""
        idle = [S for S in self.sessions.values() if S.resident and not S.busy and not S.evicting and S is not keep]
        if not idle:
            return False
        V = min(idle, key=lambda S: S.last_use)
        V.evicting = True
        self.lock.release()
        t0 = time.perf_counter()
        try:
            V.evict()
            self.evict_ms.append(1e3 * (time.perf_counter() - t0))
        finally:
            self.lock.acquire()
            V.evicting = False
            V.counted = False
            self.in_use -= V.held
            self.evictions += 1
            self.lock.notify_all()
        return True

    def _acquire(self, req: Request, need: int, owner: _Session | None = None) -> tuple[int, int]:
        """Take a slot and admit `need` bytes, or for a live session its own bytes if it was
        spilled. Requests start in arrival order: only the earliest waiting request may start,
        and it evicts idle sessions while the budget is short. Returns (slot, admitted)."""
        key = (req.arrival, req.rid)
        with self.lock:
            heapq.heappush(self.waiting, key)
            while True:
                if self.waiting[0] != key:
                    self.lock.wait()
                    continue
                if owner is not None:
                    if owner.evicting:
                        self.lock.wait()
                        continue
                    need = 0 if owner.counted else owner.held
                if self.free_slots and self.in_use + need <= self.budget:
                    break
                if self.free_slots and self._evict_one(owner):
                    continue
                self.lock.wait()
            heapq.heappop(self.waiting)
            self.lock.notify_all()  # the next request in line may start too
            slot = self.free_slots.pop(0)
            self.in_use += need
            if owner is not None:
                owner.busy = True
                owner.counted = True
            self.concurrency += 1
            self.max_concurrency = max(self.max_concurrency, self.concurrency)
            return slot, need

    def _release(self, slot: int, freed: int):
        with self.lock:
            self.in_use -= freed
            self.free_slots.append(slot)
            self.concurrency -= 1
            self.lock.notify_all()

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve the requests; arrival times are honoured when realtime is true (requests then
        start no earlier than their arrival), otherwise all arrive at t = 0."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        results: dict[int, Result] = {}
        errors = []
        t0 = time.perf_counter()

        def wait_arrival(req):
            if realtime:
                dt = t0 + req.arrival - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            return req.arrival if realtime else 0.0

        def standalone_worker(req: Request):
            t_arr = wait_arrival(req)
            need = estimate_bytes(req.dim, req.shape)
            if need > self.budget:
                errors.append((req.rid, MemoryError(f"request needs {need} B > budget {self.budget} B")))
                return
            slot, _ = self._acquire(req, need)
            t_start = time.perf_counter() - t0
            try:
                out = self._standalone(req, self.streams[slot])
                results[req.rid] = Result(rid=req.rid, t_arrival=t_arr, t_start=t_start,
                                          t_done=time.perf_counter() - t0, **out)
            except Exception as e:  # surfaced after the stream
                errors.append((req.rid, e))
            finally:
                self._release(slot, need)

        def session_worker(sid: int, sreqs: list[Request]):
            S = None
            try:
                for n, req in enumerate(sreqs):
                    t_arr = wait_arrival(req)
                    if S is None:  # the session's memory is admitted with its first request
                        need = estimate_bytes(req.dim, req.shape, self.kmax)
                        if need > self.budget:
                            raise MemoryError(f"session {sid} needs {need} B > budget {self.budget} B")
                        slot, _ = self._acquire(req, need)
                    else:  # re-admits the session's memory if it was evicted meanwhile
                        slot, _ = self._acquire(req, 0, owner=S)
                    last = n == len(sreqs) - 1
                    t_start = time.perf_counter() - t0
                    try:
                        if S is None:
                            try:
                                S = _Session(self, req, need)
                            except BaseException:
                                with self.lock:
                                    self.in_use -= need
                                raise
                            with self.lock:
                                self.sessions[sid] = S
                        elif not S.resident:
                            t_r = time.perf_counter()
                            S.restore()
                            with self.lock:
                                self.restores += 1
                                self.restore_ms.append(1e3 * (time.perf_counter() - t_r))
                        out = self._in_session(S, req)
                        results[req.rid] = Result(rid=req.rid, t_arrival=t_arr, t_start=t_start,
                                                  t_done=time.perf_counter() - t0, session=sid, index=req.step,
                                                  **out)
                    finally:
                        freed = 0
                        if S is not None:
                            with self.lock:
                                S.busy = False
                                S.last_use = time.perf_counter()
                            if last:
                                S.close()
                                with self.lock:
                                    self.sessions.pop(sid, None)
                                freed = S.held
                                S = None
                        self._release(slot, freed)
            except Exception as e:  # surfaced after the stream
                errors.append((sid, e))
                if S is not None:
                    with self.lock:
                        self.sessions.pop(sid, None)
                        if S.counted:
                            self.in_use -= S.held
                        self.lock.notify_all()
                    S.close()

        threads = []
        sessions: dict[int, list[Request]] = {}
        for req in reqs:
            if req.session is None:
                threads.append(threading.Thread(target=standalone_worker, args=(req,), daemon=True))
            else:
                sessions.setdefault(req.session, []).append(req)
        for sid, sreqs in sessions.items():
            sreqs.sort(key=lambda r: r.step)
            threads.append(threading.Thread(target=session_worker, args=(sid, sreqs), daemon=True))
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errors:
            rid, e = errors[0]
            raise RuntimeError(f"request or session {rid} failed: {e}") from e
        return [results[r.rid] for r in reqs if r.rid in results]


def poisson_requests(count: int, rate_per_s: float, seed: int = 7, q4=((100, 50), (800, 400)),
                     h8=((32, 32, 32), (96, 48, 48))) -> list[Request]:
    """The seeded standalone stream: Poisson arrivals, half 2D Q4, half 3D H8, sizes
    log-uniform between the given corners."""
    raw = w.serving_stream(count, rate_per_s=rate_per_s, seed=seed, q4_range=q4, h8_range=h8)
    return [Request(rid=i, dim=r["dim"], shape=tuple(r["shape"]), seed=r["seed"] % (2 ** 31), arrival=r["arrival"])
            for i, r in enumerate(raw)]


def session_requests(count: int, rate_per_s: float, sessions: int = 8, seed: int = 7, q4=((100, 50), (800, 400)),
                     h8=((32, 32, 32), (96, 48, 48))) -> list[Request]:
    """The seeded session stream: Poisson arrivals of the next evaluation of one of `sessions`
    optimisation runs (half 2D Q4, half 3D H8)."""
    raw = w.session_stream(count, rate_per_s=rate_per_s, sessions=sessions, seed=seed, q4_range=q4, h8_range=h8)
    return [Request(rid=i, dim=r["dim"], shape=tuple(r["shape"]), seed=r["seed"] % (2 ** 31), arrival=r["arrival"],
                    session=r["session"], step=r["step"], last=r["last"]) for i, r in enumerate(raw)]


def summarize(results: list[Result], wall: float) -> dict:
    lat = sorted(r.latency for r in results)
    pick = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)] if lat else None
    return dict(requests=len(results), evals_per_s=len(results) / wall if wall > 0 else None,
                p50_ms=1e3 * pick(0.50), p99_ms=1e3 * pick(0.99),
                hdm_fallbacks=sum(r.used_hdm for r in results),
                rom_evals=sum(r.rom_evals for r in results),
                mean_basis_size=(sum(r.k for r in results) / len(results)) if results else None)
