"""Serving form: continuous batching of trust-region design evaluations on one GPU.

A request is one major iteration of the error-aware trust-region method (Algorithm 2) for one
problem (2D Q4 MBB or 3D H8 cantilever), run by TrustRegionRun on the device:

  1. model update: the reduced basis of the run's snapshot window and its element reduced
     matrices;
  2. step: the projected-gradient target psi_x = P_C(psi_c - move g / ||g||_inf) and the trial
     steps psi_c + s (psi_x - psi_c), s = 0, 1, 1/2, ..., 1/64, all evaluated by the reduced
     model in one batched call; the candidate is the longest trial inside the error-aware trust
     region (theta <= Delta, Eq. trcon-topopt) with an Armijo decrease of the model;
  3. the full-order solve at the candidate (started from its reduced state), its compliance
     and gradient;
  4. varrho_k, acceptance and the radius update (gamma1 = 0.5, gamma2 = 1, eta1 = 0.1,
     eta2 = 0.75, Delta_max = 100 Delta_0, Section 5), and the criticality measure.

Requests either stand alone (a fresh run from a seeded design: the feasibility projection, the
full-order solve at the start, Delta_0 = tau ||f||, then one major iteration) or belong to a
session, the consecutive major iterations of one optimisation run. A session keeps its context
and its run's state (centre design and gradient, the window of the last kmax centre states,
the radius and compliances) resident in device memory between its requests.

The server keeps `slots` request slots. Requests start in arrival order as soon as a slot is
free and, for a standalone request or the first request of a session, its estimated device
memory fits the free budget (admission by free HBM). Requests of one session run in order;
requests of different sessions and standalone requests overlap on the GPU. A session's memory
is released after its last request. When a request does not fit, the least recently used idle
session (resident, between two of its requests) is evicted: the tensors that carry its run are
copied to pinned host memory and its device memory is freed. Its next request admits the
memory again and copies the state back, so an evicted session's results are the same as if it
had stayed resident. Every persistent solve uses a fixed share of the GPU (its SMs divided by
the slots), which also fixes its reduction order: a request's results are bitwise the same
alone and in a mix.

All arithmetic and every decision of the method run in libtopo's kernels; this module only
schedules and marshals.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import threading
import time

import numpy as np

from . import workloads as w
from .trust_region import TrustRegionRun


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
    J: float          # J at the centre after the iteration (J(psi_hat) when accepted)
    J_hat: float      # J(psi_hat), the full-order compliance at the candidate
    Jk: float         # m_k(psi_hat)
    Jk_c: float       # m_k(psi_c)
    theta: float      # theta_k(psi_hat), the trust-region constraint at the candidate
    delta: float      # Delta_k, the radius the iteration used
    delta_next: float # Delta_{k+1}
    ratio: float      # varrho_k
    accepted: bool
    inside: bool      # the candidate passed both tests of the step search
    step: float       # s of the candidate
    k: int            # reduced basis size
    chi: float        # criticality measure of the centre after the iteration
    hdm_iters: int    # iterations of the request's full-order solves
    rom_evals: int    # reduced evaluations of the request (the trials, centre included)
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


def estimate_bytes(dim: int, shape, k: int = 1, trials: int = 7) -> int:
    """Device memory a request (or a session with a window of k snapshots) keeps resident
    (FP64): the assembled stencil of the solve (3^d d^2 words per node) with the multigrid
    hierarchy's copies, PCG vectors and scratch, and the run's own buffers (window, basis,
    element reduced matrices, trials and vectors)."""
    nodes, nel = _sizes(dim, shape)
    ndof = dim * nodes
    nc = (9 if dim == 2 else 27) * dim * dim
    ne, N, R, L = nel, ndof, trials + 1, k
    run = 2 * L * N + (ne + 1) * L * (L + 1) // 2 + R * ne + 2 * R + R * L + L + 9 * ne + 2 * N + 32
    words = 2 * nc * nodes + 10 * ndof + 6 * nel + run
    return 8 * words + (8 << 20)


class _Session:
    """Resident state of one optimisation run (device tensors on the session's own stream)."""

    def __init__(self, srv: "Server", req: Request, held: int):
        torch = srv.torch
        self.srv = srv
        self.p = w.build_problem(req.dim, req.shape)
        self.stream = torch.cuda.Stream()
        self.seed = req.seed
        # the run's buffers come from the server's one allocation stream: blocks a spilled session
        # frees go back to that stream's pool, where the next session's allocations reuse them
        # without emptying the allocator's cache (which would synchronise the device)
        with torch.cuda.stream(self.stream):
            self._open_context()
            self.run = srv.new_run(self.T, self.p, w.design_field(self.p, req.seed), srv.kmax,
                                   alloc_stream=srv.alloc_stream)
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
        """Copy the run's carried tensors to pinned host memory, then free the context and every
        device buffer of the run."""
        torch = self.srv.torch
        with torch.cuda.stream(self.stream):
            host = {}
            for name in self.run.CARRIED:
                t = getattr(self.run, name)
                host[name] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                host[name].copy_(t, non_blocking=True)
        self.stream.synchronize()
        self.T.close()
        self.T = None
        self.run.free()
        self._host = host
        self.resident = False

    def restore(self):
        """Recreate the context and the run's buffers and copy the carried state back (bitwise
        the same)."""
        torch = self.srv.torch
        with torch.cuda.stream(self.stream):
            self._open_context()
            self.run.T = self.T
            self.run.alloc()
            for name in self.run.CARRIED:
                getattr(self.run, name).copy_(self._host[name], non_blocking=True)
        self.stream.synchronize()
        self._host = None
        self.resident = True

    def iterate(self) -> dict:
        with self.srv.torch.cuda.stream(self.stream):
            return self.run.iterate()

    def close(self):
        self.stream.synchronize()
        if self.T is not None:
            self.T.close()
            self.T = None
        if self.run is not None:
            self.run.free()


class Server:
    """Continuous-batching server over libtopo contexts."""

    def __init__(self, slots: int = 4, budget_bytes: int | None = None, tau: float = 0.1, rtol: float = 1e-8,
                 maxit: int = 400000, kmax: int = 8, trials: int = 7, move: float = 0.2, volfrac: float = 0.5):
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
        self.trials = trials
        self.move = move
        self.volfrac = volfrac
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        # every persistent solve of a request uses this many CTAs (the SMs split over the slots;
        # one solve CTA fills an SM)
        self.ctas = max(1, props.multi_processor_count // slots)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.alloc_stream = torch.cuda.Stream()  # orders a session's first allocations
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

    def new_run(self, T, p, psi0, L: int, alloc_stream=None) -> TrustRegionRun:
        return TrustRegionRun(T, p, psi0, tau=self.tau, move=self.move, trials=self.trials, volfrac=self.volfrac,
                              L=L, rtol=self.rtol, maxit=self.maxit, alloc_stream=alloc_stream)

    @staticmethod
    def _result(out: dict, hdm_iters: int, rom_evals: int) -> dict:
        return dict(J=out["J_c"], J_hat=out["J_hat"], Jk=out["Jk_hat"], Jk_c=out["Jk_c"], theta=out["theta_hat"],
                    delta=out["delta_prev"], delta_next=out["delta"], ratio=out["ratio"],
                    accepted=bool(out["accepted"]), inside=bool(out["inside"]), step=out["step"], k=out["k"],
                    chi=out["chi"], hdm_iters=hdm_iters, rom_evals=rom_evals)

    def _standalone(self, req: Request, stream) -> dict:
        torch, native = self.torch, self.native
        p = w.build_problem(req.dim, req.shape)
        with torch.cuda.stream(stream):
            T = native.Topo(p, stream=stream)
            try:
                T.topo_set_param(native.TOPO_PARAM_PCG_MAX_CTAS, self.ctas)
                run = self.new_run(T, p, w.design_field(p, req.seed), 1)
                out = run.iterate()
                res = self._result(out, run.hdm_iters, run.R)
                run.free()
            finally:
                T.close()
        return res

    def _in_session(self, S: _Session, req: Request) -> dict:
        before = S.run.hdm_iters if req.step > 0 else 0
        out = S.iterate()
        return self._result(out, S.run.hdm_iters - before, S.run.R)

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
        standalone = [r for r in reqs if r.session is None]
        for req in reqs:
            if req.session is not None:
                sessions.setdefault(req.session, []).append(req)
        for sid, sreqs in sessions.items():
            sreqs.sort(key=lambda r: r.step)
            threads.append(threading.Thread(target=session_worker, args=(sid, sreqs), daemon=True))

        def dispatch():
            # a standalone request's thread starts at its arrival, so a long stream holds threads
            # only for the requests that have arrived and not finished
            for req in standalone:
                wait_arrival(req)
                th = threading.Thread(target=standalone_worker, args=(req,), daemon=True)
                th.start()
                threads.append(th)

        for th in list(threads):
            th.start()
        dispatcher = threading.Thread(target=dispatch, daemon=True)
        dispatcher.start()
        dispatcher.join()
        for th in list(threads):
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
    ratios = [r.ratio for r in results if math.isfinite(r.ratio)]
    return dict(requests=len(results), evals_per_s=len(results) / wall if wall > 0 else None,
                p50_ms=1e3 * pick(0.50), p99_ms=1e3 * pick(0.99),
                accepted=sum(r.accepted for r in results), inside=sum(r.inside for r in results),
                median_ratio=float(np.median(ratios)) if ratios else None,
                rom_evals=sum(r.rom_evals for r in results),
                mean_basis_size=(sum(r.k for r in results) / len(results)) if results else None)
