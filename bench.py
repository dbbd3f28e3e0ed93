#!/usr/bin/env python
"""Benchmark: ROM-accelerated design evaluations of the minimum-compliance SIMP method on
one GB300, through the libtopo C ABI.

One step = one pass of the whole hot path in the shape of one trust-region major iteration
(Algorithm 2 of the paper): an HDM design evaluation at the trust-region centre
(filter -> mixed-precision PCG solve -> compliance and filtered gradient), a basis update
from the snapshot window plus the new centre state (rom_build), then R ROM design
evaluations at candidate designs (filter -> reduced solve -> residual estimate ->
compliance and filtered gradient with u_k). The metric is design evaluations per second
(1 + R per step). The plain FP64 HDM evaluation rate is measured beside it.

Workload (default): MBB half-beam, 600 x 200 Q4 elements (241,602 DOFs), E0 = 1,
Emin = 1e-9, nu = 0.3, p = 3, linear filter radius 1.5, seeded smoothed-random designs
(synthetic stand-ins for the paper's MBB benchmark).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one launch of the HDM solve kernel (pcg2_mg_kernel) at MBB 600x200,
# rtol 1e-8, from an ncu capture (dram__bytes_read.sum, dram__bytes_write.sum) of
# `python -m paper_2004_05756_gb300.profcase --call hdm --rtol 1e-8 --reps 1` (a solve from zero,
# 58 iterations; the step's solves start from the ROM prediction and run about 53). It is reported
# only while the kernel sources hash to the value they had when it was taken.
PCG_TRAFFIC = {"bytes": 280.492544e6 + 363.760384e6, "sources_sha256_16": "b61b7bcc2a3eedcf"}


def pcg_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in ("pcg2.cu", "pcg2.cuh", "common.cuh", "mg.cuh"):
        with open(os.path.join(ROOT, "paper_2004_05756_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return PCG_TRAFFIC["bytes"] if h.hexdigest()[:16] == PCG_TRAFFIC["sources_sha256_16"] else None


METRIC = "design evals/s (ROM vs plain FP64 HDM) at 1e-6 rel compliance err; p50/p99 ms"
UNIT = "design evals/s"

CONFIGS = {
    "mbb600x200": dict(kind="q4", shape=(600, 200), rmin=1.5),
    "mbb60x20": dict(kind="q4", shape=(60, 20), rmin=1.5),
    "cant96x48x48": dict(kind="h8", shape=(96, 48, 48), rmin=2.0),
    "batch256": dict(kind="batch", count=256),
    "serving": dict(kind="serving"),
}


def make_problem(cfg):
    from paper_2004_05756_gb300 import workloads as w
    c = CONFIGS[cfg]
    if c["kind"] == "q4":
        return w.mbb_2d(*c["shape"], rmin=c["rmin"])
    return w.cantilever_3d(*c["shape"], rmin=c["rmin"])


def designs(p, args):
    """Seeded inputs: per-step centre designs (warm-up, timed, then distinct ones for the
    end-to-end pass), R candidate designs, k snapshot designs."""
    from paper_2004_05756_gb300 import workloads as w
    psi0 = w.design_field(p, 0)
    nsteps = 2 * args.steps + args.warmup
    centres = w.perturbed_designs(p, psi0, nsteps, amplitude=0.05, first_seed=500)
    cands = w.perturbed_designs(p, psi0, args.rom_evals, amplitude=0.02, first_seed=2000)
    snaps = w.perturbed_designs(p, psi0, args.k, amplitude=0.1, first_seed=1)
    return psi0, centres, cands, snaps


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the --impl reference arm)
# ------------------------------------------------------------------------------------------
def host_info():
    """The host the oracle runs on: core count, CPU model, library versions, BLAS threads."""
    import platform
    import scipy
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.strip().lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    blas_threads, src = None, None
    try:
        from threadpoolctl import threadpool_info
        blas_threads = max([d.get("num_threads", 1) for d in threadpool_info()] or [1])
        src = "threadpoolctl"
    except Exception:
        for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
            if os.environ.get(var):
                blas_threads, src = int(os.environ[var]), var
                break
        if blas_threads is None:
            blas_threads, src = os.cpu_count(), "OpenBLAS default (one thread per core)"
    return {"cpu_count": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine(), "numpy": np.__version__, "scipy": scipy.__version__,
            "blas_threads": blas_threads, "blas_threads_source": src,
            "superlu_threads": 1}


def cpu_oracle_step(p, psi_c, cand, k, rom_samples):
    """One bounded sample of the step on the FP64 oracle as it stands: an HDM evaluation at the
    centre psi_c (filter, sparse assembly, SuperLU solve, compliance, filtered gradient), a basis
    update at k columns (Householder QR of an N x k window, H = Phi^T K Phi, b = Phi^T f) and
    `rom_samples` ROM evaluations at the candidate (filter, H(rho), Cholesky, residual, gradient
    with u_k). Returns the measured times and the centre's compliance."""
    from oracle import fem, hatfilter, rom
    f = p.F[:, 0]
    t0 = time.perf_counter()
    rho = hatfilter.filter_fwd(p, psi_c)
    ts = time.perf_counter()
    U = fem.solve(p, rho)
    t_solve = time.perf_counter() - ts
    J = fem.compliance(p, U)
    dc = fem.compliance_grad_rho(p, rho, U)
    hatfilter.filter_adj(p, dc)
    t_hdm = time.perf_counter() - t0
    # basis update: the window's values do not change its cost; a seeded N x k window with the
    # centre state as its last column
    t1 = time.perf_counter()
    win = np.random.default_rng(12345).standard_normal((p.ndof, k))
    win[:, -1] = U[:, 0]
    win[fem.fixed_dofs(p)] = 0.0
    Phi = rom.basis(win)
    rom.project(p, rho, Phi, f)
    t_basis = time.perf_counter() - t1
    t2 = time.perf_counter()
    for _ in range(rom_samples):
        r2 = hatfilter.filter_fwd(p, cand)
        out = rom.rom_eval(p, r2, Phi, f)
        dc2 = fem.compliance_grad_rho(p, r2, out["uk"])
        hatfilter.filter_adj(p, dc2)
    t_rom = (time.perf_counter() - t2) / max(1, rom_samples)
    return dict(J=J, t_hdm=t_hdm, t_solve=t_solve, t_basis=t_basis, t_rom=t_rom, rho=rho, U=U, Phi=Phi,
                wall=time.perf_counter() - t0)


def cpu_oracle_timing(p, psi_c, cand, args, rom_samples=2):
    """Times the FP64 oracle on a bounded sample of the step (cpu_oracle_step) and derives its
    throughput on the step's mix of 1 HDM + R ROM evaluations from the measured per-part
    times. Also splits the HDM and ROM evaluations by the paper's steps (Sec. 2.5, Sec. 3.4)."""
    from oracle import fem, hatfilter, rom
    st = cpu_oracle_step(p, psi_c, cand, args.k, rom_samples)
    t_step = st["t_hdm"] + st["t_basis"] + args.rom_evals * st["t_rom"]

    def tm(fn):
        a = time.perf_counter()
        r = fn()
        return r, time.perf_counter() - a
    rho, U, Phi, f = st["rho"], st["U"], st["Phi"], p.F[:, 0]
    _, t_filter = tm(lambda: hatfilter.filter_fwd(p, psi_c))
    _, t_asm = tm(lambda: fem.reduced_K(p, rho))
    _, t_grad = tm(lambda: hatfilter.filter_adj(p, fem.compliance_grad_rho(p, rho, U)))
    (Hk, bk), t_hb = tm(lambda: rom.project(p, rho, Phi, f))
    yk, t_chol = tm(lambda: rom.solve_reduced(Hk, bk))
    _, t_res = tm(lambda: rom.residual(p, rho, rom.reconstruct(Phi, yk), f))
    split = {"filter": t_filter, "assembly": t_asm, "solve": max(0.0, st["t_solve"] - t_asm), "gradient": t_grad,
             "H_build": t_hb, "cholesky": t_chol, "residual": t_res}
    hi = host_info()
    return dict(J=st["J"], U=st["U"], t_hdm=st["t_hdm"], t_basis=st["t_basis"], t_rom=st["t_rom"],
                value=(1 + args.rom_evals) / t_step, split_s=split, host=hi,
                cores=max(1, hi["blas_threads"] or 1),
                sample=f"1 HDM eval (SuperLU, 1 thread) at the first timed centre + basis update (k={args.k}) + "
                       f"{rom_samples} ROM evals on {p.name}; measured part times combined for the step's mix of "
                       f"1 HDM + basis update + {args.rom_evals} ROM evals; wall {st['wall']:.1f} s")


def oracle_accuracy(p, probe_in, probe, J_oracle, U_oracle=None):
    """GPU results of the accuracy probe against the FP64 oracle on the same inputs: the HDM
    compliance at the first timed centre (the oracle's SuperLU solve of the CPU baseline leg),
    and the ROM's J_k and ||r|| at candidate 0 on a basis of the first k_acc snapshot designs,
    which the oracle solves itself (SuperLU, Householder QR, Cholesky)."""
    from oracle import fem, hatfilter, rom
    out = {"J_oracle": J_oracle,
           "hdm_J_vs_oracle_rel": abs(probe["J_rtol1e-8"] - J_oracle) / abs(J_oracle),
           "hdm_J_fp64_rtol1e-13_vs_oracle_rel": abs(probe["J_fp64_rtol1e-13"] - J_oracle) / abs(J_oracle)}
    if U_oracle is not None:
        # Both FP64 solutions stop at a rounding floor of their residual; to first order
        # |J_a - J_b| <= ||u|| (||r_a|| + ||r_b||) (J - J_h = u^T r for compliance).
        rho_c = hatfilter.filter_fwd(p, probe_in["centre"])
        u_o = U_oracle[:, 0]
        r_o = rom.residual(p, rho_c, u_o, p.F[:, 0])
        nf = float(np.linalg.norm(p.F[:, 0]))
        nu = float(np.linalg.norm(u_o))
        out["oracle_relres"] = float(np.linalg.norm(r_o)) / nf
        out["hdm_J_fp64_rtol1e-13_first_order_bound_rel"] = nu * nf * (
            probe["J_fp64_rtol1e-13_relres"] + out["oracle_relres"]) / abs(J_oracle)
        out["hdm_J_rtol1e-8_first_order_bound_rel"] = nu * nf * (
            probe["J_rtol1e-8_relres"] + out["oracle_relres"]) / abs(J_oracle)
    t0 = time.perf_counter()
    S = probe_in["snaps"]
    U = np.stack([fem.solve(p, hatfilter.filter_fwd(p, S[:, i]))[:, 0] for i in range(S.shape[1])], 1)
    Phi = rom.basis(U)
    ref = rom.rom_eval(p, hatfilter.filter_fwd(p, probe_in["cand"]), Phi, p.F[:, 0])
    out.update(rom_k=int(Phi.shape[1]), Jk_oracle=ref["Jk"], rom_Jk_vs_oracle_rel=abs(probe["Jk"] - ref["Jk"]) / abs(ref["Jk"]),
               rom_resnorm_vs_oracle_rel=abs(probe["rom_resnorm"] - ref["resnorm"]) / abs(ref["resnorm"]),
               oracle_probe_s=time.perf_counter() - t0)
    return out


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_2004_05756_gb300 import build, native

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    p = make_problem(args.config)
    psi0, centres, cands, snaps = designs(p, args)
    N, Ne, k, R = p.ndof, p.nel, args.k, args.rom_evals
    prec = args.prec
    f64 = dict(dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        T = native.Topo(p, stream=stream)
        d_cent = torch.as_tensor(centres.T.copy()).to(**f64)         # (S, Ne)
        d_cand = torch.as_tensor(cands.T.copy()).to(**f64)           # (R, Ne)
        F = torch.as_tensor(p.F.T.copy()).to(**f64)                  # (1, N)
        f = F[0]
        rho = torch.empty(Ne, **f64)
        Uc = torch.zeros((1, N), **f64)
        J = torch.zeros(1, **f64)
        dc = torch.empty(Ne, **f64)
        dpsi = torch.empty(Ne, **f64)
        Usnap = torch.zeros((k, N), **f64)
        Hel = torch.zeros((Ne + 1) * k * (k + 1) // 2, **f64) if args.rom_path == "elem" else None
        Phi = torch.zeros((k, N), **f64)
        H = torch.zeros(k * k, **f64)
        b = torch.zeros(k, **f64)
        Hw = torch.zeros(k * k, **f64)
        y = torch.zeros(k, **f64)
        Jk = torch.zeros(R, **f64)
        rn = torch.zeros((R, 2), **f64)
        uk = torch.zeros(N, **f64)
        Jr = torch.zeros(R, **f64)
        dcr = torch.empty(Ne, **f64)
        dpr = torch.empty((R, Ne), **f64)
        rho_r = torch.empty(Ne, **f64)
        Jw = torch.zeros(1, **f64)
        rnw = torch.zeros(2, **f64)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
        # initial snapshot window: HDM solves of k seeded designs (setup, untimed)
        for i in range(k):
            T.topo_filter(torch.as_tensor(snaps[:, i].copy()).to(**f64), rho)
            T.topo_solve_hdm(rho, F, Usnap[i:i + 1], rtol=1e-8, maxit=400000, prec=prec)
        stream.synchronize()

    ev = lambda: torch.cuda.Event(enable_timing=True)
    copy_stream = torch.cuda.Stream(device=dev)
    stats = dict(step=[], hdm=[], solve=[], build=[], rom=[], rom_batch=[], iters=[], outer=[], relres=[], poly=[], mg=[],
                 fallback=[], start_relres=[])
    warm = {"kk": 0}  # reduced dimension of the basis the previous step left (0: none yet)

    def step(s, record=True, host_io=None):
        """One trust-region-shaped pass; host_io = (pinned inputs, pinned outputs) for e2e."""
        e0, e1, e2, e3, es0, es1 = ev(), ev(), ev(), ev(), ev(), ev()
        e0.record(stream)
        if host_io is not None:
            hin, hout = host_io
            d_cent[s].copy_(hin["centre"][s], non_blocking=True)
            # the candidates travel on a copy stream while the HDM eval and the basis update run;
            # the ROM evaluations wait for them (the previous step's readers are done: the step
            # ends with a synchronisation)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                d_cand.copy_(hin["cands"], non_blocking=True)
        T.topo_filter(d_cent[s], rho)
        kw = warm["kk"] if args.hdm_start == "rom" else 0
        if kw:
            # the HDM solve starts from the ROM prediction at the new centre on the current basis,
            # as the trust-region driver starts its solves from the reduced state
            if Hel is not None:
                T.topo_rom_solve_elem(rho, Hel, kw, b[:kw], Hw[:kw * kw], y[:kw], Jw)
            else:
                T.topo_rom_solve(rho, Phi[:kw], kw, b[:kw], Hw[:kw * kw], y[:kw], Jw, prec)
            T.topo_rom_error(rho, Phi[:kw], kw, y[:kw], f, rnw, Uc[0])
        else:
            Uc.zero_()
        es0.record(stream)
        info = T.topo_solve_hdm(rho, F, Uc, rtol=1e-8, maxit=400000, prec=prec)
        es1.record(stream)
        assert info["status"] == 0, info
        T.topo_compliance_grad(rho, Uc, F, J, dc, dpsi)
        e1.record(stream)
        Usnap[s % k].copy_(Uc[0])
        # the element path forms H(rho) per density from Hel: the build forms Phi and b only
        kk = T.topo_rom_build(rho, Usnap, Phi, None if Hel is not None else H, b, f)
        if Hel is not None:
            T.topo_rom_elem(Phi[:kk], kk, Hel)
        warm["kk"] = kk
        e2.record(stream)
        if host_io is not None:
            stream.wait_stream(copy_stream)
        rom_ev = []
        if args.rom_batch and Hel is not None:
            # all R candidates in one call: one filter, one pass over Hel per 32 candidates,
            # batched reduced solves, residuals and gradients
            a, bq = ev(), ev()
            a.record(stream)
            T.topo_rom_eval_batch(d_cand, Hel, Phi[:kk], kk, b[:kk], f, Jk, rn, None, dpr)
            bq.record(stream)
            rom_ev.append((a, bq))
        else:
            for r in range(R):
                a, bq = ev(), ev()
                a.record(stream)
                T.topo_filter(d_cand[r], rho_r)
                if Hel is not None:
                    T.topo_rom_solve_elem(rho_r, Hel, kk, b[:kk], Hw[:kk * kk], y[:kk], Jk[r:r + 1])
                else:
                    T.topo_rom_solve(rho_r, Phi[:kk], kk, b[:kk], Hw[:kk * kk], y[:kk], Jk[r:r + 1], prec)
                T.topo_rom_error(rho_r, Phi[:kk], kk, y[:kk], f, rn[r], uk)
                T.topo_compliance_grad(rho_r, uk, F, Jr[r:r + 1], dcr, dpr[r])
                bq.record(stream)
                rom_ev.append((a, bq))
        if host_io is not None:
            hout["J"].copy_(J, non_blocking=True)
            hout["dpsi"].copy_(dpsi, non_blocking=True)
            hout["Jk"].copy_(Jk, non_blocking=True)
            hout["rn"].copy_(rn, non_blocking=True)
            hout["dpr"].copy_(dpr, non_blocking=True)
        e3.record(stream)
        e3.synchronize()
        if record:
            stats["step"].append(e0.elapsed_time(e3))
            stats["hdm"].append(e0.elapsed_time(e1))
            stats["solve"].append(es0.elapsed_time(es1))
            stats["build"].append(e1.elapsed_time(e2))
            if len(rom_ev) == 1 and R > 1:  # the batched call: R evaluations that finish together
                stats["rom_batch"].append(rom_ev[0][0].elapsed_time(rom_ev[0][1]))
                stats["rom"].extend([stats["rom_batch"][-1] / R] * R)
            else:
                stats["rom"].extend(a.elapsed_time(bq) for a, bq in rom_ev)
            stats["iters"].append(info["iters"])
            stats["outer"].append(info["outer"])
            stats["poly"].append(info.get("poly", 0))
            stats["mg"].append(info.get("mg_levels", 0))
            stats["fallback"].append(info.get("fallback", 0))
            stats["relres"].append(info["relres"])
            if kw:
                stats["start_relres"].append(rnw[1].item())
        return info

    with torch.cuda.stream(stream):
        for s in range(args.warmup):
            flush.zero_()
            step(s, record=False)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = str(dev.index or 0)
        sampler = ClockSampler(gpu_id)
        sampler.start()
        n0 = native.launch_count()
        t_wall0 = time.perf_counter()
        for s in range(args.warmup, args.warmup + args.steps):
            flush.zero_()
            step(s)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        launches = native.launch_count() - n0
        clocks = sampler.stop()

        # end-to-end through the public API with host buffers: pinned inputs copied in and
        # results copied out inside every timed step
        hin = dict(centre=torch.as_tensor(centres.T.copy()).pin_memory(), cands=torch.as_tensor(cands.T.copy()).pin_memory())
        hout = dict(J=torch.zeros(1, dtype=torch.float64).pin_memory(), dpsi=torch.zeros(Ne, dtype=torch.float64).pin_memory(),
                    Jk=torch.zeros(R, dtype=torch.float64).pin_memory(), rn=torch.zeros((R, 2), dtype=torch.float64).pin_memory(),
                    dpr=torch.zeros((R, Ne), dtype=torch.float64).pin_memory())
        e2e_steps = []
        saved = stats["step"]
        stats_e2e = dict(step=[], hdm=[], solve=[], build=[], rom=[], rom_batch=[], iters=[], outer=[], relres=[], poly=[], mg=[],
                 fallback=[], start_relres=[])
        stats_main = stats
        # centres the timed pass has not visited: their states are not in the snapshot window
        for s in range(args.warmup + args.steps, args.warmup + 2 * args.steps):
            flush.zero_()
            stats = stats_e2e
            step(s, host_io=(hin, hout))
        stats = stats_main
        e2e_ms = statistics.fmean(stats_e2e["step"]) if stats_e2e["step"] else float("nan")
        h2d = (Ne + R * Ne) * 8
        d2h = (1 + Ne + R + 2 * R + R * Ne) * 8

        # plain FP64 HDM evaluation rate (the comparison path)
        hdm64 = []
        for s in range(min(2, args.steps)):
            a, bq = ev(), ev()
            a.record(stream)
            T.topo_filter(d_cent[args.warmup + s], rho)
            U64 = torch.zeros((1, N), **f64)
            info64 = T.topo_solve_hdm(rho, F, U64, rtol=1e-8, maxit=400000, prec="fp64")
            J64 = torch.zeros(1, **f64)
            T.topo_compliance_grad(rho, U64, F, J64, dc, dpsi)
            bq.record(stream)
            bq.synchronize()
            hdm64.append(a.elapsed_time(bq))

        # Accuracy probe (untimed), compared with the CPU oracle on the same inputs by the caller:
        # the HDM compliance at the first timed centre (the step's rtol 1e-8, and FP64 at rtol
        # 1e-13), and a ROM evaluation at candidate 0 on a basis of the first k_acc snapshot
        # designs, each solved by the GPU (the oracle solves them itself).
        s0 = args.warmup
        T.topo_filter(d_cent[s0], rho)
        probe = {"centre_step": s0}
        for key, rt, pr in (("J_rtol1e-8", 1e-8, prec), ("J_fp64_rtol1e-13", 1e-13, "fp64")):
            Up = torch.zeros((1, N), **f64)
            infp = T.topo_solve_hdm(rho, F, Up, rtol=rt, maxit=400000, prec=pr)
            Jp = torch.zeros(1, **f64)
            T.topo_compliance_grad(rho, Up, F, Jp, dc, dpsi)
            probe[key] = Jp.item()
            probe[key + "_relres"] = infp["relres"]
            probe[key + "_floor"] = infp["floor"]
        k_acc = min(args.k_acc, k)
        Us_acc = torch.zeros((k_acc, N), **f64)
        for i in range(k_acc):
            T.topo_filter(torch.as_tensor(snaps[:, i].copy()).to(**f64), rho)
            T.topo_solve_hdm(rho, F, Us_acc[i:i + 1], rtol=1e-13, maxit=400000, prec="fp64")
        T.topo_filter(d_cent[s0], rho)
        Phi_a = torch.zeros_like(Us_acc)
        Ha = torch.zeros(k_acc * k_acc, **f64)
        ba = torch.zeros(k_acc, **f64)
        ka = T.topo_rom_build(rho, Us_acc, Phi_a, Ha, ba, f)
        Hel_a = torch.zeros((Ne + 1) * ka * (ka + 1) // 2, **f64)
        T.topo_rom_elem(Phi_a[:ka], ka, Hel_a)
        T.topo_filter(d_cand[0], rho_r)
        Jka = torch.zeros(1, **f64)
        rna = torch.zeros(2, **f64)
        T.topo_rom_solve_elem(rho_r, Hel_a, ka, ba[:ka], Hw[:ka * ka], y[:ka], Jka)
        T.topo_rom_error(rho_r, Phi_a[:ka], ka, y[:ka], f, rna, uk)
        T.topo_check()
        probe.update(k_acc=ka, Jk=Jka.item(), rom_resnorm=rna[0].item())
        del Hel_a, Phi_a, Us_acc
        # ROM model error (a property of the method, not a numerical error): the ROM's J_k on
        # the last timed basis against the FP64 HDM compliance at the same candidates
        kk = T.topo_rom_build(rho, Usnap, Phi, H, b, f)
        if Hel is not None:
            T.topo_rom_elem(Phi[:kk], kk, Hel)
        model = {"J_rel": [], "resnorm_rel": []}
        for r in range(min(4, R)):
            T.topo_filter(d_cand[r], rho_r)
            Jr1 = torch.zeros(1, **f64)
            rn1 = torch.zeros(2, **f64)
            if Hel is not None:
                T.topo_rom_solve_elem(rho_r, Hel, kk, b[:kk], Hw[:kk * kk], y[:kk], Jr1)
            else:
                T.topo_rom_solve(rho_r, Phi[:kk], kk, b[:kk], Hw[:kk * kk], y[:kk], Jr1, prec)
            T.topo_rom_error(rho_r, Phi[:kk], kk, y[:kk], f, rn1, uk)
            Uh = torch.zeros((1, N), **f64)
            T.topo_solve_hdm(rho_r, F, Uh, rtol=1e-10, maxit=400000, prec="fp64")
            Jh = torch.zeros(1, **f64)
            T.topo_compliance_grad(rho_r, Uh, F, Jh, dcr, dpr[0])
            model["J_rel"].append(abs(Jr1.item() - Jh.item()) / abs(Jh.item()))
            model["resnorm_rel"].append(rn1[1].item())
        T.topo_check()
        J_centre = J.item()

        # K(rho) V for a block of m = 64 columns (the method's central operator at its roofline size):
        # FP32 (HBM-bound) and FP64 (ALU-bound), timed with CUDA events, L2 flushed before each
        apply_rf = None
        if p.dim == 2:
            ma = 64
            apply_rf = {}
            # FP32 with a 16-byte column pitch (the TMA-staged form), FP32 with the contiguous
            # pitch N (N % 4 == 2 here: the cp.async-staged form) and FP64
            for key, pr, dt, pad in (("fp32", "fp32", torch.float32, 4), ("fp32_cpasync", "fp32", torch.float32, 1),
                                     ("fp64", "fp64", torch.float64, 1)):
                ldp = -(-N // pad) * pad
                Va = torch.randn((ma, ldp), dtype=dt, device=dev)[:, :N]
                Ya = torch.empty((ma, ldp), dtype=dt, device=dev)[:, :N]
                T.topo_apply_K(rho, Va, Ya, pr)  # warm-up
                ts = []
                for _ in range(5):
                    flush.zero_()
                    a0, a1 = ev(), ev()
                    a0.record(stream)
                    T.topo_apply_K(rho, Va, Ya, pr)
                    a1.record(stream)
                    a1.synchronize()
                    ts.append(a0.elapsed_time(a1))
                apply_rf[key] = statistics.median(ts)
                del Va, Ya

    K = args.steps
    step_ms = statistics.fmean(stats["step"])
    t_local = sum(stats["step"]) / 1e3
    times = [t_local, t_wall, e2e_ms * K / 1e3]
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor(times, dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        times = tt.tolist()
    t_max = times[0]
    evals = (1 + R) * K * world
    value = evals / t_max
    e2e_value = evals / times[2]
    # Dominant kernel: the persistent PCG launch (one per HDM solve), FP64-ALU bound at this size
    # (the whole working set sits in L2). FP64 flops it performs per DOF and iteration: stencil
    # apply 2 * 3^d * d (36 in 2D, 162 in 3D), delta 2, the five updates, z and the two dots 13.
    hdm_ms = statistics.fmean(stats["hdm"])
    solve_ms = statistics.fmean(stats["solve"])  # the topo_solve_hdm call alone (one PCG launch)
    iters = statistics.fmean(stats["iters"])
    outer = statistics.fmean(stats["outer"])
    # FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk (4 flop) x 2.07 GHz
    # (NVIDIA's nominal FP64 rate is 1.25 TFLOP/s; an FMA microbenchmark on GB300 measured 1.19).
    fp64_peak = 152 * 4 * 2.07e9 / 1e12
    # FP32: 152 SMs x 128 FMA/clk (256 flop) x 2.07 GHz
    fp32_peak = 152 * 256 * 2.07e9 / 1e12
    poly = int(max(stats["poly"])) if stats.get("poly") else 0
    mg_levels = int(max(stats["mg"])) if stats.get("mg") else 0
    # FP32 flops of the polynomial preconditioner per DOF and iteration: d - 1 applies of the FP32
    # stencil (36 flop/DOF in 2D, 162 in 3D) with three vector updates (6 flop/DOF) each
    flop32_dof = max(0, poly - 1) * ((36.0 if p.dim == 2 else 162.0) + 6.0)
    if mg_levels:
        # FP32 V-cycle (2 Chebyshev steps per side): per level 4 stencil applies (one pre step,
        # the residual, two post steps) of 2 * 3^d * d flop/DOF plus ~6 flop/DOF of updates each;
        # coarser levels add 1/4 (2D) or 1/8 (3D) of the DOFs per level
        per = 4 * ((36.0 if p.dim == 2 else 162.0) + 6.0)
        flop32_dof = per * (4.0 / 3.0 if p.dim == 2 else 8.0 / 7.0)
    if prec == "fp64":
        # FP64 per iteration: one stencil apply (36 flop/DOF in 2D, 162 in 3D) plus the vector
        # updates and dot products
        flop_dof = 51.0 if p.dim == 2 else 177.0
        peak, peak_source = fp64_peak, "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz (measured FMA peak 1.19)"
        rkernel = ("pcg2_mg_kernel (assembled-stencil Chronopoulos-Gear PCG with the FP32 multigrid V-cycle "
                   "preconditioner, one launch per HDM solve)" if mg_levels else
                   "pcg2_kernel (assembled-stencil Chronopoulos-Gear PCG, one launch per HDM solve)")
    else:
        # FP32 inner iterations of the element-form apply (2 ndof_e^2 flop per element: 64 flop/DOF
        # in 2D, 384 in 3D) plus the updates and dots (13); the time also holds the FP64 completion
        flop_dof = 77.0 if p.dim == 2 else 397.0
        peak, peak_source = fp32_peak, "derived: 152 SMs x 256 FP32 flop/clk x 2.07 GHz"
        rkernel = "pcg_kernel<DIM, float> (FP32 inner, element form) with FP64 refinement and completion"
    flops_launch = N * flop_dof * iters
    achieved = flops_launch / (solve_ms * 1e-3) / 1e12
    achieved32 = N * flop32_dof * iters / (solve_ms * 1e-3) / 1e12 if prec == "fp64" else 0.0
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        hbm_peak = 6800.0
    rom_ms = sorted(stats["rom"])
    pct = lambda q: rom_ms[min(len(rom_ms) - 1, int(q * len(rom_ms)))] if rom_ms else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: " + (f"MBB {p.nx}x{p.ny} Q4" if p.dim == 2 else
                                                      f"cantilever {p.nx}x{p.ny}x{p.nz} H8") +
                               f" ({N} DOFs), 1 HDM eval + basis update (k={k}) + {R} ROM evals per step", "k": k, "rom_evals_per_step": R, "precision": prec,
                   "rom_path": args.rom_path, "rom_batch": bool(args.rom_batch),
                   "rtol": 1e-8, "hdm_start": ("ROM prediction at the centre on the previous step's basis"
                                               if args.hdm_start == "rom" else "zero"),
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "p50_ms": pct(0.50), "p99_ms": pct(0.99),
        "latency_note": ("p50/p99 of the per-evaluation time; with the batched ROM evaluation (one call for "
                         "all R candidates) that is the batch time / R, and every candidate of a step is "
                         "ready after rom_batch_ms") if stats["rom_batch"] else "p50/p99 of single ROM evaluations",
        "rom_batch_ms": {"p50": statistics.median(stats["rom_batch"]),
                         "max": max(stats["rom_batch"])} if stats["rom_batch"] else None,
        "rom_eval_ms_mean": statistics.fmean(rom_ms) if rom_ms else None,
        "hdm_eval_ms": hdm_ms, "hdm_fp64_eval_ms": statistics.fmean(hdm64) if hdm64 else None,
        "hdm_fp64_evals_per_s": 1e3 / statistics.fmean(hdm64) if hdm64 else None,
        "hdm_evals_per_s": 1e3 / hdm_ms, "rom_evals_per_s": 1e3 / statistics.fmean(rom_ms) if rom_ms else None,
        "basis_update_ms": statistics.fmean(stats["build"]),
        "pcg": {"inner_iters": iters, "outer": outer, "relres": max(stats["relres"]), "fp64_iters": info64["iters"],
                "start_relres_mean": statistics.fmean(stats["start_relres"]) if stats["start_relres"] else None,
                "fp64_iters_note": "fp64_iters: the plain FP64 HDM evaluation (hdm_fp64_eval_ms), started from zero"},
        "accuracy": {"probe": probe, "J_centre_last_step": J_centre},
        "rom_model_error": {"candidates": len(model["J_rel"]), "k": kk, **model,
                            "note": "|J_k - J_HDM| / J_HDM at candidate designs (FP64 HDM at rtol 1e-10), next to "
                                    "the ROM residual ||r|| / ||f||: the model error the trust region controls, "
                                    "not a numerical error"},
        "roofline": {"kernel": rkernel,
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": pcg_traffic() if (prec == "fp64" and args.config == "mbb600x200") else None,
                     "traffic_unit": "bytes per launch", "launch_ms": solve_ms,
                     "peak_source": peak_source,
                     "flop_per_dof_iter": flop_dof, "pcg_poly": poly, "mg_levels": mg_levels,
                     "mg_fallbacks": int(sum(stats["fallback"])) if stats.get("fallback") else 0,
                     "fp32_preconditioner": {"flop_per_dof_iter": flop32_dof, "achieved": achieved32,
                                             "peak": fp32_peak, "unit": "TFLOP/s",
                                             "frac": achieved32 / fp32_peak},
                     "bytes_per_dof_iter": 96.0,
                     "bytes_def": "algorithmic FP64 bytes of a CG iteration: the apply (read z, write w: 16 B/DOF) "
                                  "and ten vector streams of the update (read x, r, p, s, w; write x, r, p, s, z: "
                                  "80 B/DOF)",
                     "achieved_gbs": 96.0 * N * iters / (solve_ms * 1e-3) / 1e9,
                     "frac_hbm": 96.0 * N * iters / (solve_ms * 1e-3) / 1e9 / hbm_peak,
                     "note": "FP64 CG flops against the FP64 peak; the FP32 preconditioner's flops (the "
                             "multigrid V-cycle, else the polynomial) are counted separately against the FP32 peak. "
                             "Neither pipe is saturated: each iteration is bound by the latency of its dependent "
                             "steps (the grid barrier of the CG and the halo exchanges of the preconditioner)",
                     "hbm_peak_gbs": hbm_peak},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "every step copies its centre and its R candidate designs in from pinned host memory "
                        "(the candidates on a copy stream, overlapped with the step's HDM eval and basis "
                        "update) and reads J, dpsi, J_k, the residual norms and the R gradients back before "
                        "the step ends"},
        "apply_roofline": None if apply_rf is None else {
            "call": "topo_apply_K, m = 64 columns (node-centric 2D block apply)",
            "fp32": {"bound": "hbm", "ms": apply_rf["fp32"], "unit": "GB/s",
                     "achieved": (2 * 64 * N * 4 + p.nel * 8) / (apply_rf["fp32"] * 1e-3) / 1e9,
                     "peak": hbm_peak, "frac": (2 * 64 * N * 4 + p.nel * 8) / (apply_rf["fp32"] * 1e-3) / 1e9 / hbm_peak,
                     "bytes": 2 * 64 * N * 4 + p.nel * 8, "ld": -(-N // 4) * 4,
                     "staging": "TMA halo-row boxes, persistent grid",
                     "bytes_def": "read V + write Y (FP32) + read rho, once each"},
            "fp32_cpasync": {"bound": "hbm", "ms": apply_rf["fp32_cpasync"], "unit": "GB/s",
                             "achieved": (2 * 64 * N * 4 + p.nel * 8) / (apply_rf["fp32_cpasync"] * 1e-3) / 1e9,
                             "peak": hbm_peak,
                             "frac": (2 * 64 * N * 4 + p.nel * 8) / (apply_rf["fp32_cpasync"] * 1e-3) / 1e9 / hbm_peak,
                             "ld": N, "staging": "per-thread cp.async (leading dimension not a multiple of 4)"},
            "fp64": {"bound": "alu", "ms": apply_rf["fp64"], "unit": "TFLOP/s",
                     "achieved": 36.0 * 64 * N / (apply_rf["fp64"] * 1e-3) / 1e12,
                     "peak": fp64_peak, "frac": 36.0 * 64 * N / (apply_rf["fp64"] * 1e-3) / 1e12 / fp64_peak,
                     "flop_def": "36 flop per DOF and column (18 FMA: 3x3 blocks of 2x2 per node row)"}},
        "gpu_launches": launches, "clocks": clocks, "wall_s_timed": t_wall,
    }
    return out, p, dict(centre=centres[:, args.warmup].copy(), cand=cands[:, 0].copy(), snaps=snaps[:, :k_acc].copy())


def run_batch(args):
    """Batched form: 256 uneven MBB instances (nx log-uniform in [40, 400], ny = nx/2, 1..8
    top-edge load cases, own seeded design, a reduced basis of k in {8, 16, 32} vectors). One
    step = one HDM design evaluation of every instance (batched filter, all state solves,
    batched compliance and filtered gradient) plus one reduced solve of every instance at its
    design (all instances' reduced matrices and Cholesky solves in three launches). The bases are
    seeded random vectors orthonormalised by topo_rom_build (the reduced solve's cost does not
    depend on the basis). Metric: instances evaluated per second."""
    import torch
    from paper_2004_05756_gb300 import build, native
    from paper_2004_05756_gb300 import workloads as w

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    insts = w.batch_instances(CONFIGS["batch256"]["count"])
    probs = [d["problem"] for d in insts]
    f64 = dict(dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        B = native.TopoBatch(probs, stream=stream)
        psis = [torch.as_tensor(w.design_field(p, d["design_seed"])).to(**f64) for p, d in zip(probs, insts)]
        rhos = [torch.empty(p.nel, **f64) for p in probs]
        Fs = [torch.as_tensor(p.F.T.copy()).to(**f64) for p in probs]
        Us = [torch.zeros_like(F) for F in Fs]
        J = torch.zeros(len(probs), **f64)
        dcs = [torch.empty(p.nel, **f64) for p in probs]
        dps = [torch.empty(p.nel, **f64) for p in probs]
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        # reduced bases (setup, untimed): k seeded random vectors per instance, orthonormalised by
        # the library, and their element reduced matrices
        gen = torch.Generator(device="cuda")
        gen.manual_seed(4242)
        B.topo_batch_filter(psis, rhos)
        ks, Hels, bs, Hws, ys = [], [], [], [], []
        for i, (p, d) in enumerate(zip(probs, insts)):
            T = B.context(i)
            k = d["k"]
            snaps = torch.randn((k, p.ndof), generator=gen, **f64)
            Phi = torch.zeros((k, p.ndof), **f64)
            bvec = torch.zeros(k, **f64)
            kk = T.topo_rom_build(rhos[i], snaps, Phi, None, bvec, Fs[i][0])
            Hel = torch.empty((p.nel + 1) * kk * (kk + 1) // 2, **f64)
            T.topo_rom_elem(Phi[:kk], kk, Hel)
            ks.append(kk)
            Hels.append(Hel)
            bs.append(bvec[:kk])
            Hws.append(torch.empty(kk * kk, **f64))
            ys.append(torch.empty(kk, **f64))
            del snaps, Phi
        Jk = torch.zeros(len(probs), **f64)

        def body():
            B.topo_batch_filter(psis, rhos)
            for U in Us:
                U.zero_()
            B.topo_batch_solve_hdm(rhos, Fs, Us, rtol=1e-8, maxit=100000, info=False)
            B.topo_batch_compliance_grad(rhos, Us, Fs, J, dcs, dps)
            B.topo_batch_rom_solve_elem(rhos, Hels, ks, bs, Hws, ys, Jk)

        def timed(run):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        # eager warm-up: autotunes the CTAs per SM and stages the launch tables; the step is then
        # captured once in a CUDA graph (the identical solve call needs no host synchronisation)
        for _ in range(args.warmup):
            flush.zero_()
            timed(body)
        graph, graph_error, per_step = None, None, 0
        try:
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            n0 = native.launch_count()
            with torch.cuda.graph(g, stream=stream):
                body()
            per_step = native.launch_count() - n0
            graph = g
        except Exception as e:  # capture refused: time the eager step instead
            graph_error = str(e).splitlines()[0][:200]
        run = graph.replay if graph is not None else body
        n0 = native.launch_count()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            times.append(timed(run))
        launches = per_step * args.steps if graph is not None else native.launch_count() - n0
        infos = B.topo_batch_solve_hdm(rhos, Fs, [torch.zeros_like(F) for F in Fs], rtol=1e-8, maxit=100000)
        J_batch = J.cpu().numpy().copy()
        # the same instances' state solves as sequential topo_solve_hdm calls (one context each,
        # the single-solve path's defaults), timed the same way
        ctxs = [native.Topo(p, stream=stream) for p in probs]
        Us2 = [torch.zeros_like(F) for F in Fs]

        def sequential():
            for T, rho, F, U in zip(ctxs, rhos, Fs, Us2):
                U.zero_()
                T.topo_solve_hdm(rho, F, U, rtol=1e-8, maxit=100000, prec="fp64", info=False)

        flush.zero_()
        timed(sequential)  # warm-up: first-call scratch
        seq_times = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            seq_times.append(timed(sequential))
        seq_infos = [T.topo_solve_hdm(rho, F, torch.zeros_like(F), rtol=1e-8, maxit=100000, prec="fp64")
                     for T, rho, F in zip(ctxs, rhos, Fs)]
        for T in ctxs:
            T.close()
        solve_only = []
        for _ in range(max(1, min(args.steps, 3))):
            for U in Us:
                U.zero_()
            flush.zero_()
            solve_only.append(timed(lambda: B.topo_batch_solve_hdm(rhos, Fs, Us, rtol=1e-8, maxit=100000,
                                                                   info=False)))
        rho_host = [r.cpu().numpy() for r in rhos]
        # the reduced solves alone: the batched call against one call per instance
        rom_batch, rom_each = [], []
        ctxs = [B.context(i) for i in range(len(probs))]
        Jk1 = torch.zeros(len(probs), **f64)
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            rom_batch.append(timed(lambda: B.topo_batch_rom_solve_elem(rhos, Hels, ks, bs, Hws, ys, Jk)))
            flush.zero_()
            rom_each.append(timed(lambda: [T.topo_rom_solve_elem(rhos[i], Hels[i], ks[i], bs[i], Hws[i], ys[i],
                                                                 Jk1[i:i + 1]) for i, T in enumerate(ctxs)]))
        rom_dev = float((Jk - Jk1).abs().max().item() / Jk1.abs().max().item())
    ms = statistics.fmean(times)
    at_floor = [i for i, x in enumerate(infos) if x["relres"] > 1e-8]
    cpu = None
    if not args.no_cpu_baseline:
        # cpu_baseline leg: the oracle's HDM evaluation (filter, SuperLU solve, compliance) of the
        # instances whose batched solve stopped at its FP64 rounding floor above rtol, timed as
        # run; their compliance errors against the oracle come with it
        from oracle import fem, hatfilter
        t0 = time.perf_counter()
        errs = []
        for i in at_floor:
            pi = probs[i]
            rho_o = hatfilter.filter_fwd(pi, w.design_field(pi, insts[i]["design_seed"]))
            Jo = fem.compliance(pi, fem.solve(pi, rho_o))
            errs.append({"instance": i, "shape": [pi.nx, pi.ny], "load_cases": int(pi.F.shape[1]),
                         "relres": infos[i]["relres"], "floor": infos[i]["floor"],
                         "J_rel_err": float(abs(J_batch[i] - Jo) / abs(Jo)),
                         "rho_max_abs_err": float(np.max(np.abs(rho_host[i] - rho_o)))})
        t_cpu = time.perf_counter() - t0
        hi = host_info()
        cpu = {"value": len(at_floor) / t_cpu if at_floor else None, "unit": UNIT,
               "cores": max(1, hi["blas_threads"] or 1), "kind": "oracle",
               "sample": f"oracle HDM evaluations (filter, SuperLU solve, compliance) of the {len(at_floor)} "
                         f"instances whose batched solve stopped at the FP64 floor", "host": hi,
               "floor_limited": errs,
               "max_J_rel_err": max((e["J_rel_err"] for e in errs), default=None)}
    ndof = sum(p.ndof for p in probs)
    # FP64 work of the solves: 51 flops per DOF, load case and iteration (stencil apply 36,
    # delta 2, updates and dots 13)
    flops = sum(p.ndof * p.F.shape[1] * x["iters"] * 51.0 for p, x in zip(probs, infos))
    fp64_peak = 152 * 4 * 2.07e9
    nlc = sum(p.F.shape[1] for p in probs)
    return {"metric": METRIC, "value": len(probs) * 1e3 / ms, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch256: {len(probs)} MBB Q4 instances, nx 40..400 log-uniform, "
                                   f"{ndof} DOFs, {nlc} load cases, reduced bases k in {{8, 16, 32}}; one HDM "
                                   f"eval and one reduced solve of every instance per step",
                       "instances": len(probs), "total_dofs": ndof, "load_cases": nlc,
                       "l2": "flushed between steps (256 MB write)"},
            "max_iters": max(x["iters"] for x in infos), "all_converged": all(x["status"] == 0 for x in infos),
            "max_relres": max(x["relres"] for x in infos), "max_floor": max(x["floor"] for x in infos),
            "instances_at_floor": len(at_floor), "gpu_launches": launches,
            "batch_solve_ms": statistics.fmean(solve_only),
            "rom_reduced_solves": {"what": "all instances' reduced solves (k in {8, 16, 32}) in one "
                                           "topo_batch_rom_solve_elem call, against one topo_rom_solve_elem "
                                           "call per instance", "batched_ms": statistics.fmean(rom_batch),
                                   "per_instance_ms": statistics.fmean(rom_each),
                                   "max_rel_diff_of_Jk": rom_dev},
            "sequential": {"what": f"the same {len(probs)} state solves as sequential topo_solve_hdm calls (one "
                                   f"context per instance, multigrid-preconditioned, rtol 1e-8), CUDA events",
                           "ms": statistics.fmean(seq_times), "runs": len(seq_times),
                           "speedup_of_batch_solve": statistics.fmean(seq_times) / statistics.fmean(solve_only),
                           "max_iters": max(x["iters"] for x in seq_infos),
                           "all_converged": all(x["status"] == 0 for x in seq_infos)},
            "cpu_baseline": cpu,
            "cuda_graph": graph is not None, "cuda_graph_error": graph_error,
            "roofline": {"kernel": "pcg2_batch_kernel (all instances' solves, one launch)", "bound": "alu",
                         "achieved": flops / (ms * 1e-3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                         "frac": flops / (ms * 1e-3) / fp64_peak, "traffic": None}}


def _serving_line(srv, reqs, res, wall, clocks=None):
    from paper_2004_05756_gb300 import serving
    s = serving.summarize(res, wall)
    return {"requests": len(reqs), "evals_per_s": s["evals_per_s"], "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"],
            "accepted": s["accepted"], "inside": s["inside"], "median_ratio": s["median_ratio"],
            "rom_evals": s["rom_evals"], "mean_basis_size": s["mean_basis_size"],
            "max_concurrency": srv.max_concurrency, "session_evictions": srv.evictions,
            "session_restores": srv.restores, "evict_ms_total": sum(srv.evict_ms),
            "restore_ms_total": sum(srv.restore_ms), "wall_s": wall, "clocks": clocks}


def run_serving(args):
    """Serving form: a seeded Poisson stream of trust-region major iterations, 50/50 2D Q4
    (100x50 .. 800x400) and 3D H8 (32^3 .. 96x48x48), admitted by free HBM into slots that
    overlap on the GPU. Reports evals/s and p50/p99 latency (arrival to completion).

    With --sweep: the capacity first (a saturated stream: --cap-requests requests all queued at
    t = 0, throughput = capacity), then --sweep-requests Poisson requests (seed 7) at 0.5, 1 and
    2 times that capacity, each with the SM clocks sampled while it runs."""
    import torch
    from paper_2004_05756_gb300 import serving

    torch.cuda.set_device(0)
    srv = serving.Server(slots=args.slots)
    warm = serving.poisson_requests(2, rate_per_s=100.0, seed=99, q4=((100, 50), (120, 60)),
                                    h8=((16, 16, 16), (20, 20, 20)))
    srv.run(warm, realtime=False)
    base = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    if args.sweep:
        cap_reqs = serving.poisson_requests(args.cap_requests, rate_per_s=1.0, seed=7)
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        t0 = time.perf_counter()
        res = srv.run(cap_reqs, realtime=False)
        wall = time.perf_counter() - t0
        cap_line = _serving_line(srv, cap_reqs, res, wall, sampler.stop())
        cap = cap_line["evals_per_s"]
        runs = []
        for f in (0.5, 1.0, 2.0):
            srv = serving.Server(slots=args.slots)
            reqs = serving.poisson_requests(args.sweep_requests, rate_per_s=f * cap, seed=7)
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            t0 = time.perf_counter()
            res = srv.run(reqs, realtime=True)
            wall = time.perf_counter() - t0
            line = _serving_line(srv, reqs, res, wall, sampler.stop())
            line.update(load=f, rate_per_s=f * cap)
            runs.append(line)
        return dict(base, value=cap, config={
            "workload": f"serving sweep: capacity from {args.cap_requests} requests queued at t=0, then "
                        f"{args.sweep_requests} Poisson requests (seed 7) at 0.5/1/2 x capacity; 50/50 Q4 "
                        f"100x50..800x400 and H8 32^3..96x48x48 standalone requests (a fresh run's first major "
                        f"iteration), {args.slots} slots", "slots": args.slots},
            capacity=cap_line, sweep=runs)
    if args.sessions > 0:
        reqs = serving.session_requests(args.requests, rate_per_s=args.rate, sessions=args.sessions, seed=7)
    else:
        reqs = serving.poisson_requests(args.requests, rate_per_s=args.rate, seed=7)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    line = _serving_line(srv, reqs, res, wall)
    return dict(base, value=line["evals_per_s"], config={
        "workload": f"serving: {len(reqs)} Poisson requests at {args.rate}/s, 50/50 Q4 100x50..800x400 "
                    f"and H8 32^3..96x48x48, {args.slots} slots, " +
                    (f"{args.sessions} sessions (resident run, window {srv.kmax})" if args.sessions
                     else "standalone requests (a fresh run's first major iteration)"),
        "slots": args.slots, "rate_per_s": args.rate, "sessions": args.sessions}, **line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="mbb600x200", choices=list(CONFIGS))
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--rom-evals", type=int, default=100)
    ap.add_argument("--k-acc", type=int, default=4,
                    help="snapshots of the basis on which the accuracy probe compares the ROM with the oracle")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "fp32_bf16ke"],
                    help="arithmetic of the HDM solve (fp32 forms: FP32 inner PCG in FP64 refinement, which "
                         "stalls on these designs and completes in FP64) and of the Phi-path reduced solves")
    ap.add_argument("--rom-path", default="elem", choices=["elem", "phi"],
                    help="reduced matrix from cached element reduced matrices, or from K(rho) Phi")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hdm-start", default="rom", choices=["rom", "zero"],
                    help="initial iterate of each step's HDM solve: the ROM prediction at the new centre on "
                         "the current basis (as the trust-region driver), or zero")
    ap.add_argument("--rom-batch", type=int, default=1,
                    help="1: the step's R ROM evaluations in one topo_rom_eval_batch call; 0: one by one")
    ap.add_argument("--cpu-baseline-3d", action="store_true",
                    help="time the CPU oracle on a 3D config too (its SuperLU solve takes minutes)")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent request slots")
    ap.add_argument("--requests", type=int, default=32, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=2.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--sweep", action="store_true",
                    help="serving: measure capacity, then Poisson streams at 0.5, 1 and 2 x capacity")
    ap.add_argument("--cap-requests", type=int, default=400, help="serving sweep: requests of the capacity run")
    ap.add_argument("--sweep-requests", type=int, default=2000, help="serving sweep: requests per load level")
    ap.add_argument("--sessions", type=int, default=8,
                    help="serving: optimisation sessions the requests belong to (0 = standalone requests)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")

    if args.impl == "reference":
        # The oracle as it stands, on the host cores. Each step is one bounded sample of the
        # workload, measured as run: an HDM evaluation at that step's centre, a basis update
        # and 2 ROM evaluations (cpu_oracle_step). `value` is the oracle's throughput on the
        # step's mix (1 HDM + basis update + R ROM evals), combined from the measured part times
        # ("projected": true); ms_per_step is the measured time of what each step ran. The
        # oracle needs no warm-up, so warm-up steps are not run.
        if args.config not in ("mbb600x200", "mbb60x20", "cant96x48x48"):
            print(json.dumps({"impl": "reference", "unavailable": f"no oracle arm for config {args.config}"}))
            return
        p = make_problem(args.config)
        psi0, centres, cands, snaps = designs(p, args)
        t0 = time.perf_counter()
        parts = []
        for s in range(max(1, args.steps)):
            parts.append(cpu_oracle_step(p, centres[:, args.warmup + s], cands[:, s % cands.shape[1]], args.k, 2))
        n = len(parts)
        t_hdm = sum(x["t_hdm"] for x in parts) / n
        t_basis = sum(x["t_basis"] for x in parts) / n
        t_rom = sum(x["t_rom"] for x in parts) / n
        value = (1 + args.rom_evals) / (t_hdm + t_basis + args.rom_evals * t_rom)
        hi = host_info()
        sample = (f"per step: 1 HDM eval (SuperLU, 1 thread) at the step's centre + basis update (k={args.k}) + 2 ROM "
                  f"evals on {p.name}; value combines the measured part times for the mix 1 HDM + basis update + "
                  f"{args.rom_evals} ROM evals")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "projected": True,
                "config": {"workload": f"{args.config}: 1 HDM eval + basis update (k={args.k}) + {args.rom_evals} ROM "
                                       f"evals per step", "k": args.k, "rom_evals_per_step": args.rom_evals},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(1, hi["blas_threads"] or 1),
                                 "kind": "oracle", "sample": sample, "host": hi},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "ms_per_step": 1e3 * sum(x["wall"] for x in parts) / n,
                "evals_per_step_run": {"hdm": 1, "basis_updates": 1, "rom": 2},
                "part_ms": {"hdm_eval": 1e3 * t_hdm, "basis_update": 1e3 * t_basis, "rom_eval": 1e3 * t_rom},
                "wall_s": time.perf_counter() - t0}
        print(json.dumps(line), flush=True)
        return

    if args.config == "batch256":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.config == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    out, p, probe_in = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and p.dim == 3 and not args.cpu_baseline_3d:
            # the oracle's direct solve of a 3D mesh of this size takes minutes (fill-in), far
            # beyond a bounded sample; --cpu-baseline-3d times it anyway
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                                   "sample": "not measured: the FP64 oracle's SuperLU solve of this 3D mesh "
                                             "takes minutes, beyond a bounded sample (--cpu-baseline-3d runs it)",
                                   "host": host_info()}
        elif world == 1 and not args.no_cpu_baseline:
            cpu = cpu_oracle_timing(p, probe_in["centre"], probe_in["cand"], args)
            out["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                                   "sample": cpu["sample"], "split_s": cpu["split_s"], "host": cpu["host"],
                                   "part_ms": {"hdm_eval": 1e3 * cpu["t_hdm"], "basis_update": 1e3 * cpu["t_basis"],
                                               "rom_eval": 1e3 * cpu["t_rom"]}}
            out["accuracy"].update(oracle_accuracy(p, probe_in, out["accuracy"]["probe"], cpu["J"], cpu["U"]))
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
