"""Run one hot libtopo call on a named workload, a few times, for profiler captures.

    python -m paper_2004_05756_gb300.profcase --call pcg --prec fp64 --maxit 200
    python -m paper_2004_05756_gb300.profcase --call apply --prec fp32 --m 64 --ld-pad 4
    python -m paper_2004_05756_gb300.profcase --call rom_solve_elem --k 16
    python -m paper_2004_05756_gb300.profcase --call rom_solve --prec fp32 --k 64 --shape 96x48x48

Workloads are the seeded benchmark problems (MBB 600x200 Q4 by default). Prints the mean
CUDA-event time of the call, measured after one warm-up call.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--call", required=True, choices=["pcg", "hdm", "apply", "rom_elem", "rom_solve_elem", "rom_solve",
                                                      "rom_error", "grad", "filter", "rom_eval_batch"])
    ap.add_argument("--R", type=int, default=100, help="rom_eval_batch: candidates per call")
    ap.add_argument("--shape", default="600x200")
    ap.add_argument("--prec", default="fp64")
    ap.add_argument("--m", type=int, default=1)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--maxit", type=int, default=200)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--hdm-kernel", type=int, default=0, help="FP64 solve: 0 stencil C-G PCG, 1 element-form PCG")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="CTAs per SM of the persistent solve (0 = default)")
    ap.add_argument("--rom-tensor", type=int, default=1, help="FP32 projection contraction: 1 tcgen05, 0 SIMT")
    ap.add_argument("--apply-cols", type=int, default=0, help="columns per CTA of the 2D block apply (0 = default)")
    ap.add_argument("--apply-stages", type=int, default=3,
                    help="2D FP32 block apply: TMA units in flight per CTA (2-4), 0 = cp.async staging")
    ap.add_argument("--ld-pad", type=int, default=1, help="round the leading dimension of V, Y up to a multiple")
    ap.add_argument("--poly", type=int, default=0, help="FP64 solve: polynomial preconditioner degree (0 = auto)")
    ap.add_argument("--rtol", type=float, default=1e-30, help="pcg/hdm: relative residual target")
    ap.add_argument("--mg", type=int, default=1, help="FP64 solve: 1 multigrid preconditioner, 0 polynomial")
    ap.add_argument("--mg-deg", type=int, default=2, help="multigrid: Chebyshev smoothing steps per side")
    ap.add_argument("--filter", default="cone", choices=["cone", "helmholtz"], help="density filter")
    ap.add_argument("--rom-asm", type=int, default=1,
                    help="reduced assembly of rom_eval_batch: 1 tensor cores (Ozaki digits), 0 FP64 SIMT")
    ap.add_argument("--mg-single", type=int, default=-1,
                    help="multigrid: nodes of levels run on one CTA (-1: the library's default)")
    a = ap.parse_args(argv)
    import torch

    from paper_2004_05756_gb300 import build, native
    from paper_2004_05756_gb300 import workloads as w

    build.build()
    dims = [int(x) for x in a.shape.split("x")]
    p = w.mbb_2d(*dims) if len(dims) == 2 else w.cantilever_3d(*dims)
    T = native.Topo(p)
    T.topo_set_param(native.TOPO_PARAM_HDM_KERNEL, a.hdm_kernel)
    T.topo_set_param(native.TOPO_PARAM_PCG_BLOCKS_PER_SM, a.blocks_per_sm)
    T.topo_set_param(native.TOPO_PARAM_ROM_TENSOR, a.rom_tensor)
    T.topo_set_param(native.TOPO_PARAM_FILTER, 1 if a.filter == "helmholtz" else 0)
    T.topo_set_param(native.TOPO_PARAM_ROM_ASSEMBLY, a.rom_asm)
    T.topo_set_param(native.TOPO_PARAM_TILE_X, a.apply_cols)
    T.topo_set_param(native.TOPO_PARAM_APPLY_STAGES, a.apply_stages)
    T.topo_set_param(native.TOPO_PARAM_PCG_POLY, a.poly)
    T.topo_set_param(native.TOPO_PARAM_PCG_MG, a.mg)
    T.topo_set_param(native.TOPO_PARAM_MG_DEGREE, a.mg_deg)
    T.topo_set_param(native.TOPO_PARAM_MG_SINGLE_NODES, a.mg_single)
    f64 = dict(dtype=torch.float64, device="cuda")
    psi = torch.as_tensor(w.design_field(p, 0)).to(**f64)
    rho = torch.empty(p.nel, **f64)
    T.topo_filter(psi, rho)
    F = torch.as_tensor(p.F.T.copy()).to(**f64)
    rng = np.random.default_rng(0)
    k = a.k
    Phi = None
    if a.call.startswith("rom"):
        Q, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
        Q[p.fixed == 1] = 0.0
        Phi = torch.as_tensor(Q.T.copy()).to(**f64)
        Hel = torch.zeros((p.nel + 1) * k * (k + 1) // 2, **f64)
        b = torch.as_tensor(Q.T @ p.F[:, 0]).to(**f64)
        Hw = torch.zeros(k * k, **f64)
        y = torch.zeros(k, **f64)
        Jk = torch.zeros(1, **f64)
        rn = torch.zeros(2, **f64)
        if a.call != "rom_elem":
            T.topo_rom_elem(Phi, k, Hel)
        if a.call == "rom_eval_batch":
            cands = torch.as_tensor(w.perturbed_designs(p, w.design_field(p, 0), a.R, amplitude=0.02,
                                                        first_seed=2000).T.copy()).to(**f64)
            JkR = torch.zeros(a.R, **f64)
            rnR = torch.zeros((a.R, 2), **f64)
            dpR = torch.zeros((a.R, p.nel), **f64)
    dt = torch.float64 if a.prec == "fp64" else torch.float32
    ldp = -(-p.ndof // a.ld_pad) * a.ld_pad
    V = torch.randn((a.m, ldp), dtype=dt, device="cuda")[:, :p.ndof]
    Y = torch.empty((a.m, ldp), dtype=dt, device="cuda")[:, :p.ndof]
    U = torch.zeros((1, p.ndof), **f64)
    J = torch.zeros(1, **f64)
    dc = torch.empty(p.nel, **f64)
    dp = torch.empty(p.nel, **f64)

    last_info = {}

    def call():
        if a.call == "pcg":
            U.zero_()
            T.topo_solve_hdm(rho, F, U, rtol=a.rtol, maxit=a.maxit, prec=a.prec, info=False)
        elif a.call == "hdm":  # a full solve to --rtol (iteration count printed below)
            U.zero_()
            last_info.update(T.topo_solve_hdm(rho, F, U, rtol=a.rtol, maxit=400000, prec=a.prec))
        elif a.call == "apply":
            T.topo_apply_K(rho, V, Y, a.prec)
        elif a.call == "rom_elem":
            T.topo_rom_elem(Phi, k, Hel)
        elif a.call == "rom_solve_elem":
            T.topo_rom_solve_elem(rho, Hel, k, b, Hw, y, Jk)
        elif a.call == "rom_solve":
            T.topo_rom_solve(rho, Phi, k, b, Hw, y, Jk, a.prec)
        elif a.call == "rom_eval_batch":
            T.topo_rom_eval_batch(cands, Hel, Phi, k, b, F[0], JkR, rnR, None, dpR)
        elif a.call == "rom_error":
            T.topo_rom_error(rho, Phi, k, y, F[0], rn)
        elif a.call == "grad":
            T.topo_compliance_grad(rho, F, F, J, dc, dp)
        elif a.call == "filter":
            T.topo_filter(psi, rho)

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    e1.synchronize()
    print(f"{a.call} {a.prec} shape={a.shape} m={a.m} k={k} hdm_kernel={a.hdm_kernel} bps={a.blocks_per_sm} "
          f"rom_tensor={a.rom_tensor} apply_cols={a.apply_cols} apply_stages={a.apply_stages} ld={ldp} "
          f"filter={a.filter} rom_asm={a.rom_asm}: "
          f"{e0.elapsed_time(e1) / a.reps * 1e3:.1f} us/call" +
          (f" poly={a.poly} mg={a.mg} deg={a.mg_deg} single={a.mg_single} {last_info}" if last_info else ""))
    T.topo_check()


if __name__ == "__main__":
    main()
