"""Writes tests/golden/cant96x48x48_fp64.txt: the FP64 oracle's state solve of the 3D
cantilever at its full size, 96 x 48 x 48 H8 elements (698,691 DOFs).

The design is the seeded field psi = design_field(p, 0) (filter radius 2), rho = its
linear-filter image (oracle/hatfilter.py). The oracle's own Jacobi-preconditioned CG
(oracle/fem.py, solve_cg) runs to rtol 1e-13 on the eliminated system K_ff u_f = f_f
(Eq. linelastsoln); a direct factorisation of this 3D mesh is too large for a bounded run.
The file records the compliance J = f^T u (Section 2.3), the oracle-recomputed true relative
residual of that solution, and u at 64 seeded DOF samples.

Only oracle/ and the seeded input generators are called. Run from the repository root:
    python tests/golden/make_cant96x48x48.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fem, hatfilter  # noqa: E402
from paper_2004_05756_gb300 import workloads as w  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cant96x48x48_fp64.txt")


def main():
    p = w.cantilever_3d(96, 48, 48, rmin=2.0)
    psi = w.design_field(p, 0)
    rho = hatfilter.filter_fwd(p, psi)
    t0 = time.time()
    U, its = fem.solve_cg(p, rho, rtol=1e-13, maxit=400000)
    u = U[:, 0]
    f = p.F[:, 0]
    r = f - fem.apply_K_ebe(p, rho, u)
    r[fem.fixed_dofs(p)] = 0.0
    relres = float(np.linalg.norm(r) / np.linalg.norm(f))
    J = fem.compliance(p, u)
    free = fem.free_dofs(p)
    idx = np.sort(np.random.default_rng(96).choice(free, 64, replace=False))
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle state solve, cantilever 96x48x48 H8 (698691 DOFs), psi = design_field(p, 0),\n")
        fh.write("# rho = linear filter (radius 2); oracle Jacobi-PCG (fem.solve_cg) to rtol 1e-13.\n")
        fh.write("# Written by tests/golden/make_cant96x48x48.py (oracle only).\n")
        fh.write(f"cg_iterations {its}\n")
        fh.write(f"true_relres {relres:.17e}\n")
        fh.write(f"J {J:.17e}\n")
        fh.write(f"u_norm {np.linalg.norm(u):.17e}\n")
        for i in idx:
            fh.write(f"u {int(i)} {u[i]:.17e}\n")
    print(f"J={J:.17e} iters={its} relres={relres:.3e} {time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()
