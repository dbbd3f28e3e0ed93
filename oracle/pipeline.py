"""Design evaluations composed from the oracle's steps (Section 2.5 for the HDM map,
Section 3.4 for the ROM map, Remark topopt_compl for the compliance gradient).

HDM eval:  psi -> rho = filter(psi) -> u = K(rho)^{-1} f -> J = f^T u,
           dc = -E'(rho) u_e^T K_e u_e, dpsi = filter^T(dc).
ROM eval:  psi -> rho -> H(rho), b -> y -> J_k = b^T y, u_k = Phi y, ||f - K u_k||,
           and the same gradient formula evaluated with u_k (lambda_k = u_k for compliance,
           Section 3.2).
"""
from __future__ import annotations

import numpy as np

from . import fem, hatfilter, rom


def hdm_eval(p, psi: np.ndarray, filtered: bool = True, direct: bool = True) -> dict:
    rho = hatfilter.filter_fwd(p, psi) if filtered else np.asarray(psi, float)
    if direct:
        U = fem.solve(p, rho)
        its = 0
    else:
        U, its = fem.solve_cg(p, rho)
    J = fem.compliance(p, U)
    dc = fem.compliance_grad_rho(p, rho, U)
    dpsi = hatfilter.filter_adj(p, dc) if filtered else dc
    return dict(rho=rho, U=U, J=J, dc=dc, dpsi=dpsi, cg_iters=its)


def rom_eval_full(p, psi: np.ndarray, Phi: np.ndarray, filtered: bool = True) -> dict:
    rho = hatfilter.filter_fwd(p, psi) if filtered else np.asarray(psi, float)
    f = p.F[:, 0]
    out = rom.rom_eval(p, rho, Phi, f)
    dc = fem.compliance_grad_rho(p, rho, out["uk"])
    out.update(rho=rho, dc=dc, dpsi=hatfilter.filter_adj(p, dc) if filtered else dc)
    return out
