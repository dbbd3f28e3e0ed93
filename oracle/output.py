"""General linear outputs j(u) = l^T u (Section 2.3-2.4, Section 3.2-3.3) in plain FP64: the
adjoint solve, the adjoint-based gradient and the Galerkin ROM of the adjoint.

TEST INFRASTRUCTURE ONLY (see the package docstring).

HDM (Eq. pap_sensitivity, Eq. linelast-adj1; dj/drho = 0 for a linear output):
    K(rho) u = f,  K(rho)^T lambda = l,  J = l^T u,
    dJ/drho_e = -alpha'(rho_e) u_e^T K_e lambda_e,  dJ/dpsi = (drho/dpsi)^T dJ/drho.
ROM (Section 3.1 and 3.2), on a basis Phi:
    H = Phi^T K Phi,  y = H^-1 Phi^T f,  z = H^-1 Phi^T l,  u_k = Phi y,  lambda_k = Phi z,
    J_k = l^T u_k, primal residual r = K u_k - f, adjoint residual r_adj = K lambda_k - l,
    dJ_k/drho_e = -alpha'(rho_e) (u_k)_e^T K_e (lambda_k)_e.
For l = f every quantity is the compliance one (lambda = u, Remark topopt_compl).
"""
from __future__ import annotations

import numpy as np

from . import element, fem, hatfilter, rom


def mixed_grad_rho(p, rho: np.ndarray, U: np.ndarray, Lam: np.ndarray) -> np.ndarray:
    """-alpha'(rho_e) sum_c u_{c,e}^T K_e lambda_{c,e} (the element loop of Eq. pap_sensitivity)."""
    Ke = element.ke(p.dim, p.nu)
    ed = fem.edof(p)
    U2 = U[:, None] if U.ndim == 1 else U
    L2 = Lam[:, None] if Lam.ndim == 1 else Lam
    ce = np.zeros(p.nel)
    for c in range(U2.shape[1]):
        ue, le = U2[ed, c], L2[ed, c]
        ce += np.einsum("ei,ij,ej->e", ue, Ke, le)
    return -fem.dyoung(rho, p.E0, p.Emin, p.penal) * ce


def hdm_output(p, psi: np.ndarray, l: np.ndarray, filtered: bool = True) -> dict:
    rho = hatfilter.filter_fwd(p, psi) if filtered else np.asarray(psi, float)
    u = fem.solve(p, rho, p.F[:, :1])[:, 0]
    lam = fem.solve(p, rho, np.asarray(l, float)[:, None])[:, 0]  # K symmetric: K^T = K
    dc = mixed_grad_rho(p, rho, u, lam)
    return dict(rho=rho, u=u, lam=lam, J=float(l @ u), dc=dc,
                dpsi=hatfilter.filter_adj(p, dc) if filtered else dc)


def rom_output(p, psi: np.ndarray, Phi: np.ndarray, l: np.ndarray, filtered: bool = True) -> dict:
    rho = hatfilter.filter_fwd(p, psi) if filtered else np.asarray(psi, float)
    f = p.F[:, 0]
    H, bf = rom.project(p, rho, Phi, f)
    bl = Phi.T @ l
    y = rom.solve_reduced(H, bf)
    z = rom.solve_reduced(H, bl)
    uk, lk = Phi @ y, Phi @ z
    r = -rom.residual(p, rho, uk, f)      # K u_k - f on the free DOFs
    ra = -rom.residual(p, rho, lk, l)     # K lambda_k - l on the free DOFs
    dc = mixed_grad_rho(p, rho, uk, lk)
    return dict(rho=rho, uk=uk, lk=lk, Jk=float(l @ uk), r=r, r_adj=ra, resnorm=float(np.linalg.norm(r)),
                adj_resnorm=float(np.linalg.norm(ra)), dc=dc,
                dpsi=hatfilter.filter_adj(p, dc) if filtered else dc)


def point_output(p, node: int, comp: int = 1) -> np.ndarray:
    """l selecting one displacement component at one node (a compliant-mechanism-type output)."""
    l = np.zeros(p.ndof)
    l[p.dim * node + comp] = 1.0
    return l
