"""Galerkin reduced-order model, residual and error bounds, in plain FP64.

Section 3.1 (Eq. rom_soln, hatkbm, Jrom), Section 3.3 (residual, Theorem rom_primal_error,
the compliance form of Theorem rom_output_error), Section 4.2 (Eq. rob-optim: the basis is
an orthonormalisation of snapshots; for compliance the adjoint snapshots equal the primal
ones).

Everything here uses the oracle's own assembled operator (fem.apply_K), numpy's
Householder QR and scipy's Cholesky.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import fem


def basis(U: np.ndarray, drop_tol: float = 1e-10) -> np.ndarray:
    """Orthonormal basis of the snapshot columns (Eq. rob-optim's Gram-Schmidt step,
    computed here with Householder QR). A column is dropped when its component
    orthogonal to the columns kept before it has norm < drop_tol * max_j ||U_j||; the
    basis is then the Q factor of the kept columns."""
    U = np.asarray(U, dtype=float)
    scale = np.max(np.linalg.norm(U, axis=0)) if U.shape[1] else 0.0
    kept: list[int] = []
    for i in range(U.shape[1]):
        R = np.linalg.qr(U[:, kept + [i]], mode="r")
        if abs(R[-1, -1]) >= drop_tol * scale and scale > 0:
            kept.append(i)
    if not kept:
        return np.zeros((U.shape[0], 0))
    Q, _ = np.linalg.qr(U[:, kept])
    return Q


def pod(U: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """POD_n(U) of Section 4.2 (Eq. rob-optim): the first n left singular vectors of U (numpy's
    SVD) and all its singular values, descending."""
    Uu, s, _ = np.linalg.svd(np.asarray(U, dtype=float), full_matrices=False)
    return Uu[:, :n], s


def project(p, rho: np.ndarray, Phi: np.ndarray, f: np.ndarray):
    """H = Phi^T K(rho) Phi and b = Phi^T f (Eq. hatkbm, written as the plain product)."""
    W = fem.apply_K(p, rho, Phi)
    H = Phi.T @ W
    b = Phi.T @ f
    return H, b


def solve_reduced(H: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = H^{-1} b by Cholesky (H is SPD when Phi has full rank, Remark rom_wellposed)."""
    c = sla.cho_factor(H, lower=True)
    return sla.cho_solve(c, b)


def reconstruct(Phi: np.ndarray, y: np.ndarray) -> np.ndarray:
    return Phi @ y


def residual(p, rho: np.ndarray, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """r = f - K(rho) u restricted to the free DOFs (Section 3.3; Dirichlet DOFs are
    eliminated, so the returned vector is zero there). The paper's sign is K u - f;
    norms are sign-free."""
    r = f - fem.apply_K(p, rho, u)
    r[fem.fixed_dofs(p)] = 0.0
    return r


def rom_eval(p, rho: np.ndarray, Phi: np.ndarray, f: np.ndarray) -> dict:
    """One ROM design evaluation on a resident basis: H, b, y, J_k = b^T y, u_k = Phi y,
    the residual r = f - K u_k, ||r||_2 and ||r||_2 / ||f||_2."""
    H, b = project(p, rho, Phi, f)
    y = solve_reduced(H, b)
    uk = reconstruct(Phi, y)
    r = residual(p, rho, uk, f)
    nr = float(np.linalg.norm(r))
    return dict(H=H, b=b, y=y, Jk=float(b @ y), uk=uk, r=r, resnorm=nr,
                relres=nr / float(np.linalg.norm(f[fem.free_dofs(p)])))


def energy_norm(p, rho: np.ndarray, v: np.ndarray) -> float:
    return float(np.sqrt(v @ fem.apply_K(p, rho, v)))


def sigma_min_dense(p, rho: np.ndarray) -> float:
    """Smallest eigenvalue of the dense K_ff (tiny meshes only), for Theorem
    rom_primal_error and the compliance output bound."""
    K = fem.reduced_K(p, rho).toarray()
    return float(np.linalg.eigvalsh(K)[0])
