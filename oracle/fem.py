"""Full-order model (HDM): assembly, solve, compliance and its gradient, in plain FP64.

Section 2.1 (Eq. linelast-res1, linelastsoln, linelastU), Section 2.3 (compliance j_c),
Section 2.4 (Eq. pap_sensitivity, Remark topopt_compl) and Section 2.5 step 4-5.

Material law (the benchmark's form of alpha(rho) in Eq. linelast-res1):
    E(rho) = Emin + rho^p (E0 - Emin),  dE/drho = p rho^(p-1) (E0 - Emin).
The paper's own law alpha = rho_l + (1 - rho_l) rho^p is the case Emin = rho_l E0, E0 = 1.

Dirichlet DOFs are eliminated as in the paper (the remark after Eq. linelastU): the
oracle solves K_ff u_f = f_f. The library's operator convention keeps those DOFs in the
vectors with identity rows and columns; apply_K below restates that convention from the
eliminated operator: Y_f = K_ff V_f, Y_d = V_d.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import element


def edof(p) -> np.ndarray:
    """Global DOF numbers of each element in local order (N_e x ndof_e): the assembly
    operator P_e of Section 2.1 written as an index table."""
    dim = p.dim
    if dim == 2:
        ii, jj = np.meshgrid(np.arange(p.nx), np.arange(p.ny), indexing="xy")
        ii, jj = ii.ravel(), jj.ravel()  # element order e = i + nx j
        corners = [(0, 0), (1, 0), (1, 1), (0, 1)]
        nodes = [(ii + a) + (p.nx + 1) * (jj + b) for a, b in corners]
    else:
        kk, jj, ii = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
        nodes = [(ii + a) + (p.nx + 1) * ((jj + b) + (p.ny + 1) * (kk + c)) for a, b, c in corners]
    cols = []
    for n in nodes:
        for c in range(dim):
            cols.append(dim * n + c)
    return np.stack(cols, axis=1).astype(np.int64)


def young(rho: np.ndarray, E0: float, Emin: float, penal: float) -> np.ndarray:
    return Emin + rho ** penal * (E0 - Emin)


def dyoung(rho: np.ndarray, E0: float, Emin: float, penal: float) -> np.ndarray:
    return penal * rho ** (penal - 1.0) * (E0 - Emin)


def assemble_K(p, rho: np.ndarray) -> sp.csr_matrix:
    """Assembled K(rho) = sum_e E(rho_e) P_e K_e P_e^T without boundary conditions."""
    Ke = element.ke(p.dim, p.nu)
    ed = edof(p)
    E = young(rho, p.E0, p.Emin, p.penal)
    nd = ed.shape[1]
    rows = np.repeat(ed, nd, axis=1).ravel()
    cols = np.tile(ed, (1, nd)).ravel()
    vals = (E[:, None, None] * Ke[None, :, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(p.ndof, p.ndof)).tocsr()
    K.sum_duplicates()
    return K


def free_dofs(p) -> np.ndarray:
    return np.flatnonzero(p.fixed == 0)


def fixed_dofs(p) -> np.ndarray:
    return np.flatnonzero(p.fixed != 0)


def reduced_K(p, rho: np.ndarray) -> sp.csc_matrix:
    """K_ff: K(rho) with the Dirichlet rows and columns eliminated."""
    K = assemble_K(p, rho)
    f = free_dofs(p)
    return K[f][:, f].tocsc()


def apply_K(p, rho: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Operator convention of the library: Y_f = K_ff V_f and Y_d = V_d (N x m)."""
    V = np.asarray(V, dtype=float)
    one = V.ndim == 1
    V2 = V[:, None] if one else V
    f = free_dofs(p)
    d = fixed_dofs(p)
    Kff = reduced_K(p, rho)
    Y = np.zeros_like(V2)
    Y[f] = Kff @ V2[f]
    Y[d] = V2[d]
    return Y[:, 0] if one else Y


def apply_K_ebe(p, rho: np.ndarray, V: np.ndarray) -> np.ndarray:
    """The same operator as apply_K, element by element without assembly (Section 2.1):
    Y = sum_e E(rho_e) P_e K_e P_e^T V0 with V0 = V zeroed on the Dirichlet DOFs, then Y_d = V_d.
    For meshes whose assembled matrix is too large to build in seconds (N x m)."""
    V = np.asarray(V, dtype=float)
    one = V.ndim == 1
    V2 = (V[:, None] if one else V).copy()
    d = fixed_dofs(p)
    V0 = V2.copy()
    V0[d] = 0.0
    Ke = element.ke(p.dim, p.nu)
    ed = edof(p)
    E = young(rho, p.E0, p.Emin, p.penal)
    Y = np.zeros_like(V2)
    for j in range(V2.shape[1]):
        Ve = V0[ed, j]                         # N_e x ndof_e
        Ye = E[:, None] * (Ve @ Ke.T)          # E_e K_e v_e per element
        Y[:, j] = np.bincount(ed.ravel(), weights=Ye.ravel(), minlength=p.ndof)
    Y[d] = V2[d]
    return Y[:, 0] if one else Y


def jacobi_diag(p, rho: np.ndarray) -> np.ndarray:
    """diag(K) on free DOFs, 1 on Dirichlet DOFs (the Jacobi preconditioner)."""
    K = assemble_K(p, rho)
    dg = K.diagonal().copy()
    dg[fixed_dofs(p)] = 1.0
    return dg


def solve(p, rho: np.ndarray, F: np.ndarray | None = None) -> np.ndarray:
    """State solve u*(rho) of Eq. linelastsoln, by sparse LU (SuperLU) of K_ff, as in the
    paper's direct-solver route (Section 2.5, step 5). Returns N x nlc, zero on
    Dirichlet DOFs."""
    F = p.F if F is None else F
    F2 = F[:, None] if F.ndim == 1 else F
    f = free_dofs(p)
    lu = spla.splu(reduced_K(p, rho))
    U = np.zeros_like(F2, dtype=float)
    U[f] = lu.solve(np.ascontiguousarray(F2[f]))
    return U[:, 0] if F.ndim == 1 else U


def solve_cg(p, rho: np.ndarray, F: np.ndarray | None = None, rtol: float = 1e-13,
             maxit: int = 200000) -> tuple[np.ndarray, int]:
    """Jacobi-preconditioned CG on K_ff u_f = f_f with the assembled scipy matrix, for
    meshes where a direct factorisation is too large (3D). Plain textbook PCG, stopping
    when ||f - K u||_2 <= rtol ||f||_2. Returns (U, max iterations over load cases)."""
    F = p.F if F is None else F
    F2 = F[:, None] if F.ndim == 1 else F
    f = free_dofs(p)
    Kff = reduced_K(p, rho).tocsr()
    dinv = 1.0 / Kff.diagonal()
    U = np.zeros_like(F2, dtype=float)
    its = 0
    for c in range(F2.shape[1]):
        b = F2[f, c]
        x = np.zeros_like(b)
        r = b.copy()
        z = dinv * r
        d = z.copy()
        rz = r @ z
        nb = np.linalg.norm(b)
        it = 0
        while np.linalg.norm(r) > rtol * nb and it < maxit:
            q = Kff @ d
            a = rz / (d @ q)
            x += a * d
            r -= a * q
            z = dinv * r
            rz_new = r @ z
            d = z + (rz_new / rz) * d
            rz = rz_new
            it += 1
        U[f, c] = x
        its = max(its, it)
    return (U[:, 0] if F.ndim == 1 else U), its


def compliance(p, U: np.ndarray, F: np.ndarray | None = None) -> float:
    """j_c = f^T u (Section 2.3), summed over load cases."""
    F = p.F if F is None else F
    F2 = F.reshape(F.shape[0], -1)
    U2 = np.asarray(U).reshape(F2.shape[0], -1)
    if U2.shape != F2.shape:
        raise ValueError(f"compliance: U {U2.shape} and F {F2.shape} differ")
    return float(np.sum(F2 * U2))


def element_energy(p, U: np.ndarray) -> np.ndarray:
    """ce_e = sum over load cases of u_e^T K_e u_e (unit density)."""
    Ke = element.ke(p.dim, p.nu)
    ed = edof(p)
    U2 = U[:, None] if U.ndim == 1 else U
    ce = np.zeros(p.nel)
    for c in range(U2.shape[1]):
        ue = U2[ed, c]  # N_e x ndof_e
        ce += np.einsum("ei,ij,ej->e", ue, Ke, ue)
    return ce


def compliance_grad_rho(p, rho: np.ndarray, U: np.ndarray) -> np.ndarray:
    """dJ/drho_e = -E'(rho_e) u_e^T K_e u_e: Eq. pap_sensitivity with the compliance
    simplification lambda = u and dj/drho = 0 (Remark topopt_compl)."""
    return -dyoung(rho, p.E0, p.Emin, p.penal) * element_energy(p, U)
