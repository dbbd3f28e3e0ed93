"""Helmholtz density filter (Section 2.2, Eq. helm-soln .. cdens-star) and its adjoint, in
plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The filter maps the element densities psi to element densities rho in three steps:
  1. load vector   b(psi) = sum_e psi_e A_e b_e,  b_e[i] = integral of N_i over the element
                   (Eq. helm-res1; unit elements: 1/4 per node in 2D, 1/8 in 3D);
  2. nodal field   phi = H^-1 b,  H = sum_e A_e H_e A_e^T,
                   H_e = r^2 integral grad N_i . grad N_j + integral N_i N_j
                   (the finite-element Helmholtz equation -r^2 Lap phi + phi = psi with
                   homogeneous Neumann conditions, Eq. helm-soln, helm-res0);
  3. averaging     rho_e = (1 / N_v^e) sum of phi over the element's nodes (Eq. phitorho).
H_e is integrated by 2-point Gauss quadrature per direction (exact for Q1); H is assembled as
a scipy.sparse matrix and solved by SuperLU. The adjoint g = (d rho / d psi)^T v is written out
from the same three steps in reverse: w = (averaging)^T v, z = H^-T w, g_e = b_e^T A_e^T z.

Reading (one line of the design notes): the paper writes r = 2 sqrt(3) R for the filter radius
R; the cited reference relates a cone-filter radius R to the Helmholtz length r = R / (2 sqrt 3).
The functions here take r itself.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _gauss_q1(dim: int):
    """Shape functions and gradients of the unit Q1 element at the 2^dim Gauss points, with the
    local node order (x fastest, counter-clockwise in 2D faces: 00, 10, 11, 01, then the top
    face in 3D)."""
    corners2 = [(0, 0), (1, 0), (1, 1), (0, 1)]
    corners = corners2 if dim == 2 else [c + (0,) for c in corners2] + [c + (1,) for c in corners2]
    g = [0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)]
    pts = list(itertools.product(g, repeat=dim))
    N = np.zeros((len(pts), len(corners)))
    dN = np.zeros((len(pts), len(corners), dim))
    for q, x in enumerate(pts):
        for a, c in enumerate(corners):
            f = [x[d] if c[d] else 1.0 - x[d] for d in range(dim)]
            N[q, a] = np.prod(f)
            for d in range(dim):
                df = [(1.0 if c[dd] else -1.0) if dd == d else f[dd] for dd in range(dim)]
                dN[q, a, d] = np.prod(df)
    w = 1.0 / len(pts)  # unit element volume split over equal Gauss weights
    return N, dN, w


def element_matrices(dim: int, r: float):
    """H_e (stiffness r^2 + mass) and b_e of the unit Q1 element."""
    N, dN, w = _gauss_q1(dim)
    K = w * np.einsum("qad,qbd->ab", dN, dN)
    M = w * np.einsum("qa,qb->ab", N, N)
    b = w * N.sum(axis=0)
    return r * r * K + M, b


def element_nodes(p) -> np.ndarray:
    """Global node indices of every element in the local order of _gauss_q1 (N_e x 2^dim)."""
    nnx, nny = p.nx + 1, p.ny + 1
    if p.dim == 2:
        jj, ii = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
        n0 = (ii + nnx * jj).ravel()
        return np.stack([n0, n0 + 1, n0 + 1 + nnx, n0 + nnx], axis=1)
    kk, jj, ii = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    n0 = (ii + nnx * (jj + nny * kk)).ravel()
    face = [n0, n0 + 1, n0 + 1 + nnx, n0 + nnx]
    up = nnx * nny
    return np.stack(face + [f + up for f in face], axis=1)


def operators(p, r: float):
    """The assembled H (N_v x N_v), the load map B (N_v x N_e: b = B psi) and the averaging
    map A (N_e x N_v: rho = A phi), all scipy.sparse."""
    He, be = element_matrices(p.dim, r)
    en = element_nodes(p)
    nv = p.nnodes
    nloc = en.shape[1]
    rows = np.repeat(en, nloc, axis=1).ravel()
    cols = np.tile(en, (1, nloc)).ravel()
    vals = np.tile(He.ravel(), p.nel)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(nv, nv))
    e_idx = np.repeat(np.arange(p.nel), nloc)
    B = sp.csr_matrix((np.tile(be, p.nel), (en.ravel(), e_idx)), shape=(nv, p.nel))
    A = sp.csr_matrix((np.full(p.nel * nloc, 1.0 / nloc), (e_idx, en.ravel())), shape=(p.nel, nv))
    return H, B, A


def filter_fwd(p, psi: np.ndarray, r: float) -> np.ndarray:
    """rho = A H^-1 B psi (Eq. cdens-star)."""
    H, B, A = operators(p, r)
    phi = spla.spsolve(H.tocsc(), B @ np.asarray(psi, float))
    return A @ phi


def filter_adj(p, v: np.ndarray, r: float) -> np.ndarray:
    """g = (d rho / d psi)^T v = B^T H^-T A^T v: the adjoint of the three steps, each transposed
    explicitly (H^-T solved with H^T)."""
    H, B, A = operators(p, r)
    z = spla.spsolve(H.T.tocsc(), A.T @ np.asarray(v, float))
    return B.T @ z


def default_length(rmin: float) -> float:
    """The Helmholtz length equivalent to a cone filter of radius rmin: rmin / (2 sqrt 3)."""
    return rmin / (2.0 * math.sqrt(3.0))
