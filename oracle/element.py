"""Unit-density element stiffness matrices K_e for bilinear Q4 and trilinear H8 elements.

Section 2.1 (Eq. linelast-res1): K(rho) = sum_e alpha(rho_e) P_e K_e P_e^T with one K_e,
identical for all elements because they are all unit squares (cubes). The paper never
states E, nu or the stress state; the benchmark's reading is E = 1, nu given, plane stress
with unit thickness in 2D, isotropic 3D elasticity.

K_e = integral over the unit element of B^T D B, evaluated with 2-point Gauss quadrature
per direction (exact for Q1 on a unit square / cube: the integrand is at most quadratic
in each coordinate).

Local node order: counter-clockwise from (0,0) on the face z = 0, i.e.
(0,0), (1,0), (1,1), (0,1); in 3D the same four on z = 0 followed by the same on z = 1.
Local DOF = dim * local_node + component.
"""
from __future__ import annotations

import itertools

import numpy as np

LOCAL_NODES_2D = np.array([(0, 0), (1, 0), (1, 1), (0, 1)], dtype=float)
LOCAL_NODES_3D = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                           (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)], dtype=float)

_G = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))  # Gauss points on [0, 1]


def d_plane_stress(E: float, nu: float) -> np.ndarray:
    """Plane-stress constitutive matrix, Voigt order (xx, yy, xy with engineering shear)."""
    return E / (1.0 - nu * nu) * np.array([[1.0, nu, 0.0],
                                           [nu, 1.0, 0.0],
                                           [0.0, 0.0, (1.0 - nu) / 2.0]])


def d_isotropic_3d(E: float, nu: float) -> np.ndarray:
    """Isotropic 3D constitutive matrix from Lame parameters, Voigt order
    (xx, yy, zz, xy, yz, zx) with engineering shears."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def _grad_shape(local_nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Gradients of the Q1 shape functions N_a(x) = prod_d (x_d if a_d == 1 else 1 - x_d)
    at the point x; returns (n_nodes, dim)."""
    n, dim = local_nodes.shape
    g = np.zeros((n, dim))
    for a in range(n):
        for d in range(dim):
            val = 1.0
            for dd in range(dim):
                corner = local_nodes[a, dd]
                if dd == d:
                    val *= 1.0 if corner == 1 else -1.0
                else:
                    val *= x[dd] if corner == 1 else (1.0 - x[dd])
            g[a, d] = val
    return g


def strain_matrix(local_nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Small-strain B matrix (Voigt rows) at point x."""
    n, dim = local_nodes.shape
    dN = _grad_shape(local_nodes, x)
    if dim == 2:
        B = np.zeros((3, 2 * n))
        for a in range(n):
            B[0, 2 * a] = dN[a, 0]
            B[1, 2 * a + 1] = dN[a, 1]
            B[2, 2 * a] = dN[a, 1]
            B[2, 2 * a + 1] = dN[a, 0]
        return B
    B = np.zeros((6, 3 * n))
    for a in range(n):
        c = 3 * a
        B[0, c] = dN[a, 0]
        B[1, c + 1] = dN[a, 1]
        B[2, c + 2] = dN[a, 2]
        B[3, c] = dN[a, 1]
        B[3, c + 1] = dN[a, 0]
        B[4, c + 1] = dN[a, 2]
        B[4, c + 2] = dN[a, 1]
        B[5, c] = dN[a, 2]
        B[5, c + 2] = dN[a, 0]
    return B


def ke_q4(nu: float, E: float = 1.0) -> np.ndarray:
    """8x8 plane-stress Q4 stiffness of a unit square (unit thickness)."""
    D = d_plane_stress(E, nu)
    K = np.zeros((8, 8))
    for gx, gy in itertools.product(_G, _G):
        B = strain_matrix(LOCAL_NODES_2D, np.array([gx, gy]))
        K += 0.25 * B.T @ D @ B
    return K


def ke_h8(nu: float, E: float = 1.0) -> np.ndarray:
    """24x24 isotropic H8 stiffness of a unit cube."""
    D = d_isotropic_3d(E, nu)
    K = np.zeros((24, 24))
    for gx, gy, gz in itertools.product(_G, _G, _G):
        B = strain_matrix(LOCAL_NODES_3D, np.array([gx, gy, gz]))
        K += 0.125 * B.T @ D @ B
    return K


def ke(dim: int, nu: float) -> np.ndarray:
    return ke_q4(nu) if dim == 2 else ke_h8(nu)
