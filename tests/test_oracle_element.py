"""Pins for the oracle's element stiffness (Section 2.1): hand-derived closed forms,
exact symbolic integration (a different evaluation route than the oracle's Gauss
quadrature), and the invariants of a Q1 elasticity element."""
import os

import numpy as np
import pytest

from oracle import element

GOLD = os.path.join(os.path.dirname(__file__), "golden", "element_closed_forms.txt")


def _gold():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        el, key, v = line.split()
        out[(el, key)] = float(v)
    return out


def test_closed_forms():
    g = _gold()
    Kq = element.ke_q4(0.3)
    Kh = element.ke_h8(0.3)
    assert Kq[0, 0] == pytest.approx(g[("q4", "K00")], rel=1e-14)
    assert Kq[0, 1] == pytest.approx(g[("q4", "K01")], rel=1e-14)
    assert np.trace(Kq) == pytest.approx(g[("q4", "trace")], rel=1e-14)
    assert Kh[0, 0] == pytest.approx(g[("h8", "K00")], rel=1e-14)
    assert Kh[0, 1] == pytest.approx(g[("h8", "K01")], rel=1e-14)


def _rigid_modes(nodes):
    """Translations and infinitesimal rotations of the element's nodes."""
    n, dim = nodes.shape
    modes = []
    for c in range(dim):
        v = np.zeros((n, dim))
        v[:, c] = 1
        modes.append(v.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (2, 0)]
    for a, b in pairs:
        v = np.zeros((n, dim))
        v[:, a] = -nodes[:, b]
        v[:, b] = nodes[:, a]
        modes.append(v.ravel())
    return np.array(modes).T


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_invariants(dim, nu):
    K = element.ke(dim, nu)
    nodes = element.LOCAL_NODES_2D if dim == 2 else element.LOCAL_NODES_3D
    assert np.allclose(K, K.T, atol=1e-15)
    R = _rigid_modes(nodes)
    assert np.abs(K @ R).max() < 1e-14
    ev = np.linalg.eigvalsh(K)
    nrig = 3 if dim == 2 else 6
    assert np.all(ev[:nrig] < 1e-13) and np.all(ev[nrig:] > 1e-3)
    assert np.linalg.matrix_rank(K, tol=1e-10) == K.shape[0] - nrig


@pytest.mark.parametrize("dim", [2, 3])
def test_exact_symbolic_integration(dim):
    sympy = pytest.importorskip("sympy")
    nu = sympy.Rational(3, 10)
    X = sympy.symbols("x y z")[:dim]
    corners = [(0, 0), (1, 0), (1, 1), (0, 1)] if dim == 2 else \
        [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    N = []
    for c in corners:
        f = sympy.Integer(1)
        for d in range(dim):
            f *= X[d] if c[d] else (1 - X[d])
        N.append(f)
    nn = len(corners)
    if dim == 2:
        D = sympy.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
        B = sympy.zeros(3, 2 * nn)
        for a in range(nn):
            B[0, 2 * a] = sympy.diff(N[a], X[0])
            B[1, 2 * a + 1] = sympy.diff(N[a], X[1])
            B[2, 2 * a] = sympy.diff(N[a], X[1])
            B[2, 2 * a + 1] = sympy.diff(N[a], X[0])
    else:
        lam = nu / ((1 + nu) * (1 - 2 * nu))
        mu = 1 / (2 * (1 + nu))
        D = sympy.zeros(6, 6)
        for a in range(3):
            for b in range(3):
                D[a, b] = lam
            D[a, a] = lam + 2 * mu
            D[a + 3, a + 3] = mu
        B = sympy.zeros(6, 3 * nn)
        for a in range(nn):
            dx, dy, dz = (sympy.diff(N[a], X[d]) for d in range(3))
            c = 3 * a
            B[0, c], B[1, c + 1], B[2, c + 2] = dx, dy, dz
            B[3, c], B[3, c + 1] = dy, dx
            B[4, c + 1], B[4, c + 2] = dz, dy
            B[5, c], B[5, c + 2] = dz, dx
    integrand = B.T * D * B
    K = integrand
    for d in range(dim):
        K = K.applyfunc(lambda e, d=d: sympy.integrate(e, (X[d], 0, 1)))
    Kexact = np.array(K.evalf(30).tolist(), dtype=float)
    Ko = element.ke(dim, 0.3)
    assert np.abs(Ko - Kexact).max() < 1e-14 * np.abs(Kexact).max()
