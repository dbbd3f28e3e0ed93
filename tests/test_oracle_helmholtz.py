"""Pins of the oracle's Helmholtz filter (Section 2.2): the element matrices against their closed
forms, the assembly against an element-by-element loop, the two conservation properties the
paper relies on (a constant field is reproduced; the filter preserves volume, the property that
lets the volume constraint act on psi), the adjoint identity, and smoothing."""
import numpy as np
import pytest

from oracle import helmholtz
from paper_2004_05756_gb300 import workloads as w


def test_q4_element_matrices_closed_form():
    He, be = helmholtz.element_matrices(2, 1.0)
    M = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0
    K = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    assert np.allclose(He, K + M, atol=1e-15)
    He2, _ = helmholtz.element_matrices(2, 0.5)
    assert np.allclose(He2, 0.25 * K + M, atol=1e-15)
    assert np.allclose(be, 0.25)


def test_h8_element_matrices_properties():
    He0, be = helmholtz.element_matrices(3, 0.0)  # the mass matrix
    assert np.isclose(He0.sum(), 1.0) and np.allclose(be, 0.125)
    assert np.isclose(He0[0, 0], 8.0 / 216.0) and np.isclose(He0[0, 6], 1.0 / 216.0)  # opposite corners
    He1, _ = helmholtz.element_matrices(3, 1.0)
    K = He1 - He0
    assert np.allclose(K @ np.ones(8), 0.0, atol=1e-15)  # constants are in the stiffness null space
    assert np.isclose(K[0, 0], 1.0 / 3.0)


def test_assembly_matches_element_loop():
    p = w.mbb_2d(3, 2)
    r = 0.7
    H, B, A = helmholtz.operators(p, r)
    He, be = helmholtz.element_matrices(2, r)
    Hd = np.zeros((p.nnodes, p.nnodes))
    Bd = np.zeros((p.nnodes, p.nel))
    Ad = np.zeros((p.nel, p.nnodes))
    for e, nodes in enumerate(helmholtz.element_nodes(p)):
        for a, na in enumerate(nodes):
            Bd[na, e] += be[a]
            Ad[e, na] += 0.25
            for c, nc in enumerate(nodes):
                Hd[na, nc] += He[a, c]
    assert np.allclose(H.toarray(), Hd) and np.allclose(B.toarray(), Bd) and np.allclose(A.toarray(), Ad)
    # element 0 of the 3 x 2 mesh has nodes 0, 1, 5, 4
    assert list(helmholtz.element_nodes(p)[0]) == [0, 1, 5, 4]


@pytest.mark.parametrize("mesh", [(2, 9, 5, 1), (3, 4, 3, 3)])
def test_constants_and_volume(mesh):
    dim, nx, ny, nz = mesh
    p = w.mbb_2d(nx, ny) if dim == 2 else w.cantilever_3d(nx, ny, nz)
    r = 1.3
    c = 0.37
    assert np.allclose(helmholtz.filter_fwd(p, np.full(p.nel, c), r), c, atol=1e-14)
    psi = np.random.default_rng(1).uniform(0, 1, p.nel)
    rho = helmholtz.filter_fwd(p, psi, r)
    assert rho.sum() == pytest.approx(psi.sum(), rel=1e-13)  # volume preservation (Section 2.2)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_identity_and_self_adjointness(dim):
    p = w.mbb_2d(11, 6) if dim == 2 else w.cantilever_3d(5, 4, 3)
    rng = np.random.default_rng(2)
    psi, v = rng.normal(size=p.nel), rng.normal(size=p.nel)
    r = 0.9
    lhs = helmholtz.filter_fwd(p, psi, r) @ v
    rhs = psi @ helmholtz.filter_adj(p, v, r)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # with unit elements B = A^T and H = H^T, so the filter is its own adjoint
    assert np.allclose(helmholtz.filter_adj(p, v, r), helmholtz.filter_fwd(p, v, r), atol=1e-13)


def test_smoothing_and_zero_length_limit():
    p = w.mbb_2d(16, 8)
    jj, ii = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
    chk = ((ii + jj) % 2).ravel().astype(float)
    for r, bound in ((0.5, 0.5), (2.0, 0.05)):
        rho = helmholtz.filter_fwd(p, chk, r)
        assert np.std(rho) < bound * np.std(chk)
    # a longer length smooths more
    assert np.std(helmholtz.filter_fwd(p, chk, 2.0)) < np.std(helmholtz.filter_fwd(p, chk, 0.5))
    assert helmholtz.default_length(1.5) == pytest.approx(1.5 / (2 * np.sqrt(3)))
