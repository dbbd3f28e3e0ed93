"""topo_rom_build's basis (Section 3.1: Phi spans the snapshots, the rank rule of R8) from its
one-launch CGS2, at the edges of that kernel: repeated and zero snapshot columns, an all-zero
block, the snapshots overwritten in place, more columns than one 16-column pass of its dot
products, and more snapshot columns than free DOFs. Each case against the oracle's Householder
basis (the same rank rule): k, orthonormality, the projector and b = Phi^T f."""
import numpy as np
import pytest

from oracle import rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, host_cols, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _build(T, p, U, in_place=False):
    import torch as th
    m = U.shape[1]
    Ud = cols(U)
    Phi = Ud if in_place else th.zeros_like(Ud)
    b = th.zeros(m, dtype=th.float64, device="cuda")
    f = p.F[:, 0]
    k = T.topo_rom_build(dev(np.full(p.nel, 0.5)), Ud, Phi, None, b, dev(f))
    T.topo_check()
    return k, host_cols(Phi)[:, :k], b.cpu().numpy()[:k]


def _check(p, U, k, P, b):
    Po = rom.basis(U)
    assert k == Po.shape[1]
    if k == 0:
        return
    assert np.abs(P.T @ P - np.eye(k)).max() < 1e-12
    x = np.random.default_rng(3).standard_normal(p.ndof)
    ref = Po @ (Po.T @ x)
    assert np.linalg.norm(P @ (P.T @ x) - ref) <= 1e-10 * np.linalg.norm(ref)
    f = p.F[:, 0]
    assert np.abs(b - P.T @ f).max() <= 1e-13 * np.linalg.norm(f)


def _random_cols(p, m, seed):
    U = np.random.default_rng(seed).standard_normal((p.ndof, m))
    U[p.fixed == 1] = 0.0
    return U


def test_repeated_and_zero_columns(torch):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(37, 13)
    T = Topo(p)
    R = _random_cols(p, 3, 1)
    U = np.column_stack([R[:, 0], R[:, 1], R[:, 0], np.zeros(p.ndof), R[:, 2], 2.0 * R[:, 1], R[:, 0] + R[:, 2]])
    k, P, b = _build(T, p, U)
    assert k == 3
    _check(p, U, k, P, b)


def test_all_zero_block(torch):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(20, 10)
    T = Topo(p)
    k, _, _ = _build(T, p, np.zeros((p.ndof, 5)))
    assert k == 0


def test_in_place_equals_separate_output(torch):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(37, 13)
    T = Topo(p)
    R = _random_cols(p, 4, 2)
    U = np.column_stack([R[:, 0], R[:, 0], R[:, 1], R[:, 2], R[:, 1] - R[:, 2], R[:, 3]])
    k1, P1, b1 = _build(T, p, U)
    k2, P2, b2 = _build(T, p, U, in_place=True)
    assert k1 == k2 == 4
    assert np.array_equal(P1, P2) and np.array_equal(b1, b2)
    _check(p, U, k2, P2, b2)


@pytest.mark.parametrize("m", [17, 40, 128])
def test_wide_bases(torch, m):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(60, 20)
    T = Topo(p)
    U = _random_cols(p, m, m)
    k, P, b = _build(T, p, U)
    assert k == m
    _check(p, U, k, P, b)


def test_more_columns_than_free_dofs(torch):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(4, 3)
    T = Topo(p)
    nfree = int((p.fixed == 0).sum())
    U = _random_cols(p, nfree + 9, 5)
    k, P, b = _build(T, p, U)
    assert k == nfree
    _check(p, U, k, P, b)
