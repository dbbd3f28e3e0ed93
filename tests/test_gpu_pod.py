"""POD of a snapshot block (topo_rom_pod, Section 4.2 Eq. rob-optim) through the C ABI against
numpy's SVD: singular values, the subspace of the leading vectors (where a gap separates it),
orthonormality, the left-out column and the appended vector, and the zero vectors of singular
values at the Gram matrix's rounding level."""
import numpy as np
import pytest

from oracle import rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import dev, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _block(N, svals, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(N, len(svals))))
    W, _ = np.linalg.qr(rng.normal(size=(len(svals), len(svals))))
    return Q @ np.diag(svals) @ W.T  # N x m with the given singular values


@pytest.mark.parametrize("m,n,skip", [(1, 1, -1), (5, 3, -1), (8, 7, -1), (8, 4, 2), (17, 10, 16), (64, 40, 0)])
def test_pod_matches_svd(torch, m, n, skip):
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(37, 13)
    T = Topo(p)
    N = p.ndof
    svals = np.geomspace(1e3, 1e-2, m)
    U = _block(N, svals, m + n)
    keep = [j for j in range(m) if j != skip]
    append = np.random.default_rng(1).normal(size=N)
    Ud = dev(U.T.copy())
    Pod = th.zeros((n + 1, N), dtype=th.float64, device="cuda")
    sig = th.zeros(m, dtype=th.float64, device="cuda")
    T.topo_rom_pod(Ud, n, Pod, sig, skip=skip, append=dev(append))
    T.topo_check()
    P = Pod.cpu().numpy()
    Po, so = rom.pod(U[:, keep], n)
    s = sig.cpu().numpy()[:len(keep)]
    # through the Gram matrix a singular value carries an error of about eps sigma_max^2 / sigma_i
    assert np.all(np.abs(s - so) <= 1e-10 * so + 50 * 2.2e-16 * so[0] ** 2 / so)
    eps = 2.2e-16
    # orthonormality and the leading subspace, to the Gram route's bounds: eps sigma_max^2 /
    # (sigma_i sigma_j), and eps sigma_max^2 / (sigma_n (sigma_n - sigma_n+1)) for the subspace
    G = P[:n] @ P[:n].T
    tol = 50 * eps * so[0] ** 2 / np.outer(so[:n], so[:n]) + 1e-13
    assert np.all(np.abs(G - np.eye(n)) <= tol)
    gap = so[n - 1] - (so[n] if n < len(so) else 0.0)
    assert np.max(np.abs(P[:n].T @ (P[:n] @ Po) - Po)) <= 50 * eps * so[0] ** 2 / (so[n - 1] * gap) + 1e-12
    assert np.array_equal(P[n], append)


def test_pod_rank_deficient_gives_zero_vectors(torch):
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(20, 8)
    T = Topo(p)
    rng = np.random.default_rng(4)
    A = rng.normal(size=(p.ndof, 2))
    U = np.column_stack([A, A @ [1.0, 2.0], A[:, 0] * 3.0])  # rank 2 of 4 columns
    Pod = th.zeros((4, p.ndof), dtype=th.float64, device="cuda")
    sig = th.zeros(4, dtype=th.float64, device="cuda")
    T.topo_rom_pod(dev(U.T.copy()), 4, Pod, sig)
    P = Pod.cpu().numpy()
    assert np.allclose(P[:2] @ P[:2].T, np.eye(2), atol=1e-10)
    assert not P[2:].any()
    assert sig.cpu().numpy()[2] < 1e-6 * sig.cpu().numpy()[0]


def test_pod_invalid_arguments(torch):
    import torch as th
    from paper_2004_05756_gb300.native import Topo, TopoError
    p = w.mbb_2d(8, 4)
    T = Topo(p)
    U = th.zeros((3, p.ndof), dtype=th.float64, device="cuda")
    Pod = th.zeros((4, p.ndof), dtype=th.float64, device="cuda")
    sig = th.zeros(3, dtype=th.float64, device="cuda")
    for kw in (dict(n=4), dict(n=3, skip=1), dict(n=1, skip=3), dict(n=-1)):
        with pytest.raises(TopoError):
            T.topo_rom_pod(U, kw.pop("n"), Pod, sig, **kw)
