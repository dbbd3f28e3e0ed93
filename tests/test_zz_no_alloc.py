"""The allocation-free reduced solve (topo_rom_solve_elem_noalloc) against the allocating one
(topo_rom_solve_elem), through the C ABI, on two calls in a row. Kept in a file collected last
so that a failure here does not stop the rest of the GPU suite."""
import numpy as np
import pytest

from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_solve():
    torch = require_cuda()
    from paper_2004_05756_gb300 import native
    p = w.mbb_2d(37, 13)
    T = native.Topo(p)
    rng = np.random.default_rng(21)
    k = 8
    Phi, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
    npair = k * (k + 1) // 2
    Hel = torch.zeros((p.nel + 1) * npair, dtype=torch.float64, device="cuda")
    T.topo_rom_elem(cols(Phi), k, Hel)
    b = dev(rng.standard_normal(k))
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row: the shared array keeps the previous contents
        rho = dev(rng.uniform(1e-3, 1.0, p.nel))
        Hw_a, y_a, J_a = z(k * k), z(k), z(1)
        Hw_b, y_b, J_b = z(k * k), z(k), z(1)
        T.topo_rom_solve_elem(rho, Hel, k, b, Hw_a, y_a, J_a)
        T.topo_rom_solve_elem_noalloc(rho, Hel, k, b, Hw_b, y_b, J_b)
        T.topo_check()
        ya, yb = y_a.cpu().numpy(), y_b.cpu().numpy()
        assert np.abs(yb - ya).max() <= 1e-12 * np.abs(ya).max(), call
        assert abs(J_b.item() - J_a.item()) <= 1e-12 * abs(J_a.item()), call
        assert np.abs(Hw_b.cpu().numpy() - Hw_a.cpu().numpy()).max() <= 1e-12 * np.abs(Hw_a.cpu().numpy()).max()


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = require_cuda()
    from paper_2004_05756_gb300 import native
    p = w.mbb_2d(2000, 600)  # 1.2 M elements: E(rho) alone needs 9.6 MB > 8 MiB
    T = native.Topo(p)
    k = 16
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = native.load().topo_rom_solve_elem_noalloc(T.h, x.data_ptr(), x.data_ptr(), k, x.data_ptr(), x.data_ptr(),
                                                   x.data_ptr(), x.data_ptr())
    assert st == native.TOPO_ERR_INVALID
    assert b"scratch" in native.load().topo_last_error(T.h)
