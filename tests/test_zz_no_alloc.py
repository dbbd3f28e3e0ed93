"""The allocation-free reduced solve (topo_rom_solve_elem_noalloc) against the allocating one
(topo_rom_solve_elem), through the C ABI, on two calls in a row. Kept in a file collected last
so that a failure here does not stop the rest of the GPU suite.

Sizes cover both reduced-solve branches (the one-warp Cholesky for k <= 32 and the CTA
Cholesky for 32 < k <= 64), and a mesh whose scratch need sits just under the fixed array's
size, next to one just over it."""
import numpy as np
import pytest

from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 8 << 20  # the fixed device array of topo_rom_solve_elem_noalloc


def _need_bytes(nel, k, sms):
    """Scratch the entry point needs: a 256-byte flag block, E(rho) for N_e + 1 rows (rounded
    up to 256 bytes) and per-CTA partial sums of the packed k x k matrix (2 CTAs per SM)."""
    rows = nel + 1
    G = 2 * sms
    per = -(-rows // G)
    G = -(-rows // per)
    e_bytes = (rows * 8 + 255) & ~255
    return 256 + e_bytes + G * (k * (k + 1) // 2) * 8


def _compare(torch, T, p, k, rng, calls=2):
    Phi, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
    npair = k * (k + 1) // 2
    Hel = torch.zeros((p.nel + 1) * npair, dtype=torch.float64, device="cuda")
    T.topo_rom_elem(cols(Phi), k, Hel)
    del Phi
    b = dev(rng.standard_normal(k))
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")
    for call in range(calls):  # calls in a row: the shared array keeps the previous contents
        rho = dev(rng.uniform(1e-3, 1.0, p.nel))
        Hw_a, y_a, J_a = z(k * k), z(k), z(1)
        Hw_b, y_b, J_b = z(k * k), z(k), z(1)
        T.topo_rom_solve_elem(rho, Hel, k, b, Hw_a, y_a, J_a)
        T.topo_rom_solve_elem_noalloc(rho, Hel, k, b, Hw_b, y_b, J_b)
        T.topo_check()
        ya, yb = y_a.cpu().numpy(), y_b.cpu().numpy()
        assert np.abs(yb - ya).max() <= 1e-12 * np.abs(ya).max(), (k, call)
        assert abs(J_b.item() - J_a.item()) <= 1e-12 * abs(J_a.item()), (k, call)
        Ha, Hb = Hw_a.cpu().numpy(), Hw_b.cpu().numpy()
        assert np.abs(Hb - Ha).max() <= 1e-12 * np.abs(Ha).max(), (k, call)


@pytest.mark.parametrize("k", [8, 24, 40, 64])
def test_noalloc_matches_allocating_solve(k):
    torch = require_cuda()
    from paper_2004_05756_gb300 import native
    p = w.mbb_2d(37, 13)
    T = native.Topo(p)
    _compare(torch, T, p, k, np.random.default_rng(21 + k))


def test_noalloc_near_its_size_limit():
    """k = 64 on a mesh whose scratch need is within 2 % below the array's size: accepted and
    equal to the allocating solve; one element row more than fits is rejected."""
    torch = require_cuda()
    from paper_2004_05756_gb300 import native
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    k, nx = 64, 800
    ny = max(j for j in range(1, 2000) if _need_bytes(nx * j, k, sms) <= NOALLOC_BYTES)
    assert _need_bytes(nx * ny, k, sms) >= 0.98 * NOALLOC_BYTES
    p = w.mbb_2d(nx, ny)
    T = native.Topo(p)
    _compare(torch, T, p, k, np.random.default_rng(64), calls=1)
    T.close()
    big = w.mbb_2d(nx, ny + 1)
    assert _need_bytes(big.nel, k, sms) > NOALLOC_BYTES
    Tb = native.Topo(big)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = native.load().topo_rom_solve_elem_noalloc(Tb.h, x.data_ptr(), x.data_ptr(), k, x.data_ptr(), x.data_ptr(),
                                                   x.data_ptr(), x.data_ptr())
    assert st == native.TOPO_ERR_INVALID
    assert b"scratch" in native.load().topo_last_error(Tb.h)


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
