"""Tensor-core projection (tcgen05 kind::tf32 on an exact hi/lo split of the FP32 operands)
of the FP32 forms of topo_rom_solve, against the FP64 oracle H = Phi^T K(rho) Phi (Eq. hatkbm).

H is read back through its Cholesky factor with the reduced refinement switched off
(TOPO_PARAM_ROM_REFINE = 0), so these tests see the unrefined reduced-precision projection;
the refined J_k is checked at the 1e-6 compliance target in test_gpu_parity. Tolerance
2e-5 max-normalised: FP32 applies (unit roundoff 6e-8 over 18 (Q4) / 81 (H8) stencil terms per
row), the split products (about 2^-20 relative each) and FP32 accumulation inside 256-row
segments; the SIMT FP32 contraction (TOPO_PARAM_ROM_TENSOR = 0) meets the same bound.

Shapes: k = 1 ... 100 (one to four 64 x 64 output tiles), N from 8 to 698,691 DOFs with ragged
tails (N mod 32 != 0), and the 96x48x48 H8 cantilever at k = 64 on sampled columns."""
import numpy as np
import pytest

from oracle import fem, hatfilter
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _basis(p, k, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((p.ndof, k)))
    Q[p.fixed == 1] = 0.0
    return Q


def _H_unrefined(torch, p, rho, Phi, prec, tensor):
    from paper_2004_05756_gb300.native import TOPO_PARAM_ROM_REFINE, TOPO_PARAM_ROM_TENSOR, Topo
    T = Topo(p)
    T.topo_set_param(TOPO_PARAM_ROM_REFINE, 0)
    T.topo_set_param(TOPO_PARAM_ROM_TENSOR, tensor)
    k = Phi.shape[1]
    f64 = dict(dtype=torch.float64, device="cuda")
    Hw = torch.zeros(k * k, **f64)
    y = torch.zeros(k, **f64)
    Jk = torch.zeros(1, **f64)
    b = torch.ones(k, **f64)
    T.topo_rom_solve(dev(rho), cols(Phi), k, b, Hw, y, Jk, prec)
    T.topo_check()
    L = Hw.cpu().numpy().reshape(k, k)
    T.close()
    return L @ L.T


CASES = {
    "q4_1x1_k3": (lambda: w.mbb_2d(1, 1), 3),
    "q4_37x13_k1": (lambda: w.mbb_2d(37, 13), 1),
    "q4_60x20_k16": (lambda: w.mbb_2d(60, 20), 16),
    "q4_600x200_k64": (lambda: w.mbb_2d(600, 200), 64),
    "h8_11x9x6_k65": (lambda: w.cantilever_3d(11, 9, 6), 65),
    "h8_24x12x12_k100": (lambda: w.cantilever_3d(24, 12, 12), 100),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp32_bf16ke"])
def test_tensor_projection_matches_oracle(torch, case, prec):
    mk, k = CASES[case]
    p = mk()
    rho = hatfilter.filter_fwd(p, w.design_field(p, 0))
    Phi = _basis(p, k, 11)
    Href = Phi.T @ fem.apply_K(p, rho, Phi)
    Href = 0.5 * (Href + Href.T)
    s = np.abs(Href).max()
    Ht = _H_unrefined(torch, p, rho, Phi, prec, 1)
    Hs = _H_unrefined(torch, p, rho, Phi, prec, 0)
    et = np.abs(Ht - Href).max() / s
    es = np.abs(Hs - Href).max() / s
    assert et < TOL, (case, prec, et, es)
    assert es < TOL, (case, prec, et, es)


def test_tensor_projection_full_size_3d_sampled(torch):
    """96x48x48 H8 cantilever (698,691 DOFs), k = 64, in the launch configuration of the
    benchmark: three columns of H from the oracle's element-by-element product."""
    p = w.cantilever_3d(96, 48, 48)
    rho = hatfilter.filter_fwd(p, w.design_field(p, 0))
    Phi = _basis(p, 64, 5)
    Ht = _H_unrefined(torch, p, rho, Phi, "fp32", 1)
    J = [0, 31, 63]
    Href = Phi.T @ fem.apply_K_ebe(p, rho, Phi[:, J])
    assert np.abs(Ht[:, J] - Href).max() < TOL * np.abs(Href).max()
