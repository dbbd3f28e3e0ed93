"""The FP64 stencil solve with the multigrid V-cycle preconditioner (the default), through the
C ABI, against the oracle's direct solve on the same seeded inputs.

Meshes cover odd and even node counts per direction (the coarsening keeps the last node), a
direction of one element (it stops coarsening), 2D and 3D, several load cases, every
smoothing degree and both ends of the single-CTA threshold (only the coarsest level on one
CTA; every coarse level on one CTA). The preconditioner changes the path, not the fixed point:
every case reaches rtol 1e-13 (or the reported FP64 floor) with compliance within 1e-10 of the
oracle."""
import numpy as np
import pytest

from oracle import fem, hatfilter
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, host_cols, require_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "q4_60x20": lambda: w.mbb_2d(60, 20),       # 61 x 21 nodes (odd, odd)
    "q4_37x13": lambda: w.mbb_2d(37, 13),       # 38 x 14 nodes (even, even)
    "q4_40x1": lambda: w.mbb_2d(40, 1),         # one element high
    "q4_130x41": lambda: w.mbb_2d(130, 41),     # several units per row and CTAs per level
    "h8_6x5x4": lambda: w.cantilever_3d(6, 5, 4),
    "h8_11x9x6": lambda: w.cantilever_3d(11, 9, 6),
    "h8_24x12x12": lambda: w.cantilever_3d(24, 12, 12),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _check(p, rho, U, info, ref, rtol=1e-13):
    """Compliance within 1e-10 of the oracle's, plus the first-order bound
    ||u|| (||r_gpu|| + ||r_oracle||) of two FP64 solutions that stop at a residual rounding floor
    (J - J_h = u^T r for compliance; the bound vanishes when both residuals are tiny)."""
    Jo, Uo = ref
    assert info["status"] == 0 and info["relres"] <= max(rtol, info["floor"]), info
    Ug = host_cols(U)
    for c in range(p.F.shape[1]):
        J = fem.compliance(p, Ug[:, c], p.F[:, c])
        r = p.F[:, c] - fem.apply_K(p, rho, Ug[:, c])
        r[fem.fixed_dofs(p)] = 0
        ro = p.F[:, c] - fem.apply_K(p, rho, Uo[:, c])
        ro[fem.fixed_dofs(p)] = 0
        bound = np.linalg.norm(Uo[:, c]) * (np.linalg.norm(r) + np.linalg.norm(ro))
        assert abs(J - Jo[c]) <= 1e-10 * abs(Jo[c]) + bound, (c, J, Jo[c], bound, info)
        assert np.linalg.norm(r) <= max(1e-10, 4 * info["floor"]) * np.linalg.norm(p.F[:, c]), info


def _oracle(p, rho):
    Uo = fem.solve(p, rho)
    return [fem.compliance(p, Uo[:, c], p.F[:, c]) for c in range(p.F.shape[1])], Uo


@pytest.mark.parametrize("case", list(CASES))
def test_mg_solve_matches_oracle(torch, case):
    from paper_2004_05756_gb300.native import Topo, TOPO_PARAM_PCG_MG, TOPO_PARAM_PCG_POLY
    p = CASES[case]()
    psi = w.design_field(p, 0)
    if case == "q4_40x1":
        # one element high: the seeded field's near-void elements would leave the load hanging on
        # void (J ~ 3e12, an FP64 residual floor of ~5e-3 for any solver), so no void here
        psi = 0.3 + 0.7 * psi
    rho = hatfilter.filter_fwd(p, psi)
    Jo = _oracle(p, rho)
    T = Topo(p)
    U = torch.zeros((1, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-13, maxit=200000, prec="fp64")
    T.topo_check()
    assert info["mg_levels"] >= 2 and info["poly"] == 0 and info["fallback"] == 0, info
    _check(p, rho, U, info, Jo)
    # the same solve with Jacobi takes many more iterations
    T.topo_set_param(TOPO_PARAM_PCG_MG, 0)
    T.topo_set_param(TOPO_PARAM_PCG_POLY, 1)
    U1 = torch.zeros_like(U)
    info1 = T.topo_solve_hdm(dev(rho), cols(p.F), U1, rtol=1e-13, maxit=200000, prec="fp64")
    assert info1["mg_levels"] == 0 and info1["status"] == 0
    assert info["iters"] < info1["iters"], (info, info1)


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
@pytest.mark.parametrize("single", [-1, 0, 2048, 10 ** 9])
def test_mg_degree_and_single_cta_levels(torch, deg, single):
    from paper_2004_05756_gb300.native import Topo, TOPO_PARAM_MG_DEGREE, TOPO_PARAM_MG_SINGLE_NODES
    p = CASES["q4_130x41"]()
    rho = hatfilter.filter_fwd(p, w.design_field(p, 1))
    Jo = _oracle(p, rho)
    T = Topo(p)
    T.topo_set_param(TOPO_PARAM_MG_DEGREE, deg)
    T.topo_set_param(TOPO_PARAM_MG_SINGLE_NODES, single)
    U = torch.zeros((1, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-13, maxit=200000, prec="fp64")
    T.topo_check()
    assert info["mg_levels"] >= 3 and info["fallback"] == 0, info
    _check(p, rho, U, info, Jo)


def test_mg_multiload_and_warm_start(torch):
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d_multiload(64, 32, 4, seed=5)
    psi = 0.3 + 0.7 * w.design_field(p, 3)  # no void at the loads
    rho = hatfilter.filter_fwd(p, psi)
    Jo = _oracle(p, rho)
    T = Topo(p)
    U = torch.zeros((4, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-13, maxit=100000, prec="fp64")
    T.topo_check()
    assert info["mg_levels"] >= 2
    _check(p, rho, U, info, Jo)
    info2 = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-8, prec="fp64")
    assert info2["iters"] == 0 and info2["status"] == 0


def test_mg_full_size_600x200(torch):
    """The benchmark mesh at the benchmark's rtol 1e-8: compliance within 1e-6 of SuperLU, in
    far fewer iterations than the polynomial preconditioner needs (about 1,400)."""
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_600x200()
    rho = hatfilter.filter_fwd(p, w.design_field(p, 0))
    Jo = fem.compliance(p, fem.solve(p, rho))
    T = Topo(p)
    U = torch.zeros((1, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-8, maxit=100000, prec="fp64")
    T.topo_check()
    assert info["status"] == 0 and info["relres"] <= 1e-8 and info["mg_levels"] >= 5, info
    assert info["fallback"] == 0, info
    assert abs(fem.compliance(p, host_cols(U)) - Jo) <= 1e-6 * abs(Jo)
    assert info["iters"] < 300, info


def test_mg_parameter_ranges(torch):
    from paper_2004_05756_gb300.native import (Topo, TopoError, TOPO_PARAM_MG_DEGREE, TOPO_PARAM_MG_SINGLE_NODES,
                                               TOPO_PARAM_PCG_MG)
    T = Topo(CASES["q4_40x1"]())
    for v in (0, 1):
        T.topo_set_param(TOPO_PARAM_PCG_MG, v)
    for v in (1, 2, 3, 4):
        T.topo_set_param(TOPO_PARAM_MG_DEGREE, v)
    for v in (-1, 0, 1, 2048, 10 ** 9):
        T.topo_set_param(TOPO_PARAM_MG_SINGLE_NODES, v)
    for which, bad in ((TOPO_PARAM_PCG_MG, 2), (TOPO_PARAM_MG_DEGREE, 0), (TOPO_PARAM_MG_DEGREE, 5),
                       (TOPO_PARAM_MG_DEGREE, 1.5), (TOPO_PARAM_MG_SINGLE_NODES, -2)):
        with pytest.raises(TopoError):
            T.topo_set_param(which, bad)


def test_mg_too_small_to_coarsen_uses_polynomial(torch):
    """One element: 8 DOFs, nothing to coarsen; the solve reports the polynomial preconditioner."""
    from paper_2004_05756_gb300.native import Topo
    p = w.mbb_2d(1, 1)
    rho = hatfilter.filter_fwd(p, w.design_field(p, 0))
    Jo = _oracle(p, rho)
    T = Topo(p)
    U = torch.zeros((1, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-13, maxit=1000, prec="fp64")
    assert info["mg_levels"] == 0 and info["poly"] >= 1
    _check(p, rho, U, info, Jo)


def test_mg_stagnation_falls_back_to_polynomial(torch):
    """A seeded design whose FP32 V-cycle stalls (a stiff region held by void elements, two top-edge
    load cases: the 68x34 instance of the 256-instance batch): the solve notices that the residual
    no longer halves, finishes with the polynomial preconditioner and reports the fallback,
    instead of running to maxit."""
    from paper_2004_05756_gb300.native import Topo
    d = w.batch_instances(256)[103]
    p = d["problem"]
    assert (p.nx, p.ny, p.F.shape[1]) == (68, 34, 2)
    rho = hatfilter.filter_fwd(p, w.design_field(p, d["design_seed"]))
    Jo = _oracle(p, rho)
    T = Topo(p)
    U = torch.zeros((2, p.ndof), dtype=torch.float64, device="cuda")
    info = T.topo_solve_hdm(dev(rho), cols(p.F), U, rtol=1e-8, maxit=20000, prec="fp64")
    T.topo_check()
    assert info["status"] == 0 and info["fallback"] == 1 and info["iters"] < 2000, info
    _check(p, rho, U, info, Jo, rtol=1e-8)
