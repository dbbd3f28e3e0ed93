"""General linear outputs (Sections 2.4 and 3.2-3.3) through the C ABI against the oracle: the
adjoint solve (topo_solve_hdm with the output vector as load), topo_output_grad (J and the mixed
gradient -E' lambda_e^T K_e u_e, filtered), its compliance special case, and the ROM of the adjoint
(topo_rom_rhs for Phi^T l, reduced primal and adjoint solves, primal and adjoint residuals, the
ROM output and its gradient) on 2D and 3D meshes."""
import numpy as np
import pytest

from oracle import fem, hatfilter, output, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, host_cols, require_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "q4_30x12": lambda: w.mbb_2d(30, 12),
    "h8_8x5x4": lambda: w.cantilever_3d(8, 5, 4),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _setup(case):
    p = CASES[case]()
    psi = 0.3 + 0.6 * w.design_field(p, 4)
    node = (p.nx + 1) * p.ny + p.nx // 2 if p.dim == 2 else p.nnodes - (p.nx + 1) // 2 - 1
    l = output.point_output(p, node=node, comp=1)
    return p, psi, l


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_solve_and_output_gradient(torch, case):
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p, psi, l = _setup(case)
    ref = output.hdm_output(p, psi, l)
    T = Topo(p)
    f64 = dict(dtype=th.float64, device="cuda")
    rho = th.empty(p.nel, **f64)
    T.topo_filter(dev(psi), rho)
    U = th.zeros((1, p.ndof), **f64)
    Lam = th.zeros((1, p.ndof), **f64)
    L = dev(l[None, :].copy())
    T.topo_solve_hdm(rho, cols(p.F[:, :1]), U, rtol=1e-13, maxit=100000)
    T.topo_solve_hdm(rho, L, Lam, rtol=1e-13, maxit=100000)
    # the states carry the solve's conditioning (relres 1e-13 times cond(K) ~ 1e5); J does not
    assert np.max(np.abs(Lam.cpu().numpy()[0] - ref["lam"])) <= 1e-7 * np.max(np.abs(ref["lam"]))
    J = th.zeros(1, **f64)
    dc = th.empty(p.nel, **f64)
    dp = th.empty(p.nel, **f64)
    T.topo_output_grad(rho, U, Lam, L, J, dc, dp)
    T.topo_check()
    assert J.item() == pytest.approx(ref["J"], rel=1e-10)
    # the gradient of the GPU's own states, by the oracle's element loop
    dco = output.mixed_grad_rho(p, rho.cpu().numpy(), U.cpu().numpy()[0], Lam.cpu().numpy()[0])
    assert np.max(np.abs(dc.cpu().numpy() - dco)) <= 1e-12 * np.max(np.abs(dco))
    assert np.max(np.abs(dp.cpu().numpy() - hatfilter.filter_adj(p, dco))) <= 1e-12 * np.max(np.abs(dco))
    assert np.max(np.abs(dp.cpu().numpy() - ref["dpsi"])) <= 1e-7 * np.max(np.abs(ref["dpsi"]))


def test_compliance_is_the_special_case(torch):
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p = CASES["q4_30x12"]()
    rho = dev(hatfilter.filter_fwd(p, w.design_field(p, 1)))
    U = cols(fem.solve(p, rho.cpu().numpy()))
    F = cols(p.F)
    T = Topo(p)
    f64 = dict(dtype=th.float64, device="cuda")
    J1, J2 = th.zeros(1, **f64), th.zeros(1, **f64)
    d1, d2 = th.empty(p.nel, **f64), th.empty(p.nel, **f64)
    T.topo_compliance_grad(rho, U, F, J1, d1)
    T.topo_output_grad(rho, U, U, F, J2, d2)
    assert J1.item() == J2.item()
    # the symmetric and the full form round differently; u_e^T K_e u_e cancels for elements that
    # move nearly rigidly, so the bound is elementwise: 2 n eps E' |u_e|^T |K_e| |u_e|
    from oracle import element
    Ke = np.abs(element.ke(p.dim, p.nu))
    ue = np.abs(host_cols(U)[fem.edof(p), 0])
    bound = 2 * 8 * 2.2e-16 * np.abs(fem.dyoung(rho.cpu().numpy(), p.E0, p.Emin, p.penal)) * \
        np.einsum("ei,ij,ej->e", ue, Ke, ue)
    assert np.all(np.abs(d1.cpu().numpy() - d2.cpu().numpy()) <= bound + 1e-300)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("with_adjoint", [True, False])
def test_rom_output(torch, case, with_adjoint):
    """Primal snapshots (and, with_adjoint, the adjoint state at the evaluation point: the ROM then
    reproduces J, Remark rom_adjoint) -> basis; reduced primal and adjoint solves; residuals,
    output and gradient against the oracle on the same snapshots."""
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p, psi, l = _setup(case)
    f = p.F[:, 0]
    snaps = [fem.solve(p, hatfilter.filter_fwd(p, q), p.F[:, :1])[:, 0]
             for q in w.perturbed_designs(p, psi, 3, 0.1, first_seed=30).T]
    ref_h = output.hdm_output(p, psi, l)
    if with_adjoint:
        snaps += [ref_h["u"], ref_h["lam"]]
    S = np.column_stack(snaps)
    Phi_o = rom.basis(S)
    ref = output.rom_output(p, psi, Phi_o, l)
    T = Topo(p)
    f64 = dict(dtype=th.float64, device="cuda")
    rho = th.empty(p.nel, **f64)
    T.topo_filter(dev(psi), rho)
    m = S.shape[1]
    Phi = th.zeros((m, p.ndof), **f64)
    bf = th.zeros(m, **f64)
    k = T.topo_rom_build(rho, dev(S.T.copy()), Phi, None, bf, dev(f))
    assert k == Phi_o.shape[1]
    bl = th.zeros(k, **f64)
    T.topo_rom_rhs(Phi[:k], k, dev(l), bl)
    assert np.allclose(Phi[:k].cpu().numpy() @ l, bl.cpu().numpy(), rtol=0, atol=1e-14)
    Hel = th.zeros((p.nel + 1) * k * (k + 1) // 2, **f64)
    T.topo_rom_elem(Phi[:k], k, Hel)
    y, z = th.zeros(k, **f64), th.zeros(k, **f64)
    Hw = th.zeros(k * k, **f64)
    Jf, Jl = th.zeros(1, **f64), th.zeros(1, **f64)
    T.topo_rom_solve_elem(rho, Hel, k, bf[:k], Hw, y, Jf)
    T.topo_rom_solve_elem(rho, Hel, k, bl, Hw, z, Jl)
    rn, ra = th.zeros(2, **f64), th.zeros(2, **f64)
    uk, lk = th.zeros((1, p.ndof), **f64), th.zeros((1, p.ndof), **f64)
    T.topo_rom_error(rho, Phi[:k], k, y, dev(f), rn, uk[0])
    T.topo_rom_error(rho, Phi[:k], k, z, dev(l), ra, lk[0])
    J = th.zeros(1, **f64)
    dc = th.empty(p.nel, **f64)
    dp = th.empty(p.nel, **f64)
    T.topo_output_grad(rho, uk, lk, dev(l[None, :].copy()), J, dc, dp)
    T.topo_check()
    # J_k cancels like the compliance J_k (rounding of y^T H y style sums): 1e-10 plus a margin
    assert J.item() == pytest.approx(ref["Jk"], rel=1e-9)
    if with_adjoint:  # both states are in the basis: the residuals sit at the rounding floor
        assert rn[0].item() <= 1e-9 * np.linalg.norm(f) and ra[0].item() <= 1e-9 * np.linalg.norm(l)
        assert ref["resnorm"] <= 1e-9 * np.linalg.norm(f) and ref["adj_resnorm"] <= 1e-9 * np.linalg.norm(l)
    else:
        assert rn[0].item() == pytest.approx(ref["resnorm"], rel=1e-7)
        assert ra[0].item() == pytest.approx(ref["adj_resnorm"], rel=1e-7)
    assert np.max(np.abs(dp.cpu().numpy() - ref["dpsi"])) <= 1e-8 * np.max(np.abs(ref["dpsi"]))
    if with_adjoint:
        assert J.item() == pytest.approx(ref_h["J"], rel=1e-9)
    else:
        # a real model error, inside Theorem rom_output_error's bound for linear outputs
        assert abs(J.item() - ref_h["J"]) > 1e-9 * abs(ref_h["J"])
        if p.ndof <= 4000:
            smin = rom.sigma_min_dense(p, ref_h["rho"])
            assert abs(J.item() - ref_h["J"]) <= rn[0].item() * ra[0].item() / smin * (1 + 1e-6)
