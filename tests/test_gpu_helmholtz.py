"""The Helmholtz density filter (Section 2.2) through the C ABI (TOPO_PARAM_FILTER = 1) against
the oracle's assembled sparse solve: forward and adjoint on 2D and 3D meshes whose node counts
span several 64-wide tiles of the transforms with ragged edges, one element wide, at several
lengths r; constants and volume preserved; the batched filter inside topo_rom_eval_batch and the
filtered gradient of topo_compliance_grad; switching back to the cone filter."""
import math

import numpy as np
import pytest

from oracle import fem, hatfilter, helmholtz
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu

MESHES = {
    "q4_9x5": lambda: w.mbb_2d(9, 5),
    "q4_1x6": lambda: w.mbb_2d(1, 6),
    "q4_70x37": lambda: w.mbb_2d(70, 37),       # 71 x 38 nodes: two tiles along x, ragged
    "q4_130x41": lambda: w.mbb_2d(130, 41),
    "h8_5x4x3": lambda: w.cantilever_3d(5, 4, 3),
    "h8_20x9x7": lambda: w.cantilever_3d(20, 9, 7),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _ctx(p, r=0.0):
    from paper_2004_05756_gb300.native import Topo, TOPO_PARAM_FILTER, TOPO_PARAM_HELMHOLTZ_R
    T = Topo(p)
    T.topo_set_param(TOPO_PARAM_FILTER, 1)
    T.topo_set_param(TOPO_PARAM_HELMHOLTZ_R, r)
    return T


def _filter(T, x, adjoint=False):
    import torch as th
    out = th.empty(len(x), dtype=th.float64, device="cuda")
    T.topo_filter(dev(x), out, adjoint)
    T.topo_check()
    return out.cpu().numpy()


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("r", [0.0, 0.3, 2.5])
def test_forward_and_adjoint_match_oracle(torch, mesh, r):
    p = MESHES[mesh]()
    T = _ctx(p, r)
    rr = r if r > 0 else helmholtz.default_length(p.rmin)
    rng = np.random.default_rng(abs(hash((mesh, r))) % 2 ** 32)
    psi = w.design_field(p, 3)
    v = rng.normal(size=p.nel)
    ref = helmholtz.filter_fwd(p, psi, rr)
    got = _filter(T, psi)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
    ref_a = helmholtz.filter_adj(p, v, rr)
    got_a = _filter(T, v, adjoint=True)
    assert np.max(np.abs(got_a - ref_a)) <= 1e-12 * np.max(np.abs(ref_a))


def test_constants_volume_and_determinism(torch):
    p = MESHES["h8_20x9x7"]()
    T = _ctx(p, 1.1)
    assert np.allclose(_filter(T, np.full(p.nel, 0.42)), 0.42, rtol=0, atol=1e-13)
    psi = np.random.default_rng(5).uniform(0, 1, p.nel)
    a = _filter(T, psi)
    assert a.sum() == pytest.approx(psi.sum(), rel=1e-12)
    assert np.array_equal(a, _filter(T, psi))


def test_batched_filter_and_gradient(torch):
    """topo_rom_eval_batch filters its candidates with the batched Helmholtz path: each candidate's
    reduced compliance equals the one-candidate path on topo_filter's density; the filtered
    gradient of topo_compliance_grad is the oracle's adjoint of the GPU's element gradient."""
    import torch as th
    from paper_2004_05756_gb300.native import TOPO_PARAM_ROM_ASSEMBLY
    p = MESHES["q4_70x37"]()
    T = _ctx(p)
    # the comparison is of the batched filter: the one-candidate reduced solve assembles in FP64
    # SIMT, so the batch does too (the tensor-core assembly has its own tests)
    T.topo_set_param(TOPO_PARAM_ROM_ASSEMBLY, 0)
    rr = helmholtz.default_length(p.rmin)
    f64 = dict(dtype=th.float64, device="cuda")
    psi0 = w.design_field(p, 1)
    rho0 = _filter(T, psi0)
    assert np.max(np.abs(rho0 - helmholtz.filter_fwd(p, psi0, rr))) <= 1e-12
    U = fem.solve(p, rho0)
    # gradient with the Helmholtz adjoint
    J = th.zeros(1, **f64)
    dc = th.empty(p.nel, **f64)
    dp = th.empty(p.nel, **f64)
    T.topo_compliance_grad(dev(rho0), cols(U), cols(p.F), J, dc, dp)
    ref = helmholtz.filter_adj(p, dc.cpu().numpy(), rr)
    assert np.max(np.abs(dp.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    # a 3-snapshot basis and 5 candidates
    snaps = np.stack([fem.solve(p, _filter(T, w.perturbed_designs(p, psi0, 1, 0.1, first_seed=s)[:, 0]))[:, 0]
                      for s in (11, 12, 13)], 0)
    k = 3
    Phi = th.zeros((k, p.ndof), **f64)
    b = th.zeros(k, **f64)
    f = dev(p.F[:, 0])
    kk = T.topo_rom_build(dev(rho0), dev(snaps), Phi, None, b, f)
    Hel = th.zeros((p.nel + 1) * kk * (kk + 1) // 2, **f64)
    T.topo_rom_elem(Phi[:kk], kk, Hel)
    cands = w.perturbed_designs(p, psi0, 5, 0.05, first_seed=40).T.copy()
    Jk = th.zeros(5, **f64)
    rn = th.zeros((5, 2), **f64)
    T.topo_rom_eval_batch(dev(cands), Hel, Phi[:kk], kk, b[:kk], f, Jk, rn, None, None)
    for r in range(5):
        rho_r = th.empty(p.nel, **f64)
        T.topo_filter(dev(cands[r]), rho_r)
        y = th.zeros(kk, **f64)
        Hw = th.zeros(kk * kk, **f64)
        J1 = th.zeros(1, **f64)
        T.topo_rom_solve_elem(rho_r, Hel, kk, b[:kk], Hw, y, J1)
        assert Jk[r].item() == pytest.approx(J1.item(), rel=1e-12)
    T.topo_check()


def test_switch_back_to_cone_and_parameters(torch):
    from paper_2004_05756_gb300.native import Topo, TopoError, TOPO_PARAM_FILTER, TOPO_PARAM_HELMHOLTZ_R
    p = MESHES["q4_9x5"]()
    T = _ctx(p, 0.7)
    psi = w.design_field(p, 2)
    _filter(T, psi)
    T.topo_set_param(TOPO_PARAM_FILTER, 0)
    assert np.array_equal(_filter(T, psi), _filter(Topo(p), psi))
    assert np.allclose(_filter(T, psi), hatfilter.filter_fwd(p, psi), atol=1e-14)
    for which, bad in ((TOPO_PARAM_FILTER, 2), (TOPO_PARAM_FILTER, -1), (TOPO_PARAM_HELMHOLTZ_R, -0.5),
                       (TOPO_PARAM_HELMHOLTZ_R, math.nan)):
        with pytest.raises(TopoError):
            T.topo_set_param(which, bad)
