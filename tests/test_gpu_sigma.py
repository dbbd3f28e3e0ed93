"""sigma_min(K(rho)) by shift-invert Lanczos (topo_sigma_min) against the oracle's dense
eigenvalue, and its use in the a posteriori bounds of Section 3.3: the compliance error of a ROM
evaluation stays below ||r||^2 / sigma_min with the GPU's lower bound."""
import numpy as np
import pytest

from oracle import fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import dev, require_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "q4_20x8": lambda: w.mbb_2d(20, 8),
    "q4_37x13": lambda: w.mbb_2d(37, 13),
    "h8_5x4x3": lambda: w.cantilever_3d(5, 4, 3),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.mark.parametrize("case", list(CASES))
def test_sigma_min_matches_dense(torch, case):
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p = CASES[case]()
    rho = hatfilter.filter_fwd(p, 0.2 + 0.8 * w.design_field(p, 2))
    ref = rom.sigma_min_dense(p, rho)
    T = Topo(p)
    out = th.zeros(4, dtype=th.float64, device="cuda")
    T.topo_sigma_min(dev(rho), out, steps=40, rtol=1e-12)
    T.topo_check()
    est, low, theta, res = out.cpu().numpy()
    assert est == pytest.approx(ref, rel=1e-6), (est, ref, res)
    assert low <= ref * (1 + 1e-9) and est >= ref * (1 - 1e-6)
    assert theta == pytest.approx(1.0 / est, rel=1e-14)


def test_certified_compliance_bound(torch):
    """A ROM evaluation on a basis of nearby snapshots: |J - J_k| <= ||r||^2 / sigma_min (the
    compliance form of Theorem rom_output_error) holds with the GPU's lower bound."""
    import torch as th
    from paper_2004_05756_gb300.native import Topo
    p = CASES["q4_37x13"]()
    psi = 0.2 + 0.8 * w.design_field(p, 5)
    rho = hatfilter.filter_fwd(p, psi)
    f = p.F[:, 0]
    snaps = np.column_stack([fem.solve(p, hatfilter.filter_fwd(p, q))[:, 0]
                             for q in w.perturbed_designs(p, psi, 3, 0.1, first_seed=60).T])
    Phi = rom.basis(snaps)
    ev = rom.rom_eval(p, rho, Phi, f)
    J = fem.compliance(p, fem.solve(p, rho))
    T = Topo(p)
    out = th.zeros(4, dtype=th.float64, device="cuda")
    T.topo_sigma_min(dev(rho), out, steps=30, rtol=1e-12)
    low = out.cpu().numpy()[1]
    err = abs(J - ev["Jk"])
    assert err > 0 and err <= ev["resnorm"] ** 2 / low


def test_invalid_arguments(torch):
    import torch as th
    from paper_2004_05756_gb300.native import Topo, TopoError
    p = CASES["q4_20x8"]()
    T = Topo(p)
    rho = th.full((p.nel,), 0.5, dtype=th.float64, device="cuda")
    out = th.zeros(4, dtype=th.float64, device="cuda")
    for kw in (dict(steps=1), dict(steps=65), dict(rtol=0.0), dict(rtol=0.5)):
        with pytest.raises(TopoError):
            T.topo_sigma_min(rho, out, **kw)
