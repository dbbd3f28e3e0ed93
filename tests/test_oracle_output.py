"""Pins of the oracle's general-output functions (Section 2.4 and 3.2-3.3): the adjoint gradient
against central finite differences of J(psi), the compliance special case (lambda = u), the ROM's
exactness when the basis holds both the primal and the adjoint state (Remark rom_adjoint), the
dual-weighted identity J - J_k = -(lambda - lambda_k)^T r, and Theorem rom_output_error's bound
for a linear output."""
import numpy as np
import pytest

from oracle import fem, hatfilter, output, rom
from paper_2004_05756_gb300 import workloads as w


def _case():
    p = w.mbb_2d(14, 6)
    psi = 0.3 + 0.6 * w.design_field(p, 2)
    l = output.point_output(p, node=(p.nx + 1) * p.ny + p.nx // 2, comp=1)  # top-middle node, y
    return p, psi, l


def test_adjoint_gradient_matches_finite_differences():
    p, psi, l = _case()
    h = output.hdm_output(p, psi, l)
    rng = np.random.default_rng(0)
    for e in rng.choice(p.nel, 6, replace=False):
        d = 1e-6
        Jp = output.hdm_output(p, np.where(np.arange(p.nel) == e, psi + d, psi), l)["J"]
        Jm = output.hdm_output(p, np.where(np.arange(p.nel) == e, psi - d, psi), l)["J"]
        fd = (Jp - Jm) / (2 * d)
        assert h["dpsi"][e] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.max(np.abs(h["dpsi"])))


def test_compliance_special_case():
    p, psi, _ = _case()
    f = p.F[:, 0]
    h = output.hdm_output(p, psi, f)
    assert np.allclose(h["lam"], h["u"], rtol=1e-12, atol=1e-14 * np.max(np.abs(h["u"])))
    assert h["J"] == pytest.approx(fem.compliance(p, h["u"][:, None]), rel=1e-13)
    assert np.allclose(h["dc"], fem.compliance_grad_rho(p, h["rho"], h["u"][:, None]), rtol=1e-10)


def test_rom_exact_with_primal_and_adjoint_in_the_basis():
    p, psi, l = _case()
    h = output.hdm_output(p, psi, l)
    Phi = rom.basis(np.column_stack([h["u"], h["lam"]]))
    r = output.rom_output(p, psi, Phi, l)
    assert r["Jk"] == pytest.approx(h["J"], rel=1e-10)
    assert np.allclose(r["lk"], h["lam"], atol=1e-9 * np.max(np.abs(h["lam"])))
    assert np.allclose(r["dpsi"], h["dpsi"], atol=1e-8 * np.max(np.abs(h["dpsi"])))


def test_dual_weighted_identity_and_output_bound():
    p, psi, l = _case()
    h = output.hdm_output(p, psi, l)
    snaps = [fem.solve(p, hatfilter.filter_fwd(p, q), p.F[:, :1])[:, 0]
             for q in w.perturbed_designs(p, psi, 3, 0.1, first_seed=30).T]
    Phi = rom.basis(np.column_stack(snaps))
    r = output.rom_output(p, psi, Phi, l)
    err = h["J"] - r["Jk"]
    assert abs(err) > 1e-8 * abs(h["J"])  # a basis without the adjoint: a real model error
    assert err == pytest.approx(-(h["lam"] - r["lk"]) @ r["r"], rel=1e-8)
    smin = rom.sigma_min_dense(p, h["rho"])
    assert abs(err) <= r["resnorm"] * r["adj_resnorm"] / smin * (1 + 1e-10)
