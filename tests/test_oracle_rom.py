"""Pins for the oracle's reduced model (Sections 3.1-3.3 and the linear-output case of the
proofs in Appendix C): exact reproduction when u lies in span(Phi) (Remark rom_exact),
Galerkin orthogonality, J - J_k = r^T K^{-1} r >= 0, monotone energy error under
enrichment (Remark rom_refine), Theorem rom_primal_error and the compliance output bound,
and the orthonormal basis with its rank rule."""
import numpy as np
import pytest

from oracle import fem, hatfilter, pipeline, rom
from paper_2004_05756_gb300 import workloads as w


def _setup(kind="q4"):
    p = w.mbb_2d(10, 5) if kind == "q4" else w.cantilever_3d(4, 3, 3)
    psi = w.design_field(p, 0)
    snaps = w.perturbed_designs(p, psi, 4)
    U = np.stack([pipeline.hdm_eval(p, snaps[:, i])["U"][:, 0] for i in range(4)], 1)
    return p, psi, U


@pytest.mark.parametrize("kind", ["q4", "h8"])
def test_exact_when_u_in_span(kind):
    p, psi, U = _setup(kind)
    hdm = pipeline.hdm_eval(p, psi)
    Phi = rom.basis(np.concatenate([U, hdm["U"]], 1))
    r = pipeline.rom_eval_full(p, psi, Phi)
    assert r["Jk"] == pytest.approx(hdm["J"], rel=1e-10)
    assert np.abs(r["uk"] - hdm["U"][:, 0]).max() < 1e-9 * np.abs(hdm["U"]).max()
    assert r["relres"] < 1e-9
    assert np.abs(r["dpsi"] - hdm["dpsi"]).max() < 1e-8 * np.abs(hdm["dpsi"]).max()


@pytest.mark.parametrize("kind", ["q4", "h8"])
def test_galerkin_identities_and_bounds(kind):
    p, psi, U = _setup(kind)
    Phi = rom.basis(U)
    hdm = pipeline.hdm_eval(p, psi)
    r = pipeline.rom_eval_full(p, psi, Phi)
    rho = r["rho"]
    # Galerkin orthogonality: Phi^T r = 0
    assert np.abs(Phi.T @ r["r"]).max() < 1e-10 * np.linalg.norm(r["r"]) + 1e-14
    # compliance: J - J_k = r^T K^{-1} r = ||u - u_k||_K^2 >= 0
    f = fem.free_dofs(p)
    e = hdm["U"][:, 0] - r["uk"]
    eK2 = rom.energy_norm(p, rho, e) ** 2
    Kinv_r = np.zeros(p.ndof)
    Kinv_r[f] = fem.solve(p, rho, r["r"][:, None])[f, 0]
    assert hdm["J"] - r["Jk"] >= 0
    assert hdm["J"] - r["Jk"] == pytest.approx(eK2, rel=1e-6)
    assert hdm["J"] - r["Jk"] == pytest.approx(float(r["r"] @ Kinv_r), rel=1e-6)
    # Theorem rom_primal_error and the compliance output bound
    smin = rom.sigma_min_dense(p, rho)
    assert np.sqrt(eK2) <= smin ** -0.5 * r["resnorm"] * (1 + 1e-12)
    assert hdm["J"] - r["Jk"] <= r["resnorm"] ** 2 / smin * (1 + 1e-12)
    # H symmetric positive definite (Remark rom_wellposed)
    assert np.abs(r["H"] - r["H"].T).max() < 1e-12 * np.abs(r["H"]).max()
    assert np.linalg.eigvalsh(0.5 * (r["H"] + r["H"].T))[0] > 0


def test_monotone_under_enrichment():
    p, psi, U = _setup("q4")
    hdm = pipeline.hdm_eval(p, psi)
    errs = []
    for k in range(1, U.shape[1] + 1):
        Phi = rom.basis(U[:, :k])
        r = pipeline.rom_eval_full(p, psi, Phi)
        errs.append(rom.energy_norm(p, r["rho"], hdm["U"][:, 0] - r["uk"]))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-10) for i in range(len(errs) - 1))


def test_basis_rank_rule():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 3))
    U = np.concatenate([A, A[:, :1] * 2 + A[:, 1:2], rng.standard_normal((50, 1))], 1)
    Phi = rom.basis(U)
    assert Phi.shape[1] == 4
    assert np.abs(Phi.T @ Phi - np.eye(4)).max() < 1e-14
    # span check: projection of U onto span(Phi) reproduces U
    assert np.abs(Phi @ (Phi.T @ U) - U).max() < 1e-12 * np.abs(U).max()
    assert rom.basis(np.zeros((10, 2))).shape == (10, 0)


def test_cholesky_solve_matches_library():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((8, 8))
    H = A @ A.T + 8 * np.eye(8)
    b = rng.standard_normal(8)
    assert np.abs(rom.solve_reduced(H, b) - np.linalg.solve(H, b)).max() < 1e-13


def test_pod_pins():
    """POD_n (Section 4.2): orthonormal vectors, singular values equal to the square roots of the
    Gram matrix's eigenvalues (an independent route), the Eckart-Young projection error, a rank-one
    closed form and optimality against random subspaces."""
    rng = np.random.default_rng(9)
    U = rng.normal(size=(200, 7)) @ np.diag([10, 5, 3, 1, 0.5, 0.1, 0.01]) @ rng.normal(size=(7, 7))
    for n in range(0, 8):
        P, s = rom.pod(U, n)
        assert P.shape == (200, n)
        assert np.allclose(P.T @ P, np.eye(n), atol=1e-12)
        err = np.linalg.norm(U - P @ (P.T @ U)) ** 2
        assert err == pytest.approx(np.sum(s[n:] ** 2), rel=1e-9, abs=1e-20)
        for _ in range(5):
            Q, _ = np.linalg.qr(rng.normal(size=(200, n)))
            assert np.linalg.norm(U - Q @ (Q.T @ U)) ** 2 >= err * (1 - 1e-12)
    _, s = rom.pod(U, 3)
    assert np.allclose(np.sort(s ** 2), np.sort(np.linalg.eigvalsh(U.T @ U)), rtol=1e-9)
    a, b = rng.normal(size=50), rng.normal(size=4)
    P1, s1 = rom.pod(np.outer(a, b), 1)
    assert s1[0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b), rel=1e-13)
    assert abs(abs(P1[:, 0] @ a) / np.linalg.norm(a) - 1) < 1e-13


def test_sigma_min_dense_by_shift_invert():
    """sigma_min of K_ff (dense eigvalsh) against scipy's shift-invert Lanczos (ARPACK): two
    independent routes to the smallest eigenvalue that the Section 3.3 bounds use."""
    import scipy.sparse.linalg as spla
    for p in (w.mbb_2d(12, 5), w.cantilever_3d(4, 3, 2)):
        rho = hatfilter.filter_fwd(p, w.design_field(p, 1))
        s_dense = rom.sigma_min_dense(p, rho)
        s_arpack = spla.eigsh(fem.reduced_K(p, rho), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
        assert s_dense == pytest.approx(s_arpack, rel=1e-9)
        assert s_dense > 0
