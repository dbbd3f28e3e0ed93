"""Pins for the oracle's full-order model (Sections 2.1, 2.3, 2.4): symmetry and rigid-body
null space of K(rho), SPD after Dirichlet elimination, the Q1 patch test (exact linear
solution and closed-form compliance), f^T u = u^T K u, two independent solve routes,
and central finite differences of the filtered compliance gradient."""
import numpy as np
import pytest

from oracle import fem, hatfilter, pipeline
from paper_2004_05756_gb300 import workloads as w


def _rbm(p):
    """Rigid-body modes of the whole grid (nodal coordinates = grid indices)."""
    dim = p.dim
    if dim == 2:
        jj, ii = np.meshgrid(np.arange(p.ny + 1), np.arange(p.nx + 1), indexing="ij")
        X = np.stack([ii.ravel(), jj.ravel()], 1).astype(float)
        pairs = [(0, 1)]
    else:
        kk, jj, ii = np.meshgrid(np.arange(p.nz + 1), np.arange(p.ny + 1), np.arange(p.nx + 1), indexing="ij")
        X = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1).astype(float)
        pairs = [(0, 1), (1, 2), (2, 0)]
    modes = []
    for c in range(dim):
        v = np.zeros_like(X)
        v[:, c] = 1
        modes.append(v.ravel())
    for a, b in pairs:
        v = np.zeros_like(X)
        v[:, a] = -X[:, b]
        v[:, b] = X[:, a]
        modes.append(v.ravel())
    return np.array(modes).T


@pytest.mark.parametrize("prob", ["q4", "h8"])
def test_symmetry_null_space_spd(prob):
    p = w.mbb_2d(5, 3) if prob == "q4" else w.cantilever_3d(3, 2, 2)
    rho = np.random.default_rng(3).uniform(0.05, 1.0, p.nel)
    K = fem.assemble_K(p, rho)
    assert abs(K - K.T).max() < 1e-15 * abs(K).max()
    R = _rbm(p)
    assert np.abs(K @ R).max() < 1e-13 * abs(K).max() * np.abs(R).max()
    ev = np.linalg.eigvalsh(fem.reduced_K(p, rho).toarray())
    assert ev[0] > 0


def _patch_problem(dim, n, sigma):
    if dim == 2:
        p = w.Problem(2, n[0], n[1], 0, None, None)
    else:
        p = w.Problem(3, n[0], n[1], n[2], None, None)
    N = p.ndof
    fixed = np.zeros(N, np.uint8)
    F = np.zeros((N, 1))
    nzr = range(p.nz + 1) if dim == 3 else [0]
    for k in nzr:
        for j in range(p.ny + 1):
            for i in range(p.nx + 1):
                nd = w.node_id(p, i, j, k)
                if i == 0:
                    fixed[dim * nd + 0] = 1
                if j == 0:
                    fixed[dim * nd + 1] = 1
                if dim == 3 and k == 0:
                    fixed[dim * nd + 2] = 1
                if i == p.nx:
                    # consistent nodal force of a uniform traction sigma on unit faces
                    wy = 0.5 if j in (0, p.ny) else 1.0
                    wz = (0.5 if k in (0, p.nz) else 1.0) if dim == 3 else 1.0
                    F[dim * nd + 0, 0] = sigma * wy * wz
    p.fixed, p.F = fixed, F
    return p


@pytest.mark.parametrize("dim,n", [(2, (4, 3)), (2, (7, 2)), (3, (3, 2, 2))])
@pytest.mark.parametrize("c", [1.0, 0.4])
def test_patch_test(dim, n, c):
    """Uniform tension: u_x = s x/E, u_y = -nu s y/E (u_z = -nu s z/E), J = s^2 vol/E."""
    sigma = 0.7
    p = _patch_problem(dim, n, sigma)
    rho = np.full(p.nel, c)
    E = fem.young(np.array([c]), p.E0, p.Emin, p.penal)[0]
    U = fem.solve(p, rho)[:, 0]
    coords = []
    for k in (range(p.nz + 1) if dim == 3 else [0]):
        for j in range(p.ny + 1):
            for i in range(p.nx + 1):
                coords.append((i, j, k))
    coords = np.array(coords, float)
    ex = np.zeros(p.ndof)
    ex[0::dim] = sigma * coords[:, 0] / E
    ex[1::dim] = -p.nu * sigma * coords[:, 1] / E
    if dim == 3:
        ex[2::dim] = -p.nu * sigma * coords[:, 2] / E
    assert np.abs(U - ex).max() < 1e-10 * np.abs(ex).max()
    vol = p.nx * p.ny * (p.nz if dim == 3 else 1)
    J = fem.compliance(p, U)
    assert J == pytest.approx(sigma ** 2 * vol / E, rel=1e-10)


@pytest.mark.parametrize("prob", ["q4", "h8"])
def test_compliance_energy_and_cg(prob):
    p = w.mbb_2d(12, 6) if prob == "q4" else w.cantilever_3d(4, 3, 3)
    psi = w.design_field(p, 5)
    rho = hatfilter.filter_fwd(p, psi)
    U = fem.solve(p, rho)
    J = fem.compliance(p, U)
    JU = float(U[:, 0] @ fem.apply_K(p, rho, U[:, 0]))
    assert JU == pytest.approx(J, rel=1e-10)
    Ucg, its = fem.solve_cg(p, rho, rtol=1e-13)
    assert its > 0
    assert np.abs(Ucg - U).max() < 1e-8 * np.abs(U).max()
    assert fem.compliance(p, Ucg) == pytest.approx(J, rel=1e-10)


def test_apply_convention():
    """Library operator convention: identity rows/cols on Dirichlet DOFs, K_ff elsewhere."""
    p = w.mbb_2d(4, 3)
    rho = np.random.default_rng(1).uniform(0.1, 1, p.nel)
    V = np.random.default_rng(2).standard_normal((p.ndof, 3))
    Y = fem.apply_K(p, rho, V)
    K = fem.assemble_K(p, rho).toarray()
    d = fem.fixed_dofs(p)
    K[d, :] = 0
    K[:, d] = 0
    K[d, d] = 1
    assert np.abs(Y - K @ V).max() < 1e-14 * np.abs(Y).max()


@pytest.mark.parametrize("mk", [lambda: w.mbb_2d(7, 5), lambda: w.cantilever_3d(4, 3, 5), lambda: w.mbb_2d(1, 1)])
def test_apply_element_by_element(mk):
    """The unassembled product equals the assembled one (same convention), and on a mesh
    without supports it annihilates the rigid-body modes."""
    import dataclasses
    p = mk()
    rng = np.random.default_rng(3)
    rho = rng.uniform(1e-3, 1, p.nel)
    V = rng.standard_normal((p.ndof, 3))
    Y = fem.apply_K_ebe(p, rho, V)
    assert np.abs(Y - fem.apply_K(p, rho, V)).max() < 1e-13 * np.abs(Y).max()
    assert np.abs(fem.apply_K_ebe(p, rho, V[:, 1]) - Y[:, 1]).max() < 1e-13 * np.abs(Y).max()
    pf = dataclasses.replace(p, fixed=np.zeros_like(p.fixed))
    R = _rbm(pf)
    KR = fem.apply_K_ebe(pf, rho, R)
    assert np.abs(KR).max() < 1e-12 * np.abs(R).max()
    assert np.abs(fem.apply_K_ebe(pf, rho, V)).max() > 1e-3


@pytest.mark.parametrize("prob", ["q4", "h8"])
@pytest.mark.parametrize("filtered", [False, True])
def test_gradient_finite_differences(prob, filtered):
    p = w.mbb_2d(4, 2) if prob == "q4" else w.cantilever_3d(2, 2, 2)
    psi = np.random.default_rng(11).uniform(0.2, 0.9, p.nel)
    base = pipeline.hdm_eval(p, psi, filtered=filtered)
    g = base["dpsi"]
    assert np.all(base["dc"] <= 0)
    if filtered:
        assert np.all(g <= 0)
    fd = np.zeros(p.nel)
    for e in range(p.nel):
        h = 1e-6 * max(1.0, psi[e])
        pp = psi.copy()
        pp[e] += h
        pm = psi.copy()
        pm[e] -= h
        fd[e] = (pipeline.hdm_eval(p, pp, filtered)["J"] - pipeline.hdm_eval(p, pm, filtered)["J"]) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()


def test_planted_mistake_caught_by_fd(monkeypatch):
    """A plausible slip (dropping the exponent's factor p in E') must fail the FD pin."""
    p = w.mbb_2d(4, 2)
    psi = np.random.default_rng(11).uniform(0.2, 0.9, p.nel)
    monkeypatch.setattr(fem, "dyoung", lambda rho, E0, Emin, pen: rho ** (pen - 1.0) * (E0 - Emin))
    g = pipeline.hdm_eval(p, psi, filtered=True)["dpsi"]
    monkeypatch.undo()
    h = 1e-6
    fd = []
    for e in range(p.nel):
        pp = psi.copy(); pp[e] += h
        pm = psi.copy(); pm[e] -= h
        fd.append((pipeline.hdm_eval(p, pp)["J"] - pipeline.hdm_eval(p, pm)["J"]) / (2 * h))
    assert np.abs(np.array(fd) - g).max() > 1e-3 * np.abs(g).max()
