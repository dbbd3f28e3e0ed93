"""topo_rom_eval_batch (the ROM design evaluations of many candidates on one basis in one
call) against the one-candidate calls and the FP64 oracle, through the C ABI.

Candidate counts below, at and above the internal group of 32 (1, 5, 32, 45), 2D and 3D, k on
both reduced-solve paths (one warp for k <= 32; CTA Cholesky above), filtered designs and raw
densities. Each candidate's results must match the one-candidate calls to FP64 rounding and
the oracle's rom_eval to the tolerances of the ROM parity tests."""
import numpy as np
import pytest

from oracle import fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _setup(torch, p, k, seed):
    from paper_2004_05756_gb300.native import Topo
    T = Topo(p)
    rng = np.random.default_rng(seed)
    psi0 = w.design_field(p, seed)
    snaps = w.perturbed_designs(p, psi0, k, amplitude=0.1, first_seed=seed + 1)
    U = np.stack([fem.solve(p, hatfilter.filter_fwd(p, snaps[:, i]))[:, 0] for i in range(k)], 1)
    Phi = rom.basis(U)
    kk = Phi.shape[1]
    f = p.F[:, 0]
    Phid = cols(Phi)
    Hel = torch.zeros((p.nel + 1) * kk * (kk + 1) // 2, dtype=torch.float64, device="cuda")
    T.topo_rom_elem(Phid, kk, Hel)
    b = dev(Phi.T @ f)
    return T, Phi, Phid, kk, Hel, b, dev(f), psi0, rng


@pytest.mark.parametrize("case,k,R,filtered", [("q4_60x20", 6, 1, True), ("q4_60x20", 6, 45, True),
                                               ("q4_37x13", 16, 32, True), ("q4_37x13", 40, 5, True),
                                               ("h8_6x5x4", 5, 33, True), ("q4_60x20", 8, 7, False)])
def test_rom_eval_batch_matches_single_calls_and_oracle(torch, case, k, R, filtered):
    p = {"q4_60x20": lambda: w.mbb_2d(60, 20), "q4_37x13": lambda: w.mbb_2d(37, 13),
         "h8_6x5x4": lambda: w.cantilever_3d(6, 5, 4)}[case]()
    if k > 20:  # a 40-column basis: orthonormal random columns (the snapshot space of this mesh is small)
        from paper_2004_05756_gb300.native import Topo
        T = Topo(p)
        rng = np.random.default_rng(3)
        Phi, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
        Phi[p.fixed == 1] = 0.0
        Phi, _ = np.linalg.qr(Phi)
        kk = k
        Phid = cols(Phi)
        Hel = torch.zeros((p.nel + 1) * kk * (kk + 1) // 2, dtype=torch.float64, device="cuda")
        T.topo_rom_elem(Phid, kk, Hel)
        f = p.F[:, 0]
        b = dev(Phi.T @ f)
        fd = dev(f)
        psi0 = w.design_field(p, 3)
    else:
        T, Phi, Phid, kk, Hel, b, fd, psi0, rng = _setup(torch, p, k, 11)
    cands = w.perturbed_designs(p, psi0, R, amplitude=0.02, first_seed=300)  # N_e x R
    if not filtered:
        cands = np.stack([hatfilter.filter_fwd(p, cands[:, r]) for r in range(R)], 1)
    psi = dev(np.ascontiguousarray(cands.T))  # (R, N_e)
    f64 = dict(dtype=torch.float64, device="cuda")
    Jk = torch.zeros(R, **f64)
    rn = torch.zeros((R, 2), **f64)
    y = torch.zeros((R, kk), **f64)
    dpsi = torch.zeros((R, p.nel), **f64)
    T.topo_rom_eval_batch(psi, Hel, Phid, kk, b, fd, Jk, rn, y, dpsi, filtered=filtered)
    T.topo_check()
    Jk_h, rn_h, y_h, dp_h = Jk.cpu().numpy(), rn.cpu().numpy(), y.cpu().numpy(), dpsi.cpu().numpy()
    # one-candidate calls
    rho = torch.empty(p.nel, **f64)
    F = fd.reshape(1, -1)
    for r in range(R):
        if filtered:
            T.topo_filter(psi[r], rho)
        else:
            rho.copy_(psi[r])
        Hw = torch.zeros(kk * kk, **f64)
        y1 = torch.zeros(kk, **f64)
        J1 = torch.zeros(1, **f64)
        T.topo_rom_solve_elem(rho, Hel, kk, b, Hw, y1, J1)
        rn1 = torch.zeros(2, **f64)
        uk = torch.zeros(p.ndof, **f64)
        T.topo_rom_error(rho, Phid, kk, y1, fd, rn1, uk)
        Jg = torch.zeros(1, **f64)
        dc = torch.zeros(p.nel, **f64)
        dp1 = torch.zeros(p.nel, **f64)
        T.topo_compliance_grad(rho, uk, F, Jg, dc, dp1 if filtered else None)
        T.topo_check()
        assert abs(Jk_h[r] - J1.item()) <= 1e-12 * abs(J1.item()), r
        assert np.abs(y_h[r] - y1.cpu().numpy()).max() <= 1e-10 * np.abs(y1.cpu().numpy()).max(), r
        assert abs(rn_h[r, 0] - rn1[0].item()) <= 1e-12 * rn1[0].item() + 1e-14, r
        assert abs(rn_h[r, 1] - rn1[1].item()) <= 1e-12 * rn1[1].item() + 1e-14, r
        g1 = (dp1 if filtered else dc).cpu().numpy()
        assert np.abs(dp_h[r] - g1).max() <= 1e-10 * np.abs(g1).max(), r
    # the oracle on a few candidates. J_k = y^T H y cancels heavily for snapshot bases (their
    # near-rigid components): two FP64 evaluations in different orders differ by up to about
    # eps |y|^T (|Phi|^T |K| |Phi|) |y|, which the tolerance adds to 1e-10 |J_k|.
    f = p.F[:, 0]
    mask = (p.fixed == 0).astype(float)
    for r in sorted({0, R // 2, R - 1}):
        rho_o = hatfilter.filter_fwd(p, cands[:, r]) if filtered else cands[:, r]
        ref = rom.rom_eval(p, rho_o, Phi, f)
        Kabs = abs(fem.assemble_K(p, rho_o)).multiply(mask[:, None]).multiply(mask[None, :]).tocsr()
        A = np.abs(Phi)
        ya = np.abs(ref["y"])
        rb = 2 * np.finfo(float).eps * (ya @ (A.T @ (Kabs @ A)) @ ya)
        assert abs(Jk_h[r] - ref["Jk"]) <= 1e-10 * abs(ref["Jk"]) + rb, (r, Jk_h[r], ref["Jk"], rb)
        dr = np.linalg.norm(rom.residual(p, rho_o, Phi @ y_h[r], f) - ref["r"])
        assert abs(rn_h[r, 0] - ref["resnorm"]) <= 1e-10 * ref["resnorm"] + dr + 1e-14 * np.linalg.norm(f), r
        dco = fem.compliance_grad_rho(p, rho_o, ref["uk"])
        go = hatfilter.filter_adj(p, dco) if filtered else dco
        assert np.abs(dp_h[r] - go).max() <= 1e-8 * np.abs(go).max(), r


def test_rom_eval_batch_is_independent_of_its_batch(torch):
    """A candidate's results are bitwise the same evaluated alone and inside a batch."""
    p = w.mbb_2d(37, 13)
    T, Phi, Phid, kk, Hel, b, fd, psi0, rng = _setup(torch, p, 6, 21)
    cands = w.perturbed_designs(p, psi0, 40, amplitude=0.02, first_seed=900)
    psi = dev(np.ascontiguousarray(cands.T))
    f64 = dict(dtype=torch.float64, device="cuda")
    out = []
    for sl in (slice(0, 40), slice(17, 18)):
        R = sl.stop - sl.start
        Jk, rn, dp = torch.zeros(R, **f64), torch.zeros((R, 2), **f64), torch.zeros((R, p.nel), **f64)
        T.topo_rom_eval_batch(psi[sl], Hel, Phid, kk, b, fd, Jk, rn, None, dp)
        out.append((Jk.cpu().numpy(), rn.cpu().numpy(), dp.cpu().numpy()))
    T.topo_check()
    assert out[0][0][17] == out[1][0][0]
    assert np.array_equal(out[0][1][17], out[1][1][0])
    assert np.array_equal(out[0][2][17], out[1][2][0])


def test_rom_eval_batch_invalid_arguments(torch):
    from paper_2004_05756_gb300 import native
    p = w.mbb_2d(20, 10)
    T = native.Topo(p)
    L = native.load()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    P = x.data_ptr()
    assert L.topo_rom_eval_batch(T.h, 0, P, p.nel, 1, P, P, 4, p.ndof, P, P, P, P, None, None) == native.TOPO_OK
    assert L.topo_rom_eval_batch(T.h, -1, P, p.nel, 1, P, P, 4, p.ndof, P, P, P, P, None, None) == native.TOPO_ERR_INVALID
    assert L.topo_rom_eval_batch(T.h, 2, P, p.nel - 1, 1, P, P, 4, p.ndof, P, P, P, P, None, None) == native.TOPO_ERR_INVALID
    assert L.topo_rom_eval_batch(T.h, 2, P, p.nel, 1, P, P, 0, p.ndof, P, P, P, P, None, None) == native.TOPO_ERR_INVALID
    assert L.topo_rom_eval_batch(T.h, 2, P, p.nel, 1, P, P, 4, p.ndof, P, P, P, P, None, P) == native.TOPO_ERR_INVALID
    assert L.topo_rom_eval_batch(T.h, 2, None, p.nel, 1, P, P, 4, p.ndof, P, P, P, P, None, None) == native.TOPO_ERR_INVALID
    T.topo_check()
