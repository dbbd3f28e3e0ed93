"""Batched form: uneven instances solved in one persistent launch, each matching its own
single-instance solve and the oracle; batched filter, gradient and reduced solves."""
import numpy as np
import pytest

from oracle import fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, host_cols, relerr, require_cuda

pytestmark = pytest.mark.gpu


def _instances():
    # uneven sizes and load-case counts; one instance with a single element column
    shapes = [(20, 10, 1), (37, 13, 3), (60, 20, 2), (9, 4, 1), (48, 24, 5), (1, 3, 1)]
    out = []
    for i, (nx, ny, nlc) in enumerate(shapes):
        p = w.mbb_2d_multiload(nx, ny, nlc, seed=40 + i)
        psi = 0.3 + 0.7 * w.design_field(p, 50 + i)  # no void at the loads: FP64 floor << rtol
        out.append((p, psi))
    return out


@pytest.mark.parametrize("mg", [1, 0], ids=["multigrid", "jacobi"])
def test_batched_solve_matches_singles_and_oracle(mg):
    """Both launches of the batched solve: the multigrid one (default; the two smallest meshes
    do not coarsen and run the polynomial inside it) and the Jacobi one."""
    torch = require_cuda()
    from paper_2004_05756_gb300.native import Topo, TopoBatch, TOPO_PARAM_PCG_MG
    inst = _instances()
    B = TopoBatch([p for p, _ in inst])
    B.set_param(TOPO_PARAM_PCG_MG, mg)
    rhos = [dev(hatfilter.filter_fwd(p, psi)) for p, psi in inst]
    Fs = [cols(p.F) for p, _ in inst]
    Us = [torch.zeros_like(F) for F in Fs]
    infos = B.topo_batch_solve_hdm(rhos, Fs, Us, rtol=1e-13, maxit=100000)
    for i, (p, psi) in enumerate(inst):
        assert infos[i]["status"] == 0 and infos[i]["relres"] <= max(1e-13, infos[i]["floor"]), (i, infos[i])
        if mg and p.ndof > 400:
            assert infos[i]["mg_levels"] >= 2 and infos[i]["fallback"] == 0, (i, infos[i])
        if not mg:
            assert infos[i]["mg_levels"] == 0 and infos[i]["poly"] == 1, (i, infos[i])
        rho = rhos[i].cpu().numpy()
        Uo = fem.solve(p, rho)
        Ug = host_cols(Us[i])
        for c in range(p.F.shape[1]):
            Jo = fem.compliance(p, Uo[:, c], p.F[:, c])
            assert abs(fem.compliance(p, Ug[:, c], p.F[:, c]) - Jo) <= 1e-10 * abs(Jo), (i, c)
        T = Topo(p)
        Us1 = torch.zeros_like(Fs[i])
        T.topo_solve_hdm(rhos[i], Fs[i], Us1, rtol=1e-13, maxit=100000)
        assert relerr(Ug, host_cols(Us1)) < 1e-8
    # batched gradient and filter equal the single-instance calls
    J = torch.zeros(len(inst), dtype=torch.float64, device="cuda")
    dcs = [torch.zeros(p.nel, dtype=torch.float64, device="cuda") for p, _ in inst]
    dps = [torch.zeros(p.nel, dtype=torch.float64, device="cuda") for p, _ in inst]
    B.topo_batch_compliance_grad(rhos, Us, Fs, J, dcs, dps)
    for i, (p, psi) in enumerate(inst):
        Ug = host_cols(Us[i])
        assert abs(J[i].item() - fem.compliance(p, Ug)) <= 1e-12 * abs(J[i].item())
        dco = fem.compliance_grad_rho(p, rhos[i].cpu().numpy(), Ug)
        assert relerr(dcs[i].cpu().numpy(), dco) < 1e-9
    outs = [torch.zeros(p.nel, dtype=torch.float64, device="cuda") for p, _ in inst]
    B.topo_batch_filter([dev(psi) for _, psi in inst], outs)
    for i, (p, psi) in enumerate(inst):
        assert relerr(outs[i].cpu().numpy(), hatfilter.filter_fwd(p, psi)) < 1e-14


@pytest.mark.parametrize("ks", [[4, 6, 8, 3], [32, 16, 8, 1], [32, 16, 8, 40]],
                         ids=["small", "k_up_to_32", "one_k_above_32"])
def test_batched_rom_solve_elem(ks):
    """Reduced solves of every instance: bases up to 32 vectors take the three-launch path
    (all instances' assemblies in one launch, one warp per Cholesky), a basis above 32 the
    per-instance calls; both against the oracle's reduced solve, and the cached path of an
    identical second call bitwise equal to the first."""
    torch = require_cuda()
    from paper_2004_05756_gb300.native import TopoBatch
    inst = _instances()[:4]
    B = TopoBatch([p for p, _ in inst])
    from paper_2004_05756_gb300.native import load
    import ctypes
    rng = np.random.default_rng(3)
    rhos, Hels, bs, Hws, ys, refs = [], [], [], [], [], []
    for i, (p, psi) in enumerate(inst):
        k = min(ks[i], p.ndof)
        ks[i] = k
        Phi, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
        rho = rng.uniform(1e-3, 1, p.nel)
        npair = k * (k + 1) // 2
        Hel = torch.zeros((p.nel + 1) * npair, dtype=torch.float64, device="cuda")
        ctx = ctypes.c_void_p()
        load().topo_batch_context(B.h, i, ctypes.byref(ctx))
        load().topo_rom_elem(ctx, cols(Phi).data_ptr(), k, p.ndof, Hel.data_ptr())
        b = rng.standard_normal(k)
        H = Phi.T @ fem.apply_K(p, rho, Phi)
        refs.append(b @ rom.solve_reduced(0.5 * (H + H.T), b))
        rhos.append(dev(rho)); Hels.append(Hel); bs.append(dev(b))
        Hws.append(torch.zeros(k * k, dtype=torch.float64, device="cuda"))
        ys.append(torch.zeros(k, dtype=torch.float64, device="cuda"))
    Jk = torch.zeros(len(inst), dtype=torch.float64, device="cuda")
    B.topo_batch_rom_solve_elem(rhos, Hels, ks, bs, Hws, ys, Jk)
    first = Jk.cpu().numpy().copy()
    for i in range(len(inst)):
        assert abs(first[i] - refs[i]) <= 1e-10 * abs(refs[i]), (i, ks[i], first[i], refs[i])
    B.topo_batch_rom_solve_elem(rhos, Hels, ks, bs, Hws, ys, Jk)
    assert np.array_equal(Jk.cpu().numpy(), first)


def test_batched_step_in_cuda_graph():
    """The batched design evaluation (filter, all state solves in one persistent launch,
    gradient) captured in a CUDA graph after one eager call: a replay on new designs written
    into the same buffers gives bitwise the eager results, which match the oracle."""
    torch = require_cuda()
    from paper_2004_05756_gb300 import native
    from paper_2004_05756_gb300.native import TopoBatch
    inst = _instances()
    probs = [p for p, _ in inst]
    stream = torch.cuda.Stream()
    f64 = dict(dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        B = TopoBatch(probs, stream=stream)
        psis = [dev(psi) for _, psi in inst]
        rhos = [torch.zeros(p.nel, **f64) for p in probs]
        Fs = [cols(p.F) for p in probs]
        Us = [torch.zeros_like(F) for F in Fs]
        J = torch.zeros(len(probs), **f64)
        dcs = [torch.zeros(p.nel, **f64) for p in probs]
        dps = [torch.zeros(p.nel, **f64) for p in probs]

        def body():
            B.topo_batch_filter(psis, rhos)
            for U in Us:
                U.zero_()
            B.topo_batch_solve_hdm(rhos, Fs, Us, rtol=1e-13, maxit=100000, info=False)
            B.topo_batch_compliance_grad(rhos, Us, Fs, J, dcs, dps)

        body()  # eager: autotunes and stages the launch tables
        body()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        n0 = native.launch_count()
        with torch.cuda.graph(g, stream=stream):
            body()
        assert native.launch_count() - n0 >= 1  # the captured calls launched library kernels
        # new designs into the captured buffers, then replay
        new = [0.3 + 0.7 * w.design_field(p, 90 + i) for i, p in enumerate(probs)]
        for t, x in zip(psis, new):
            t.copy_(torch.as_tensor(x))
        g.replay()
        stream.synchronize()
        Jg = J.clone()
        dg = [d.clone() for d in dps]
        body()  # eager on the same designs
        stream.synchronize()
    assert torch.equal(Jg, J)
    for a, b in zip(dg, dps):
        assert torch.equal(a, b)
    for i, p in enumerate(probs):
        rho = hatfilter.filter_fwd(p, new[i])
        Jo = fem.compliance(p, fem.solve(p, rho))
        assert abs(Jg[i].item() - Jo) <= 1e-10 * abs(Jo), (i, Jg[i].item(), Jo)
