"""Serving form: continuous batching of design-evaluation requests. Each request's results
are bitwise the same alone and in the mix; one request is checked against the oracle; a tight
memory budget admits one request at a time."""
import numpy as np
import pytest

from oracle import fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu

REQS = [(2, (40, 20), 11), (3, (8, 8, 8), 12), (2, (64, 32), 13), (3, (12, 6, 6), 14), (2, (30, 15), 15),
        (3, (10, 5, 5), 16)]


def _requests():
    from paper_2004_05756_gb300.serving import Request
    return [Request(rid=i, dim=d, shape=s, seed=sd, arrival=0.01 * i) for i, (d, s, sd) in enumerate(REQS)]


def test_alone_equals_mix_bitwise():
    require_cuda()
    from paper_2004_05756_gb300.serving import Server
    srv = Server(slots=3)
    mix = {r.rid: r for r in srv.run(_requests(), realtime=True)}
    assert srv.max_concurrency >= 2  # requests did overlap
    for req in _requests():
        alone = Server(slots=3).run([req], realtime=False)[0]
        m = mix[req.rid]
        assert (alone.J, alone.theta, alone.Jk, alone.used_hdm) == (m.J, m.theta, m.Jk, m.used_hdm), req


def test_request_matches_oracle():
    require_cuda()
    from paper_2004_05756_gb300.serving import Request, Server
    d, shape, seed = REQS[0]
    res = Server(slots=1).run([Request(rid=0, dim=d, shape=shape, seed=seed)], realtime=False)[0]
    p = w.build_problem(d, shape)
    psi_c = w.design_field(p, seed)
    psi_x = w.perturbed_designs(p, psi_c, 1, amplitude=0.05, first_seed=seed % 100000 + 1)[:, 0]
    rho_c = hatfilter.filter_fwd(p, psi_c)
    rho_x = hatfilter.filter_fwd(p, psi_x)
    u_c = fem.solve(p, rho_c)[:, 0]
    Phi = rom.basis(u_c[:, None])
    ev = rom.rom_eval(p, rho_x, Phi, p.F[:, 0])
    assert res.theta == pytest.approx(ev["resnorm"], rel=1e-6)
    assert res.Jk == pytest.approx(ev["Jk"], rel=1e-8)
    delta = 0.1 * np.linalg.norm(p.F[:, 0])
    assert res.used_hdm == (ev["resnorm"] > delta)
    Jo = fem.compliance(p, fem.solve(p, rho_x)) if res.used_hdm else ev["Jk"]
    assert res.J == pytest.approx(Jo, rel=1e-8)


def test_admission_by_memory_budget():
    require_cuda()
    from paper_2004_05756_gb300.serving import Server, estimate_bytes
    reqs = _requests()
    biggest = max(estimate_bytes(r.dim, r.shape) for r in reqs)
    srv = Server(slots=3, budget_bytes=int(1.2 * biggest))
    out = srv.run(reqs, realtime=False)
    assert len(out) == len(reqs) and srv.max_concurrency == 1
