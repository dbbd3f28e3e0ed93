"""Serving form: continuous batching of design-evaluation requests. Each request's results
are bitwise the same alone and in the mix; one request is checked against the oracle; a tight
memory budget admits one request at a time; under a budget too small for all sessions at once,
idle sessions are spilled to host memory and restored with the same results."""
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


def _oracle_step(p, psi_c, psi_x, Phi, halvings=6):
    """The candidate of a request by the oracle: the largest step s = 1, 1/2, ... toward the
    proposal whose reduced residual satisfies theta <= 0.1 ||f||, else the proposal itself by
    a direct solve. Returns (s, theta, J_k, J, fallback)."""
    f = p.F[:, 0]
    delta = 0.1 * np.linalg.norm(f)
    s, first = 1.0, None
    for h in range(halvings + 1):
        psi = psi_x if h == 0 else psi_c + s * (psi_x - psi_c)
        ev = rom.rom_eval(p, hatfilter.filter_fwd(p, psi), Phi, f)
        if first is None:
            first = ev
        if ev["resnorm"] <= delta:
            return s, ev["resnorm"], ev["Jk"], ev["Jk"], False
        s *= 0.5
    rho_x = hatfilter.filter_fwd(p, psi_x)
    return 1.0, first["resnorm"], first["Jk"], fem.compliance(p, fem.solve(p, rho_x)), True


def test_request_matches_oracle():
    require_cuda()
    from paper_2004_05756_gb300.serving import Request, Server
    d, shape, seed = REQS[0]
    res = Server(slots=1).run([Request(rid=0, dim=d, shape=shape, seed=seed)], realtime=False)[0]
    p = w.build_problem(d, shape)
    psi_c = w.design_field(p, seed)
    psi_x = w.perturbed_designs(p, psi_c, 1, amplitude=0.05, first_seed=seed % 100000 + 1)[:, 0]
    u_c = fem.solve(p, hatfilter.filter_fwd(p, psi_c))[:, 0]
    Phi = rom.basis(u_c[:, None])
    s, theta, Jk, J, fallback = _oracle_step(p, psi_c, psi_x, Phi)
    assert res.step == s and res.used_hdm == fallback
    assert res.theta == pytest.approx(theta, rel=1e-6)
    assert res.Jk == pytest.approx(Jk, rel=1e-8)
    assert res.J == pytest.approx(J, rel=1e-8)


def test_admission_by_memory_budget():
    require_cuda()
    from paper_2004_05756_gb300.serving import Server, estimate_bytes
    reqs = _requests()
    biggest = max(estimate_bytes(r.dim, r.shape) for r in reqs)
    srv = Server(slots=3, budget_bytes=int(1.2 * biggest))
    out = srv.run(reqs, realtime=False)
    assert len(out) == len(reqs) and srv.max_concurrency == 1


SESS = [(2, (40, 20)), (3, (8, 8, 8)), (2, (30, 15))]


def _session_requests(steps=4):
    from paper_2004_05756_gb300.serving import Request
    out = []
    for t in range(steps):
        for s, (d, shape) in enumerate(SESS):
            out.append(Request(rid=len(out), dim=d, shape=shape, seed=100 + s, arrival=0.01 * len(out), session=s,
                               step=t, last=t == steps - 1))
    return out


def test_sessions_alone_equal_mix_and_basis_grows():
    """Sessions keep their basis between requests: results are bitwise the same when a
    session runs alone and when its requests interleave with the others', the basis grows
    with the session, and the reduced model takes over from the full-order fallback."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Server
    reqs = _session_requests()
    srv = Server(slots=3, kmax=4)
    # all requests queued at t = 0 (started in arrival order): the three sessions overlap
    mix = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert srv.max_concurrency >= 2
    for s in range(len(SESS)):
        mine = [r for r in _session_requests() if r.session == s]
        alone = Server(slots=3, kmax=4).run(mine, realtime=False)
        for a in alone:
            m = mix[a.rid]
            assert (a.J, a.theta, a.Jk, a.used_hdm, a.k, a.step) == (m.J, m.theta, m.Jk, m.used_hdm, m.k, m.step), \
                (s, a.index)
        assert [a.k for a in sorted(alone, key=lambda r: r.index)] == [1, 2, 3, 4]
    # the trust-region step search finds admissible candidates: the reduced model answers
    assert sum(not r.used_hdm for r in mix.values()) >= len(mix) // 2, \
        [(r.session, r.index, r.step, r.theta / r.delta) for r in mix.values()]


def test_session_request_matches_oracle():
    """Step 1 of a session: a two-snapshot window (centres of steps 0 and 1), the reduced
    evaluation at the candidate, against the oracle's direct solves and reduced model."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Request, Server
    d, shape = SESS[0]
    reqs = [Request(rid=t, dim=d, shape=shape, seed=100, arrival=0.0, session=0, step=t, last=t == 1)
            for t in range(2)]
    res = sorted(Server(slots=1, kmax=4).run(reqs, realtime=False), key=lambda r: r.index)[1]
    p = w.build_problem(d, shape)
    psi0 = w.design_field(p, 100)
    psi1 = w.perturbed_designs(p, psi0, 1, amplitude=0.02, first_seed=w.seed_for("walk100", 2))[:, 0]
    psix = w.perturbed_designs(p, psi1, 1, amplitude=0.05, first_seed=w.seed_for("walk100", 3))[:, 0]
    U = np.stack([fem.solve(p, hatfilter.filter_fwd(p, q))[:, 0] for q in (psi0, psi1)], 1)
    Phi = rom.basis(U)
    s, theta, Jk, J, fallback = _oracle_step(p, psi1, psix, Phi)
    assert res.k == Phi.shape[1] == 2
    assert res.step == s and res.used_hdm == fallback
    assert res.theta == pytest.approx(theta, rel=1e-6)
    assert res.Jk == pytest.approx(Jk, rel=1e-7)
    assert res.J == pytest.approx(J, rel=1e-7)


def test_idle_sessions_evicted_under_memory_pressure_same_results():
    """A budget that holds the largest session and little more: sessions are admitted by
    evicting idle ones (state copied to pinned host memory, device memory freed) and restored
    for their next request. Every result equals the run with room for all sessions, bitwise."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Server, estimate_bytes
    reqs = _session_requests(steps=3)
    roomy = Server(slots=3, kmax=4)
    ref = {r.rid: r for r in roomy.run(reqs, realtime=False)}
    assert roomy.evictions == 0
    need = {s: estimate_bytes(d, shape, 4) for s, (d, shape) in enumerate(SESS)}
    budget = max(need.values()) + min(need.values()) // 2
    tight = Server(slots=3, kmax=4, budget_bytes=budget)
    got = {r.rid: r for r in tight.run(_session_requests(steps=3), realtime=False)}
    assert tight.evictions >= 1 and tight.restores >= 1, (tight.evictions, tight.restores)
    assert tight.in_use == 0 and not tight.sessions
    assert set(got) == set(ref)
    for rid, a in ref.items():
        b = got[rid]
        assert (a.J, a.theta, a.Jk, a.used_hdm, a.k, a.step) == (b.J, b.theta, b.Jk, b.used_hdm, b.k, b.step), rid
