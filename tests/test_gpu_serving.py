"""Serving form: continuous batching of trust-region major iterations (Algorithm 2). Each
request's results are bitwise the same alone and in the mix; a standalone request and the
requests of a session are replayed against the oracle's major iterations; a tight memory budget
admits one request at a time; under a budget too small for all sessions at once, idle sessions
are spilled to host memory and restored with the same results."""
import numpy as np
import pytest

from oracle import trust
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu

REQS = [(2, (40, 20), 11), (3, (8, 8, 8), 12), (2, (64, 32), 13), (3, (12, 6, 6), 14), (2, (30, 15), 15),
        (3, (10, 5, 5), 16)]


def _requests():
    from paper_2004_05756_gb300.serving import Request
    return [Request(rid=i, dim=d, shape=s, seed=sd, arrival=0.01 * i) for i, (d, s, sd) in enumerate(REQS)]


FIELDS = ("J", "J_hat", "Jk", "Jk_c", "theta", "delta", "delta_next", "ratio", "accepted", "inside", "step", "k",
          "chi")


def _key(r):
    return tuple(getattr(r, f) for f in FIELDS)


def test_alone_equals_mix_bitwise():
    require_cuda()
    from paper_2004_05756_gb300.serving import Server
    srv = Server(slots=3)
    mix = {r.rid: r for r in srv.run(_requests(), realtime=True)}
    assert srv.max_concurrency >= 2  # requests did overlap
    for req in _requests():
        alone = Server(slots=3).run([req], realtime=False)[0]
        assert _key(alone) == _key(mix[req.rid]), req


def _compare(res, o, it=0):
    """A served major iteration against the oracle's: decisions equal, values within what their
    FP64 arithmetic allows (compliances to about 1e-10, the residual norm's cancellation)."""
    assert (res.step, res.inside, res.accepted, res.k) == (o["step"], o["inside"], o["accepted"], o["k"]), it
    assert res.J_hat == pytest.approx(o["J_hat"], rel=1e-10), it
    assert res.Jk == pytest.approx(o["Jk_hat"], rel=1e-9), it
    assert res.Jk_c == pytest.approx(o["Jk_c"], rel=1e-9), it
    assert res.theta == pytest.approx(o["theta_hat"], rel=1e-7), it
    assert res.delta == pytest.approx(o["delta"], rel=1e-14), it
    assert res.delta_next == pytest.approx(o["delta_next"], rel=1e-14), it
    pred = o["Jk_c"] - o["Jk_hat"]
    tol = 1e-9 * (abs(o["J_c"]) + abs(o["J_hat"]) + abs(o["ratio"]) * (abs(o["Jk_c"]) + abs(o["Jk_hat"])))
    assert abs(res.ratio - o["ratio"]) <= tol / pred, (it, res.ratio, o["ratio"])
    assert res.chi == pytest.approx(o["chi"], rel=1e-8), it


def test_request_matches_oracle():
    """A standalone request is one major iteration of a fresh run: the oracle's start and major
    iteration on the same seeded design give the same decisions and values."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Request, Server
    d, shape, seed = REQS[0]
    res = Server(slots=1, rtol=1e-13).run([Request(rid=0, dim=d, shape=shape, seed=seed)], realtime=False)[0]
    p = w.build_problem(d, shape)
    prm = trust.default_params(L=1)
    run = trust.start(p, w.design_field(p, seed), prm)
    _compare(res, trust.major_iteration(p, run, prm))
    assert res.rom_evals == prm["trials"] + 1


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
    """Sessions keep their run between requests: results are bitwise the same when a session
    runs alone and when its requests interleave with the others', the basis grows with every
    accepted step up to the window, and accepted steps decrease the compliance."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Server
    reqs = _session_requests()
    srv = Server(slots=3, kmax=4)
    # all requests queued at t = 0 (started in arrival order): the three sessions overlap
    mix = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert srv.max_concurrency >= 2
    for s in range(len(SESS)):
        mine = [r for r in _session_requests() if r.session == s]
        alone = sorted(Server(slots=3, kmax=4).run(mine, realtime=False), key=lambda r: r.index)
        for a in alone:
            assert _key(a) == _key(mix[a.rid]), (s, a.index)
        acc = 0
        J = None
        for a in alone:
            assert a.k == min(1 + acc, 4), (s, a.index, a.k, acc)
            if a.accepted:
                acc += 1
                assert a.J == a.J_hat and (J is None or a.J < J)
            J = a.J
        assert acc >= 2, [(a.ratio, a.accepted) for a in alone]


def test_session_requests_match_oracle():
    """Three requests of one session against three major iterations of the oracle's run."""
    require_cuda()
    from paper_2004_05756_gb300.serving import Request, Server
    d, shape = SESS[0]
    reqs = [Request(rid=t, dim=d, shape=shape, seed=100, arrival=0.0, session=0, step=t, last=t == 2)
            for t in range(3)]
    res = sorted(Server(slots=1, kmax=4, rtol=1e-13).run(reqs, realtime=False), key=lambda r: r.index)
    p = w.build_problem(d, shape)
    prm = trust.default_params(L=4)
    run = trust.start(p, w.design_field(p, 100), prm)
    for t in range(3):
        _compare(res[t], trust.major_iteration(p, run, prm), t)


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
        assert _key(a) == _key(b), rid
