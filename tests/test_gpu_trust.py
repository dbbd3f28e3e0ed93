"""The trust-region step of Algorithm 2 through the C ABI, against the oracle (oracle/trust.py):

* topo_tr_project against the oracle's exact projection onto the feasible set, on meshes of one
  to many tiles with ragged tails, with and without a gradient step, with the volume bound
  active, inactive, zero or infinite, and on designs with many tied values;
* topo_tr_trials bit for bit against psi_c + s (psi_x - psi_c);
* topo_tr_select and topo_tr_update on crafted values, row by row of the selection and radius
  rules, including a predicted reduction that is not positive and a NaN compliance;
* a whole run (TrustRegionRun) replayed against the oracle's major iterations: the selected
  trial, acceptance and radius of every iteration equal, and varrho_k, the compliances and the
  designs within the bounds their FP64 arithmetic allows.
"""
import math

import numpy as np
import pytest

from oracle import hatfilter, trust
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import dev, require_cuda

pytestmark = pytest.mark.gpu

MESHES = {
    "q4_24x8": lambda: w.mbb_2d(24, 8),          # 192 elements: part of one tile
    "q4_130x41": lambda: w.mbb_2d(130, 41),      # 5,330: three tiles, ragged
    "q4_300x100": lambda: w.mbb_2d(300, 100),    # 30,000: fifteen tiles
    "h8_11x9x6": lambda: w.cantilever_3d(11, 9, 6),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _ctx(p):
    from paper_2004_05756_gb300.native import Topo
    return Topo(p)


def _project(T, psi, g, t, scaled, vmax):
    import torch as th
    out = th.empty(len(psi), dtype=th.float64, device="cuda")
    stats = th.zeros(4, dtype=th.float64, device="cuda")
    T.topo_tr_project(dev(psi), None if g is None else dev(g), t, scaled, vmax, out, stats)
    T.topo_check()
    return out.cpu().numpy(), stats.cpu().numpy()


def _check_projection(P, stats, z, psi, g, vmax):
    Po, mu = trust.project(z, vmax)
    assert np.max(np.abs(P - Po)) <= 1e-13 * max(1.0, abs(mu)), np.max(np.abs(P - Po))
    assert abs(stats[2] - mu) <= 1e-13 * max(1.0, abs(mu))
    d = Po - psi
    assert stats[1] == pytest.approx(np.linalg.norm(d), rel=1e-11, abs=1e-300)
    if g is not None:
        assert stats[0] == pytest.approx(g @ d, rel=1e-11, abs=1e-13 * np.abs(g).sum())
    assert stats[3] == pytest.approx(Po.sum(), rel=1e-13)
    if mu > 0:
        assert stats[3] <= vmax * (1 + 1e-13)


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("case", ["plain", "scaled", "unit", "inactive", "infinite", "zero", "ties"])
def test_project_matches_oracle(torch, mesh, case):
    p = MESHES[mesh]()
    T = _ctx(p)
    rng = np.random.default_rng(abs(hash((mesh, case))) % 2 ** 32)
    psi = w.design_field(p, 7)
    g = None
    vmax = 0.5 * p.nel
    if case == "plain":
        psi = rng.normal(0.5, 0.6, p.nel)
        t, scaled = 0.0, False
    elif case == "scaled":
        g = rng.normal(0, 1, p.nel) * np.exp(rng.normal(0, 2, p.nel))
        t, scaled = 0.2, True
    elif case == "unit":
        g = -np.abs(rng.normal(0, 3, p.nel))  # compliance gradients are non-positive
        t, scaled = 1.0, False
    elif case == "inactive":
        g = rng.normal(0, 0.01, p.nel)
        t, scaled, vmax = 1.0, False, 0.99 * p.nel
    elif case == "infinite":
        psi = rng.normal(0.5, 0.6, p.nel)
        t, scaled, vmax = 0.0, False, math.inf
    elif case == "zero":
        t, scaled, vmax = 0.0, False, 0.0
    else:  # many equal values: breakpoints shared by hundreds of elements
        psi = np.round(rng.uniform(-0.2, 1.4, p.nel), 1)
        t, scaled, vmax = 0.0, False, 0.3 * p.nel
    P, stats = _project(T, psi, g, t, scaled, vmax)
    if g is None:
        z = psi
    else:
        tau = t / np.max(np.abs(g)) if scaled else t
        z = psi - tau * g
    _check_projection(P, stats, z, psi, g, vmax)
    if case == "zero":
        assert not P.any()
    if case in ("inactive", "infinite"):
        assert stats[2] == 0.0 and np.array_equal(P, np.clip(z, 0, 1))


def test_project_in_place_and_deterministic(torch):
    import torch as th
    p = MESHES["q4_130x41"]()
    T = _ctx(p)
    psi = np.random.default_rng(3).normal(0.5, 0.6, p.nel)
    g = np.random.default_rng(4).normal(0, 1, p.nel)
    ref, st_ref = _project(T, psi, g, 0.3, True, 0.4 * p.nel)
    for _ in range(3):
        P, st = _project(T, psi, g, 0.3, True, 0.4 * p.nel)
        assert np.array_equal(P, ref) and np.array_equal(st, st_ref)
    x = dev(psi)
    stats = th.zeros(4, dtype=th.float64, device="cuda")
    T.topo_tr_project(x, dev(g), 0.3, True, 0.4 * p.nel, x, stats)
    assert np.array_equal(x.cpu().numpy(), ref)


def test_trials_bitwise(torch):
    import torch as th
    p = MESHES["q4_130x41"]()
    T = _ctx(p)
    rng = np.random.default_rng(5)
    pc, px = rng.uniform(0, 1, p.nel), rng.uniform(0, 1, p.nel)
    R = 8
    trials = th.empty((R, p.nel), dtype=th.float64, device="cuda")
    T.topo_tr_trials(dev(pc), dev(px), trials)
    got = trials.cpu().numpy()
    d = px - pc
    for r in range(R):
        s = 0.0 if r == 0 else 2.0 ** -(r - 1)
        assert np.array_equal(got[r], pc + s * d), r


def _state(**kw):
    import ctypes
    from paper_2004_05756_gb300 import native
    s = native.topo_tr_state()
    for k, v in kw.items():
        setattr(s, k, v)
    buf = np.frombuffer(bytes(s), dtype=np.float64).copy()
    return dev(buf)


SELECT_CASES = [
    # (delta, Jk, theta, gtd, expected sel, inside)
    (1.0, [10, 9, 9.5, 9.8], [0, 0.5, 0.3, 0.1], -1.0, 1, 1),      # the full step fits
    (0.4, [10, 9, 9.5, 9.8], [0, 0.5, 0.3, 0.1], -1.0, 2, 1),      # outside the region, then inside
    (1.0, [10, 10.5, 9.9, 9.8], [0, 0.1, 0.1, 0.1], -1.0, 2, 1),   # no decrease, then decrease
    (1.0, [10, 10, 10, 10], [0, 0.1, 0.1, 0.1], -1.0, 3, 0),       # Armijo fails everywhere
    (0.05, [10, 9, 9.5, 9.8], [0, 0.5, 0.3, 0.1], -1.0, 3, 0),     # nothing inside the region
    (1.0, [10, float("nan"), 9.5, 9.8], [0, 0.1, 0.1, 0.1], -1.0, 2, 1),  # a failed reduced solve
]


@pytest.mark.parametrize("case", range(len(SELECT_CASES)))
def test_select_rule(torch, case):
    import torch as th
    from paper_2004_05756_gb300 import native
    p = MESHES["q4_24x8"]()
    T = _ctx(p)
    delta, Jk, theta, gtd, sel_exp, inside_exp = SELECT_CASES[case]
    R, k = len(Jk), 3
    rng = np.random.default_rng(case)
    st = _state(delta=delta)
    res = np.zeros((R, 2))
    res[:, 0] = theta
    trials = dev(rng.uniform(0, 1, (R, p.nel)))
    Phi = dev(rng.normal(0, 1, (k, p.ndof)))
    yhat = dev(rng.normal(0, 1, R * k))
    psi_hat = th.empty(p.nel, dtype=th.float64, device="cuda")
    u_hat = th.empty(p.ndof, dtype=th.float64, device="cuda")
    prm = native.tr_params(c1=0.1)
    T.topo_tr_select(st, prm, dev(np.array(Jk, float)), dev(res), dev(np.array([gtd])), trials, Phi, k, yhat,
                     psi_hat, u_hat)
    s = native.tr_state_read(st)
    assert (s["sel"], s["inside"]) == (sel_exp, inside_exp)
    assert s["step"] == 2.0 ** -(sel_exp - 1) and s["gtd"] == gtd
    assert s["Jk_c"] == Jk[0] and s["theta_hat"] == theta[sel_exp]
    assert np.array_equal(psi_hat.cpu().numpy(), trials[sel_exp].cpu().numpy())
    y = yhat.cpu().numpy()[sel_exp * k:(sel_exp + 1) * k]
    assert np.allclose(u_hat.cpu().numpy(), Phi.cpu().numpy().T @ y, rtol=1e-14, atol=1e-13)


UPDATE_CASES = [
    # (J_c, J_hat, Jk_c, Jk_hat, delta)
    (10.0, 9.95, 10.0, 9.0, 2.0),     # varrho = 0.05: rejected, shrink
    (10.0, 9.5, 10.0, 9.0, 2.0),      # 0.5: accepted, same radius
    (10.0, 9.1, 10.0, 9.0, 2.0),      # 0.9: accepted, grow
    (10.0, 9.1, 10.0, 9.0, 80.0),     # 0.9 near Delta_max: capped
    (10.0, 9.0, 10.0, 10.0, 2.0),     # no predicted reduction: -inf, rejected
    (10.0, 9.0, 10.0, 10.5, 2.0),     # a model increase: -inf, rejected
    (10.0, 9.875, 10.0, 8.75, 2.0),   # varrho = 0.125 / 1.25 = eta1 in FP64: accepted
    (10.0, float("nan"), 10.0, 9.0, 2.0),  # a failed full-order solve: rejected, shrink
]


@pytest.mark.parametrize("case", range(len(UPDATE_CASES)))
def test_update_rule_rows(torch, case):
    import torch as th
    from paper_2004_05756_gb300 import native
    p = MESHES["q4_24x8"]()
    T = _ctx(p)
    J_c, J_hat, Jk_c, Jk_hat, delta = UPDATE_CASES[case]
    st = _state(delta=delta, delta_max=100.0, J_c=J_c, Jk_c=Jk_c, Jk_hat=Jk_hat, iter=4)
    rng = np.random.default_rng(10 + case)
    bufs = {n: rng.normal(0, 1, p.nel if n.startswith(("psi", "g")) else p.ndof)
            for n in ("psi_c", "psi_hat", "u_c", "u_hat", "g_c", "g_hat", "slot")}
    d = {n: dev(v) for n, v in bufs.items()}
    T.topo_tr_update(st, native.tr_params(), dev(np.array([J_hat])), d["psi_c"], d["psi_hat"], d["u_c"],
                     d["u_hat"], d["g_c"], d["g_hat"], d["slot"])
    s = native.tr_state_read(st)
    prm = trust.default_params()
    ratio = trust.ratio(J_c, J_hat, Jk_c, Jk_hat)
    acc, dn = trust.radius_update(ratio, delta, 100.0, prm)
    if math.isnan(ratio):
        assert math.isnan(s["ratio"])
    else:
        assert s["ratio"] == ratio
    assert (bool(s["accepted"]), s["delta"], s["delta_prev"], s["iter"]) == (acc, dn, delta, 5)
    assert s["J_c"] == (J_hat if acc else J_c)
    for c, h in (("psi_c", "psi_hat"), ("u_c", "u_hat"), ("g_c", "g_hat"), ("slot", "u_hat")):
        assert np.array_equal(d[c].cpu().numpy(), bufs[h] if acc else bufs[c]), c


def test_init(torch):
    import torch as th
    from paper_2004_05756_gb300 import native
    p = MESHES["q4_130x41"]()
    T = _ctx(p)
    st = native.tr_state_tensor()
    f = p.F[:, 0].copy()
    f[np.flatnonzero(p.fixed)[:3]] = 5.0  # values on Dirichlet DOFs do not count
    T.topo_tr_init(st, dev(f), 0.1, 100.0, dev(np.array([123.5])))
    s = native.tr_state_read(st)
    ref = 0.1 * np.linalg.norm(p.F[:, 0][p.fixed == 0])
    assert s["delta"] == pytest.approx(ref, rel=1e-15) and s["delta_max"] == 100.0 * s["delta"]
    assert s["J_c"] == 123.5 and s["iter"] == 0 and s["accepted"] == 0


def test_parameter_validation(torch):
    import torch as th
    from paper_2004_05756_gb300 import native
    from paper_2004_05756_gb300.native import TopoError
    p = MESHES["q4_24x8"]()
    T = _ctx(p)
    x = th.zeros(p.nel, dtype=th.float64, device="cuda")
    stats = th.zeros(4, dtype=th.float64, device="cuda")
    with pytest.raises(TopoError):
        T.topo_tr_project(x, None, 0.0, False, -1.0, x.clone(), stats)
    with pytest.raises(TopoError):
        T.topo_tr_project(x, x, 1.0, False, 1.0, x, stats)  # out aliases g
    with pytest.raises(TopoError):
        T.topo_tr_trials(x, x, th.zeros((1, p.nel), dtype=th.float64, device="cuda"))
    st = native.tr_state_tensor()
    one = th.ones(1, dtype=th.float64, device="cuda")
    for bad in (native.tr_params(gamma1=0.0), native.tr_params(eta1=0.8), native.tr_params(grow=0.5),
                native.tr_params(gamma2=1.5)):
        with pytest.raises(TopoError):
            T.topo_tr_update(st, bad, one, x, x, x, x, x, x)
    with pytest.raises(TopoError):
        T.topo_tr_init(st, th.zeros(p.ndof, dtype=th.float64, device="cuda"), 0.0, 100.0, one)


RUNS = [("q4", (48, 16), 3, 6, None), ("h8", (8, 6, 4), 5, 4, None), ("q4_pod", (48, 16), 3, 7, 2),
        ("h8_pod", (8, 6, 4), 5, 6, 2)]


def _margins(o, prm):
    """Relative distance of every decision of one oracle iteration from its threshold."""
    s = [0.0] + [2.0 ** -r for r in range(prm["trials"])]
    m = []
    for r in range(1, o["sel"] + 1):
        m.append(abs(o["theta"][r] - o["delta"]) / o["delta"])
        rhs = o["Jk_c"] + prm["c1"] * s[r] * o["gtd"]
        m.append(abs(o["Jk"][r] - rhs) / abs(o["Jk_c"]))
    if np.isfinite(o["ratio"]):
        m += [abs(o["ratio"] - prm["eta1"]), abs(o["ratio"] - prm["eta2"])]
    return min(m)


@pytest.mark.parametrize("run", RUNS, ids=[r[0] for r in RUNS])
def test_run_replays_oracle(torch, run):
    """Every major iteration of a run on the device against the oracle's, from the same start."""
    from paper_2004_05756_gb300.trust_region import TrustRegionRun
    kind, shape, seed, iters, n_max = run
    p = w.build_problem(2 if kind.startswith("q4") else 3, shape)
    psi0 = w.design_field(p, seed)
    L = 4 if n_max is None else 3
    prm = trust.default_params(L=L, n_max=n_max)
    orc = trust.start(p, psi0, prm)
    T = _ctx(p)
    gpu = TrustRegionRun(T, p, psi0, L=L, rtol=1e-13, pod_nmax=n_max)
    s0 = gpu.state()
    assert s0["J_c"] == pytest.approx(orc.J, rel=1e-10)
    assert s0["delta"] == pytest.approx(orc.delta, rel=1e-14)
    assert np.max(np.abs(gpu.psi_c.cpu().numpy() - orc.psi)) <= 1e-13
    accepted = 0
    for it in range(iters):
        o = trust.major_iteration(p, orc, prm)
        assert _margins(o, prm) > 1e-7, (it, "the seeded run has a near-tie; pick another seed")
        g = gpu.iterate()
        assert g["k"] == o["k"], it
        assert (g["sel"], bool(g["inside"]), bool(g["accepted"])) == (o["sel"], o["inside"], o["accepted"]), it
        assert g["step"] == o["step"]
        assert g["Jk_c"] == pytest.approx(o["Jk_c"], rel=1e-9), it
        assert g["Jk_hat"] == pytest.approx(o["Jk_hat"], rel=1e-9), it
        assert g["J_hat"] == pytest.approx(o["J_hat"], rel=1e-10), it
        assert g["theta_hat"] == pytest.approx(o["theta_hat"], rel=1e-7), it
        assert g["gtd"] == pytest.approx(o["gtd"], rel=1e-10), it
        # varrho_k: the compliances carry relative errors of about 1e-10; the bound follows
        pred = o["Jk_c"] - o["Jk_hat"]
        if np.isfinite(o["ratio"]):
            tol = 1e-9 * (abs(o["J_c"]) + abs(o["J_hat"]) + abs(o["ratio"]) * (abs(o["Jk_c"]) + abs(o["Jk_hat"])))
            assert abs(g["ratio"] - o["ratio"]) <= tol / pred, (it, g["ratio"], o["ratio"])
        else:
            assert g["ratio"] == -math.inf
        assert g["delta_prev"] == pytest.approx(o["delta"], rel=1e-14)
        assert g["delta"] == pytest.approx(o["delta_next"], rel=1e-14)
        assert g["chi"] == pytest.approx(o["chi"], rel=1e-8), it
        assert np.max(np.abs(gpu.psi_c.cpu().numpy() - orc.psi)) <= 1e-10, it
        accepted += int(o["accepted"])
    assert accepted >= 2
    assert gpu.state()["iter"] == iters
