"""Pins of the oracle's trust-region step (Algorithm 2) against what the mathematics fixes:
a hand-solved projection, the KKT conditions and the variational inequality of a Euclidean
projection onto a convex set, a general-purpose QP solver on small cases, the rows of the
radius rule, the model's exactness at the centre (Section 4.2: the centre's state lies in the
basis) and the first-order limit varrho_k -> 1 for short steps."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import fem, hatfilter, pipeline, rom, trust
from paper_2004_05756_gb300 import workloads as w


def test_projection_hand_case():
    # z = (1.2, 0.6, 0.1), vmax = 1: on mu in [0.2, 0.6] the volume is 1.8 - 2 mu, so mu = 0.4
    P, mu = trust.project(np.array([1.2, 0.6, 0.1]), 1.0)
    assert mu == pytest.approx(0.4, abs=1e-15)
    assert np.allclose(P, [0.8, 0.2, 0.0], atol=1e-15)


def test_projection_inactive_volume_is_box_clip():
    rng = np.random.default_rng(0)
    z = rng.uniform(-0.5, 1.5, 50)
    P, mu = trust.project(z, 50.0)
    assert mu == 0.0 and np.array_equal(P, np.clip(z, 0, 1))
    y = rng.uniform(0, 1, 40)
    y *= 10.0 / y.sum()
    P2, mu2 = trust.project(y, 10.0 + 1e-9)
    assert mu2 == 0.0 and np.array_equal(P2, y)  # a feasible point is its own projection


@pytest.mark.parametrize("seed", range(6))
def test_projection_kkt_and_variational_inequality(seed):
    rng = np.random.default_rng(seed)
    n = 200 + 37 * seed
    z = rng.normal(0.5, 0.8, n)
    vmax = 0.3 * n
    P, mu = trust.project(z, vmax)
    assert mu > 0
    assert np.all(P >= 0) and np.all(P <= 1)
    assert P.sum() == pytest.approx(vmax, rel=1e-13)
    assert np.allclose(P, np.clip(z - mu, 0, 1), atol=0, rtol=0)
    # (z - P) . (y - P) <= 0 for every feasible y
    for _ in range(200):
        y = rng.uniform(0, 1, n)
        if y.sum() > vmax:
            y *= vmax / y.sum()
        assert (z - P) @ (y - P) <= 1e-10


@pytest.mark.parametrize("seed", range(4))
def test_projection_matches_a_qp_solver(seed):
    rng = np.random.default_rng(100 + seed)
    n = 12
    z = rng.normal(0.6, 0.7, n)
    vmax = 0.4 * n
    P, _ = trust.project(z, vmax)
    res = so.minimize(lambda x: 0.5 * np.sum((x - z) ** 2), np.full(n, 0.4), jac=lambda x: x - z,
                      bounds=[(0, 1)] * n, constraints=[dict(type="ineq", fun=lambda x: vmax - x.sum(),
                                                             jac=lambda x: -np.ones(n))],
                      method="SLSQP", options=dict(ftol=1e-14, maxiter=500))
    assert res.success
    assert np.allclose(P, res.x, atol=1e-7)


def test_projection_exact_on_breakpoint_ties():
    # repeated values and a root exactly at a breakpoint
    z = np.array([1.5, 1.5, 0.5, 0.5, -0.2])
    P, mu = trust.project(z, 2.0)  # mu = 0.5 gives 1 + 1 + 0 + 0 + 0 = 2
    assert mu == pytest.approx(0.5, abs=1e-15) and np.allclose(P, [1, 1, 0, 0, 0], atol=1e-15)


def test_criticality_closed_forms():
    psi = np.full(10, 0.5)
    assert trust.criticality(psi, np.zeros(10), 6.0) == 0.0
    g = np.linspace(-0.1, 0.1, 10)  # sum(psi - g) = 5 <= 6 and inside the box: chi = ||g||
    assert trust.criticality(psi, g, 6.0) == pytest.approx(np.linalg.norm(g), rel=1e-15)


def test_ratio_and_radius_rule_rows():
    prm = trust.default_params()
    assert trust.ratio(10.0, 9.0, 10.0, 8.0) == 0.5
    assert trust.ratio(10.0, 9.0, 10.0, 10.0) == -np.inf  # no predicted reduction
    assert trust.ratio(10.0, 9.0, 10.0, 10.5) == -np.inf
    d, dmax = 2.0, 100.0
    assert trust.radius_update(-np.inf, d, dmax, prm) == (False, 1.0)
    assert trust.radius_update(0.0999, d, dmax, prm) == (False, 1.0)
    assert trust.radius_update(0.1, d, dmax, prm) == (True, 2.0)   # eta1 itself is accepted
    assert trust.radius_update(0.7499, d, dmax, prm) == (True, 2.0)
    assert trust.radius_update(0.75, d, dmax, prm) == (True, 4.0)  # eta2 itself is very successful
    assert trust.radius_update(3.0, 60.0, dmax, prm) == (True, 100.0)  # capped at Delta_max


def _problem():
    return w.mbb_2d(24, 8)


def test_start_is_feasible_and_scaled():
    p = _problem()
    prm = trust.default_params()
    run = trust.start(p, w.design_field(p, 3), prm)
    assert run.psi.sum() <= prm["volfrac"] * p.nel * (1 + 1e-14) and run.psi.min() >= 0 and run.psi.max() <= 1
    assert run.delta == pytest.approx(0.1 * np.linalg.norm(p.F[:, 0]), rel=1e-15)
    assert run.delta_max == 100 * run.delta
    assert run.J == pytest.approx(fem.compliance(p, fem.solve(p, hatfilter.filter_fwd(p, run.psi))), rel=1e-14)


def test_major_iteration_invariants():
    p = _problem()
    prm = trust.default_params()
    run = trust.start(p, w.design_field(p, 3), prm)
    vmax = prm["volfrac"] * p.nel
    J_prev = run.J
    accepted = 0
    for it in range(5):
        out = trust.major_iteration(p, run, prm)
        # the model is exact at the centre: the centre's state lies in the basis
        assert out["Jk_c"] == pytest.approx(out["J_c"], rel=1e-10)
        assert out["theta"][0] <= 1e-8 * np.linalg.norm(p.F[:, 0])
        # a descent direction, feasible target and candidate
        assert out["gtd"] < 0
        for q in (out["psi_x"], out["psi_hat"]):
            assert q.min() >= 0 and q.max() <= 1 and q.sum() <= vmax * (1 + 1e-13)
        # the selection rule: the taken trial passes both tests, every longer one fails one
        s = [0.0] + [2.0 ** -r for r in range(prm["trials"])]
        ok = [out["theta"][r] <= out["delta"] and out["Jk"][r] <= out["Jk_c"] + prm["c1"] * s[r] * out["gtd"]
              for r in range(len(s))]
        if out["inside"]:
            assert ok[out["sel"]] and not any(ok[1:out["sel"]])
        else:
            assert not any(ok[1:]) and out["sel"] == len(s) - 1
        # an accepted step decreases the full-order compliance
        if out["accepted"]:
            accepted += 1
            assert out["J_hat"] < J_prev and run.J == out["J_hat"]
            J_prev = run.J
        else:
            assert run.J == out["J_c"]
        assert out["chi"] >= 0
    assert accepted >= 3


def test_ratio_tends_to_one_for_short_steps():
    """m_k and J agree to first order at the centre (equal values and gradients, Section 4.2),
    so varrho_k -> 1 as the step shrinks; a sign or index error in either reduction breaks it."""
    p = _problem()
    prm = trust.default_params(move=1e-4)
    run = trust.start(p, w.design_field(p, 4), prm)
    out = trust.major_iteration(p, run, prm)
    assert out["inside"] and out["sel"] == 1
    assert abs(out["ratio"] - 1.0) < 2e-2, out["ratio"]


def test_rejected_step_keeps_centre_and_shrinks_radius():
    p = _problem()
    prm = trust.default_params()
    run = trust.start(p, w.design_field(p, 5), prm)
    run.delta = 1e-30  # no trial fits: the shortest is taken, whatever its ratio
    psi0, J0 = run.psi.copy(), run.J
    out = trust.major_iteration(p, run, prm)
    assert not out["inside"] and out["sel"] == prm["trials"]
    if not out["accepted"]:
        assert np.array_equal(run.psi, psi0) and run.J == J0 and run.delta == 0.5e-30
