"""One major iteration of the error-aware trust-region method (Algorithm 2, Section 4.2) for
compliance, in plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): it restates the steps in the paper's
order so that the library's trust-region calls can be replayed against it.

Pieces, each following the passage named in its docstring:
  project        -- Euclidean projection onto the feasible set C of Eq. feaset-topopt
  criticality    -- ||psi - P_C(psi - grad J)||, the stopping measure of Section 4.1
  ratio          -- the actual-to-predicted reduction varrho_k (Algorithm 2, step 4)
  radius_update  -- step acceptance and trust-region update (Algorithm 2, steps 5 and 6)
  start          -- a run's initial state (Section 5: Delta_0 = tau ||r(0, rho(psi_0))||)
  major_iteration-- model update, step computation, ratio, acceptance, radius

Readings where the paper leaves a choice (each is one line of the design notes):
  * Unit element volumes (every element of the benchmark meshes is a unit square or cube), so
    C = {psi in [0,1]^Ne : sum_e psi_e <= vmax} with vmax = volfrac * Ne.
  * The subproblem (Algorithm 2, step 3) is solved approximately by one projected-gradient
    step with backtracking, standing in for the paper's MMA: the target
    psi_x = P_C(psi_c - (move / ||g||_inf) g) with g = grad J(psi_c) = grad m_k(psi_c), trial
    steps psi_c + s (psi_x - psi_c) for s = 1, 1/2, ..., 2^-(trials-1), and the largest s that
    lies in the error-aware trust region (theta <= Delta, Eq. trcon-topopt) and decreases the
    model by the Armijo rule m_k(psi_s) <= m_k(psi_c) + c1 s g.(psi_x - psi_c) (Bertsekas,
    Nonlinear Programming, Section 2.3: the Armijo rule along a feasible direction). When no
    trial passes both tests, the shortest trial is the candidate. The segment stays in C
    because C is convex.
  * varrho_k = -inf when the predicted reduction m_k(psi_c) - m_k(psi_hat) is not positive
    (the ratio then carries no information and the step is rejected).
  * Inside the intervals of the radius rule the update takes gamma1 Delta when varrho < eta1,
    gamma2 Delta when eta1 <= varrho < eta2, and min(grow Delta, Delta_max) when
    varrho >= eta2 (Section 5 fixes gamma1 = 0.5, gamma2 = 1, eta1 = 0.1, eta2 = 0.75,
    Delta_max = 100 Delta_0; grow = 2 is not given by the paper).
  * The reduced basis is the orthonormalisation of the L most recent centre snapshots, the
    newest being the current centre's (Eq. rob-optim with every POD vector of the window
    kept; for compliance the adjoint snapshots equal the primal ones). A rejected step adds
    no snapshot, since the centre does not move. With prm["n_max"] set, the basis is Eq.
    rob-optim with POD truncation instead: GramSchmidt([POD_n(U_prev), u_c]) where U_prev holds
    the L most recent previous centres and n = min(number of previous centres - 1, n_max)
    (n_k = min(k - 1, n_max) of Section 4.2, k previous centres).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fem, pipeline, rom

PAPER_CONSTANTS = dict(tau=0.1, gamma1=0.5, gamma2=1.0, eta1=0.1, eta2=0.75, dmax_factor=100.0)


def project(z: np.ndarray, vmax: float) -> tuple[np.ndarray, float]:
    """P_C(z) = argmin_{psi in C} ||psi - z||_2 for C = [0,1]^Ne intersected with
    {sum psi <= vmax} (Eq. feaset-topopt, unit element volumes). Returns (P_C(z), mu).

    The KKT conditions of the projection give psi = clip(z - mu, 0, 1) with a multiplier
    mu >= 0 of the volume constraint and mu (sum psi - vmax) = 0. If the box projection clip(z)
    already satisfies the volume bound, mu = 0. Otherwise mu is the root of
    v(mu) = sum_e clip(z_e - mu, 0, 1) - vmax, which is continuous, piecewise linear and
    nonincreasing with breakpoints {z_e, z_e - 1}. The root is located exactly: bisection over
    the sorted breakpoints finds the piece [a, b] on which v changes sign, and on that piece
    every element is either saturated (z_e - mu >= 1 throughout), void (z_e - mu <= 0
    throughout) or linear (z_e - mu in [0, 1] throughout), so
    mu = (n_sat + sum_{linear} z_e - vmax) / n_linear."""
    z = np.asarray(z, dtype=float)
    if vmax < 0:
        raise ValueError("vmax must be non-negative")

    def v(mu):
        return float(np.clip(z - mu, 0.0, 1.0).sum()) - vmax

    if v(0.0) <= 0.0:
        return np.clip(z, 0.0, 1.0), 0.0
    bp = np.unique(np.concatenate([z, z - 1.0]))
    bp = bp[bp > 0.0]
    # v(0) > 0 and v(max z) = -vmax <= 0; find the first breakpoint where v <= 0
    lo, hi = -1, len(bp) - 1  # v > 0 at 0 (index -1 stands for mu = 0), v <= 0 at bp[hi]
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if v(bp[mid]) <= 0.0:
            hi = mid
        else:
            lo = mid
    a = 0.0 if lo < 0 else bp[lo]
    b = bp[hi]
    c = 0.5 * (a + b)
    sat = z - c >= 1.0
    lin = (z - c > 0.0) & (z - c < 1.0)
    n = int(lin.sum())
    mu = (int(sat.sum()) + float(z[lin].sum()) - vmax) / n if n > 0 else b
    mu = min(max(mu, a), b)
    return np.clip(z - mu, 0.0, 1.0), mu


def criticality(psi: np.ndarray, g: np.ndarray, vmax: float) -> float:
    """||psi - P_C(psi - g)||_2: zero exactly at the first-order critical points of
    min_{psi in C} J (the stopping test of Section 4.1)."""
    P, _ = project(np.asarray(psi, float) - np.asarray(g, float), vmax)
    return float(np.linalg.norm(np.asarray(psi, float) - P))


def ratio(J_c: float, J_hat: float, Jk_c: float, Jk_hat: float) -> float:
    """varrho_k = (J(psi_c) - J(psi_hat)) / (m_k(psi_c) - m_k(psi_hat)) (Algorithm 2, step 4);
    -inf when the predicted reduction is not positive."""
    pred = Jk_c - Jk_hat
    if not pred > 0.0:
        return -np.inf
    return (J_c - J_hat) / pred


def radius_update(varrho: float, delta: float, delta_max: float, prm: dict) -> tuple[bool, float]:
    """Algorithm 2, steps 5-6: accept when varrho >= eta1; the new radius is gamma1 Delta below
    eta1, gamma2 Delta on [eta1, eta2) and min(grow Delta, Delta_max) from eta2 on."""
    accepted = bool(varrho >= prm["eta1"])  # False for NaN as well
    if not accepted:
        return accepted, prm["gamma1"] * delta
    if varrho < prm["eta2"]:
        return accepted, prm["gamma2"] * delta
    return accepted, min(prm["grow"] * delta, delta_max)


@dataclasses.dataclass
class Run:
    """State of one optimisation run between major iterations."""
    psi: np.ndarray      # centre psi^(k)
    u: np.ndarray        # u*(psi^(k))
    J: float             # J(psi^(k))
    g: np.ndarray        # grad J(psi^(k)) (filtered)
    delta: float         # Delta_k
    delta_max: float
    window: list         # centre snapshots, oldest first
    iters: int = 0


def default_params(**over) -> dict:
    prm = dict(PAPER_CONSTANTS, grow=2.0, move=0.2, c1=1e-4, trials=7, volfrac=0.5, L=8)
    prm.update(over)
    return prm


def start(p, psi0: np.ndarray, prm: dict) -> Run:
    """Feasible start (projection onto C: the closest feasible design, the feasibility
    restoration of Section 4.1), the full-order solve there, and Delta_0 = tau ||r(0, rho)|| =
    tau ||f|| on the free DOFs (Eq. trrad0), Delta_max = 100 Delta_0 (Section 5)."""
    vmax = prm["volfrac"] * p.nel
    psi, _ = project(psi0, vmax)
    h = pipeline.hdm_eval(p, psi)
    f = p.F[:, 0]
    d0 = prm["tau"] * float(np.linalg.norm(f[fem.free_dofs(p)]))
    return Run(psi=psi, u=h["U"][:, 0], J=float(h["J"]), g=h["dpsi"], delta=d0,
               delta_max=prm["dmax_factor"] * d0, window=[h["U"][:, 0]])


def major_iteration(p, run: Run, prm: dict) -> dict:
    """Algorithm 2 once (steps 2-6) from run's centre; updates run in place and returns the
    quantities of the iteration."""
    vmax = prm["volfrac"] * p.nel
    # step 2: model from the basis of the window (whose newest snapshot is the centre's)
    if prm.get("n_max") is None:
        Phi = rom.basis(np.stack(run.window[-prm["L"]:], axis=1))
    else:
        prev = run.window[:-1][-prm["L"]:]
        n = max(0, min(len(prev) - 1, prm["n_max"]))
        P = rom.pod(np.stack(prev, axis=1), n)[0] if n > 0 else np.zeros((p.ndof, 0))
        Phi = rom.basis(np.column_stack([P, run.window[-1]]))
    # step 3: projected-gradient target, trial steps, the largest admissible one
    g = run.g
    t = prm["move"] / float(np.max(np.abs(g)))
    psi_x, mu = project(run.psi - t * g, vmax)
    d = psi_x - run.psi
    gtd = float(g @ d)
    s = [0.0] + [2.0 ** -r for r in range(prm["trials"])]
    ev = [pipeline.rom_eval_full(p, run.psi + si * d, Phi) for si in s]
    Jk_c = ev[0]["Jk"]
    sel, inside = len(s) - 1, False
    for r in range(1, len(s)):
        if ev[r]["resnorm"] <= run.delta and ev[r]["Jk"] <= Jk_c + prm["c1"] * s[r] * gtd:
            sel, inside = r, True
            break
    psi_hat = run.psi + s[sel] * d
    # step 4: the full-order model at the candidate and the ratio
    h = pipeline.hdm_eval(p, psi_hat)
    J_hat = float(h["J"])
    varrho = ratio(run.J, J_hat, Jk_c, ev[sel]["Jk"])
    # steps 5-6
    accepted, delta_next = radius_update(varrho, run.delta, run.delta_max, prm)
    out = dict(k=Phi.shape[1], mu=mu, gtd=gtd, Jk=[e["Jk"] for e in ev], theta=[e["resnorm"] for e in ev],
               sel=sel, inside=inside, step=s[sel], J_c=run.J, Jk_c=Jk_c, Jk_hat=ev[sel]["Jk"], J_hat=J_hat,
               theta_hat=ev[sel]["resnorm"], ratio=varrho, accepted=accepted, delta=run.delta,
               delta_next=delta_next, psi_x=psi_x, psi_hat=psi_hat)
    if accepted:
        run.psi, run.u, run.J, run.g = psi_hat, h["U"][:, 0], J_hat, h["dpsi"]
        run.window = (run.window + [run.u])[-(prm["L"] + (0 if prm.get("n_max") is None else 1)):]
    run.delta = delta_next
    run.iters += 1
    out["chi"] = criticality(run.psi, run.g, vmax)
    return out
