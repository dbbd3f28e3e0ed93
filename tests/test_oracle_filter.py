"""Pins for the oracle's linear density filter: brute-force O(N_e^2) distance loop,
preservation of constants, the adjoint identity, and the interior normaliser in closed
form."""
import math

import numpy as np
import pytest

from oracle import hatfilter
from paper_2004_05756_gb300 import workloads as w


@pytest.mark.parametrize("prob", [("q4", 1.5), ("q4", 2.5), ("h8", 2.0), ("h8", 1.2)])
def test_bruteforce(prob):
    kind, r = prob
    p = w.mbb_2d(7, 5, rmin=r) if kind == "q4" else w.cantilever_3d(4, 3, 3, rmin=r)
    psi = np.random.default_rng(4).uniform(0, 1, p.nel)
    a = hatfilter.filter_fwd(p, psi)
    b = hatfilter.filter_bruteforce(p, psi)
    assert np.abs(a - b).max() < 1e-15 * 10


@pytest.mark.parametrize("kind", ["q4", "h8"])
def test_constant_and_adjoint(kind):
    p = w.mbb_2d(9, 4) if kind == "q4" else w.cantilever_3d(5, 3, 4)
    assert np.allclose(hatfilter.filter_fwd(p, np.full(p.nel, 0.37)), 0.37, atol=1e-15, rtol=0)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal(p.nel)
    v = rng.standard_normal(p.nel)
    lhs = hatfilter.filter_fwd(p, psi) @ v
    rhs = psi @ hatfilter.filter_adj(p, v)
    assert abs(lhs - rhs) < 1e-14 * (np.abs(psi).sum() * np.abs(v).max())


def test_interior_normaliser():
    p = w.mbb_2d(6, 6, rmin=1.5)
    W = hatfilter.weight_matrix(p)
    Hs = np.asarray(W.sum(axis=1)).ravel()
    e = 3 + 6 * 3
    assert Hs[e] == pytest.approx(1.5 + 4 * 0.5 + 4 * (1.5 - math.sqrt(2.0)), rel=1e-15)
    p3 = w.cantilever_3d(5, 5, 5, rmin=2.0)
    W3 = hatfilter.weight_matrix(p3)
    Hs3 = np.asarray(W3.sum(axis=1)).ravel()
    e3 = 2 + 5 * (2 + 5 * 2)
    exp = 2.0 + 6 * 1.0 + 12 * (2 - math.sqrt(2)) + 8 * (2 - math.sqrt(3))
    assert Hs3[e3] == pytest.approx(exp, rel=1e-15)
