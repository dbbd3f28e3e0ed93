"""Seeded input generators: sizes of the benchmark problems, determinism, value ranges."""
import numpy as np

from paper_2004_05756_gb300 import workloads as w


def test_problem_sizes():
    p = w.mbb_60x20()
    assert p.ndof == 2562 and int(p.fixed.sum()) == 22 and p.nel == 1200
    assert p.F.shape == (2562, 1) and p.F.sum() == -1.0
    p2 = w.mbb_600x200()
    assert p2.ndof == 241602 and p2.nel == 120000
    p3 = w.cantilever_3d(96, 48, 48)
    assert p3.ndof == 698691 and int(p3.fixed.sum()) == 7203 and p3.nel == 221184
    assert np.isclose(p3.F.sum(), -48.0)
    assert np.all(p3.F[p3.fixed == 1] == 0) and np.all(p.F[p.fixed == 1] == 0)


def test_design_field_deterministic_and_bounded():
    p = w.mbb_2d(40, 20)
    a = w.design_field(p, 3)
    b = w.design_field(p, 3)
    c = w.design_field(p, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 1e-3 and a.max() <= 1.0
    # smoothed: neighbouring elements are strongly correlated
    g = a.reshape(p.shape_el)
    assert np.corrcoef(g[:, 1:].ravel(), g[:, :-1].ravel())[0, 1] > 0.6
    snaps = w.perturbed_designs(p, a, 3)
    assert snaps.shape == (p.nel, 3) and snaps.min() >= 1e-3 and snaps.max() <= 1


def test_batch_and_stream():
    inst = w.batch_instances(16)
    assert len(inst) == 16
    for d in inst:
        p = d["problem"]
        assert 40 <= p.nx <= 400 and p.ny == p.nx // 2 and 1 <= p.F.shape[1] <= 8 and d["k"] in (8, 16, 32)
    s = w.serving_stream(50)
    assert all(s[i]["arrival"] < s[i + 1]["arrival"] for i in range(49))
    assert {r["dim"] for r in s} == {2, 3}
