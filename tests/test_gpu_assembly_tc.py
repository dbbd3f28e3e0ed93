"""The per-density reduced assembly H_r = sum_e E_r,e Hel_e (Section 3.4, Remark rom_assemble)
on the tensor cores (TOPO_PARAM_ROM_ASSEMBLY = 1: the Ozaki scheme's exact split of each FP64
operand into 8 BF16 digits, exact FP32 sums over 512 element rows, FP64 beyond) against exact
and FP64 references, through topo_rom_assemble_batch and topo_rom_eval_batch.

- Integer-valued inputs whose sums FP64 holds exactly: the tensor path, the FP64 SIMT path and
  numpy agree bit for bit (any lost digit, level, drain or scale would show).
- Moduli of SIMP designs (1e-9 .. 1) against element matrices of a random and of a snapshot
  basis (whose soft elements carry the largest element matrices): every entry against the exactly
  rounded sum (Dekker's product and fsum), within the method's bound with the balancing
  s_e = 2^floor(log2 max_p |Hel_e,p|) over each 64-column tile: 2^-54 (max_e |E_e s_e|
  sum_e |Hel_e / s_e| + max_e |Hel_e / s_e| sum_e |E_e s_e|) (truncation below scales of at most
  twice the maxima) plus 2^-51 sum_e |E_e Hel_e| (dropped digit levels, FP64 combination); and
  within 2^-46 of the candidate's largest |H| entry (the balancing's purpose).
- Shapes: a ragged last chunk and block (482 rows), several exact-accumulation drains per CTA
  (120,001 rows), one and several column tiles (k = 8, 16, 24, 40), R = 1, 100, 128 and 130 (two
  passes); candidates evaluated alone and inside a batch agree bit for bit, also through
  topo_rom_eval_batch with 150 candidates.
- topo_rom_eval_batch with either contraction: J_k and y differ by no more than the first-order
  effect of the assembly bound, |y|^T B |y| and |H^-1| B |y| with B = 3 eps sum_e |E_e| |Hel_e|."""
import math

import numpy as np
import pytest

from oracle import fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import cols, dev, require_cuda

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _ctx(p, tensor):
    from paper_2004_05756_gb300.native import Topo, TOPO_PARAM_ROM_ASSEMBLY
    T = Topo(p)
    T.topo_set_param(TOPO_PARAM_ROM_ASSEMBLY, 1 if tensor else 0)
    return T


def _assemble(T, E, Hel, k):
    import torch as th
    H = th.zeros(E.shape[0] * k * k, dtype=th.float64, device="cuda")
    Hd = Hel if isinstance(Hel, th.Tensor) else dev(Hel)
    T.topo_rom_assemble_batch(dev(np.ascontiguousarray(E)), Hd, k, H)
    T.topo_check()
    return H.cpu().numpy().reshape(E.shape[0], k, k)


def _unpack(Hp, k):
    """Packed upper-triangle rows (i <= j, row-major) -> symmetric k x k."""
    iu = np.triu_indices(k)
    out = np.zeros(Hp.shape[:-1] + (k, k))
    out[..., iu[0], iu[1]] = Hp
    out[..., iu[1], iu[0]] = Hp
    return out


def _exact_dot(a, b):
    """The correctly rounded sum_e a_e b_e: Dekker's exact product (Veltkamp splitting) and fsum."""
    def split(x):
        c = 134217729.0 * x
        hi = c - (c - x)
        return hi, x - hi
    prod = a * b
    ah, al = split(a)
    bh, bl = split(b)
    err = ((ah * bh - prod) + ah * bl + al * bh) + al * bl
    return math.fsum(np.concatenate([prod, err]))


def _bound(E, Hh):
    """The tensor-core assembly's error bound per packed entry (R x P): per 64-column tile the
    balancing s_e = 2^floor(log2 max_p |Hel_e,p|), truncation below scales of at most twice the
    balanced maxima, and the dropped levels with the FP64 combination."""
    out = np.zeros((E.shape[0], Hh.shape[1]))
    for t0 in range(0, Hh.shape[1], 64):
        Ht = Hh[:, t0:t0 + 64]
        m = np.abs(Ht).max(1)
        s = np.ldexp(1.0, np.frexp(np.where(m > 0, m, 1.0))[1] - 1)
        Eb, Hb = np.abs(E) * s[None, :], np.abs(Ht) / s[:, None]
        out[:, t0:t0 + 64] = 2.0 ** -54 * (Eb.max(1)[:, None] * Hb.sum(0)[None, :] +
                                           Hb.max(0)[None, :] * Eb.sum(1)[:, None]) \
            + 2.0 ** -51 * (np.abs(E) @ np.abs(Ht))
    return out


def _moduli(p, rhos):
    E = fem.young(np.asarray(rhos), p.E0, p.Emin, p.penal)
    return np.concatenate([E, np.ones((E.shape[0], 1))], 1)


@pytest.mark.parametrize("mesh,k,R", [("q4_37x13", 16, 5), ("q4_37x13", 8, 130), ("q4_600x200", 16, 100),
                                      ("q4_600x200", 24, 3), ("q4_37x13", 40, 9),
                                      ("q4_600x200", 16, 128)])
def test_integer_inputs_exact(torch, mesh, k, R):
    p = {"q4_37x13": lambda: w.mbb_2d(37, 13), "q4_600x200": lambda: w.mbb_2d(600, 200)}[mesh]()
    rows, P = p.nel + 1, k * (k + 1) // 2
    rng = np.random.default_rng(R + k)
    E = rng.integers(1, 65, (R, rows)) / 64.0
    Hel = rng.integers(-4096, 4097, (rows, P)).astype(float)
    ref = _unpack(E @ Hel, k)  # every partial sum is an exact FP64 number
    got_tc = _assemble(_ctx(p, True), E, Hel.ravel(), k)
    got_simt = _assemble(_ctx(p, False), E, Hel.ravel(), k)
    assert np.array_equal(got_simt, ref)
    assert np.array_equal(got_tc, ref)


@pytest.mark.parametrize("mesh,k,R,basis", [("q4_37x13", 6, 33, "random"), ("q4_60x20", 8, 20, "snapshots"),
                                            ("q4_600x200", 16, 100, "random"), ("h8_12x6x6", 24, 7, "random")])
def test_simp_moduli_within_bound(torch, mesh, k, R, basis):
    import torch as th
    p = {"q4_37x13": lambda: w.mbb_2d(37, 13), "q4_60x20": lambda: w.mbb_2d(60, 20),
         "q4_600x200": lambda: w.mbb_2d(600, 200), "h8_12x6x6": lambda: w.cantilever_3d(12, 6, 6)}[mesh]()
    T = _ctx(p, True)
    rng = np.random.default_rng(k)
    psi0 = w.design_field(p, 3)
    if basis == "random":
        Phi, _ = np.linalg.qr(rng.standard_normal((p.ndof, k)))
        Phi[p.fixed == 1] = 0.0
    else:
        snaps = w.perturbed_designs(p, psi0, k, amplitude=0.1, first_seed=12)
        Phi = rom.basis(np.stack([fem.solve(p, hatfilter.filter_fwd(p, snaps[:, i]))[:, 0] for i in range(k)], 1))
        k = Phi.shape[1]
    Hel = th.zeros((p.nel + 1) * k * (k + 1) // 2, dtype=th.float64, device="cuda")
    T.topo_rom_elem(cols(Phi), k, Hel)
    Hh = Hel.cpu().numpy().reshape(p.nel + 1, -1)
    rhos = np.stack([hatfilter.filter_fwd(p, c) for c in w.perturbed_designs(p, psi0, R, 0.05, first_seed=70).T])
    E = _moduli(p, rhos)
    got = _assemble(T, E, Hel, k)
    iu = np.triu_indices(k)
    gotp = got[:, iu[0], iu[1]]
    bound = _bound(E, Hh)
    P = Hh.shape[1]
    entries = [(r, q) for r in range(R) for q in range(P)]
    if len(entries) > 400:
        entries = [entries[i] for i in np.random.default_rng(0).choice(len(entries), 400, replace=False)]
    hmax = np.abs(gotp).max(1)
    for r, q in entries:
        ex = _exact_dot(E[r], Hh[:, q])
        assert abs(gotp[r, q] - ex) <= bound[r, q], (r, q, gotp[r, q] - ex, bound[r, q])
        # normwise: the balancing keeps the error at FP64 size relative to H (a scale common to
        # all elements loses up to 2^-42 of it on a snapshot basis)
        assert abs(gotp[r, q] - ex) <= 2.0 ** -46 * hmax[r], (r, q, gotp[r, q] - ex, hmax[r])
    # and the whole H against the definition Phi^T K(rho) Phi on the oracle for two candidates
    f = p.F[:, 0]
    for r in (0, R - 1):
        Ho, _ = rom.project(p, rhos[r], Phi, f)
        scale = np.abs(Phi).T @ (abs(fem.assemble_K(p, rhos[r])) @ np.abs(Phi))
        assert np.all(np.abs(got[r] - Ho) <= 1e-12 * scale)


def test_independent_of_the_batch(torch):
    p = w.mbb_2d(600, 200)
    k = 16
    T = _ctx(p, True)
    rng = np.random.default_rng(4)
    P = k * (k + 1) // 2
    Hel = rng.standard_normal((p.nel + 1) * P) * np.exp(rng.uniform(-20, 0, (p.nel + 1) * P))
    E = rng.uniform(1e-9, 1.0, (128, p.nel + 1)) ** 3
    full = _assemble(T, E, Hel, k)
    for r in (0, 77, 127):
        assert np.array_equal(_assemble(T, E[r:r + 1], Hel, k)[0], full[r])


def test_rom_eval_batch_more_than_one_pass(torch):
    """150 candidates in one topo_rom_eval_batch call (two tensor-core passes of up to 128, groups
    of 32 inside each): every candidate's J_k, residual norms, y and gradient equal its own
    one-candidate call bit for bit."""
    import torch as th
    p = w.mbb_2d(30, 12)
    k = 6
    T = _ctx(p, True)
    psi0 = w.design_field(p, 2)
    snaps = w.perturbed_designs(p, psi0, k, amplitude=0.1, first_seed=21)
    Phi = rom.basis(np.stack([fem.solve(p, hatfilter.filter_fwd(p, snaps[:, i]))[:, 0] for i in range(k)], 1))
    kk = Phi.shape[1]
    f = p.F[:, 0]
    f64 = dict(dtype=th.float64, device="cuda")
    Hel = th.zeros((p.nel + 1) * kk * (kk + 1) // 2, **f64)
    T.topo_rom_elem(cols(Phi), kk, Hel)
    b, fd = dev(Phi.T @ f), dev(f)
    R = 150
    psi = dev(np.ascontiguousarray(w.perturbed_designs(p, psi0, R, amplitude=0.02, first_seed=500).T))

    def run(ps):
        n = ps.shape[0]
        out = (th.zeros(n, **f64), th.zeros((n, 2), **f64), th.zeros((n, kk), **f64), th.zeros((n, p.nel), **f64))
        T.topo_rom_eval_batch(ps, Hel, cols(Phi), kk, b, fd, *out)
        T.topo_check()
        return [o.cpu().numpy() for o in out]

    full = run(psi)
    for r in (0, 31, 127, 128, 149):
        one = run(psi[r:r + 1].contiguous())
        for a, o in zip(full, one):
            assert np.array_equal(a[r], o[0]), r


def test_rom_eval_batch_both_contractions(torch):
    """topo_rom_eval_batch with the tensor-core and the SIMT contraction on a snapshot basis."""
    import torch as th
    p = w.mbb_2d(60, 20)
    k = 8
    psi0 = w.design_field(p, 5)
    snaps = w.perturbed_designs(p, psi0, k, amplitude=0.1, first_seed=12)
    U = np.stack([fem.solve(p, hatfilter.filter_fwd(p, snaps[:, i]))[:, 0] for i in range(k)], 1)
    Phi = rom.basis(U)
    kk = Phi.shape[1]
    f = p.F[:, 0]
    R = 45
    cands = w.perturbed_designs(p, psi0, R, amplitude=0.02, first_seed=400)
    psi = dev(np.ascontiguousarray(cands.T))
    f64 = dict(dtype=th.float64, device="cuda")
    res = {}
    for tensor in (True, False):
        T = _ctx(p, tensor)
        Hel = th.zeros((p.nel + 1) * kk * (kk + 1) // 2, **f64)
        T.topo_rom_elem(cols(Phi), kk, Hel)
        Jk, rn, y, dp = th.zeros(R, **f64), th.zeros((R, 2), **f64), th.zeros((R, kk), **f64), th.zeros((R, p.nel), **f64)
        T.topo_rom_eval_batch(psi, Hel, cols(Phi), kk, dev(Phi.T @ f), dev(f), Jk, rn, y, dp)
        T.topo_check()
        res[tensor] = (Jk.cpu().numpy(), y.cpu().numpy(), rn.cpu().numpy(), dp.cpu().numpy(), Hel.cpu().numpy())
    Hh = res[False][4].reshape(p.nel + 1, -1)
    assert np.array_equal(res[True][4], res[False][4])  # the same element matrices
    for r in range(R):
        rho = hatfilter.filter_fwd(p, cands[:, r])
        E = _moduli(p, rho[None, :])[0]
        B = 3 * EPS * _unpack(np.abs(E) @ np.abs(Hh), kk)
        H = _unpack(E @ Hh, kk)
        ya = np.abs(res[False][1][r])
        dJ = ya @ B @ ya
        dy = np.abs(np.linalg.inv(H)) @ (B @ ya)
        J0 = res[False][0][r]
        assert abs(res[True][0][r] - J0) <= 2 * dJ + 1e-13 * abs(J0), r
        assert np.all(np.abs(res[True][1][r] - res[False][1][r]) <= 2 * dy + 1e-13 * np.abs(res[False][1][r]).max())
        # residual norms and gradients follow y: compare at the oracle-parity tolerances
        assert res[True][2][r, 0] == pytest.approx(res[False][2][r, 0], rel=1e-8, abs=1e-14)
        assert np.abs(res[True][3][r] - res[False][3][r]).max() <= 1e-8 * np.abs(res[False][3][r]).max()


def test_invalid_arguments(torch):
    from paper_2004_05756_gb300 import native
    p = w.mbb_2d(20, 10)
    T = native.Topo(p)
    L = native.load()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    P = x.data_ptr()
    rows = p.nel + 1
    assert L.topo_rom_assemble_batch(T.h, 0, P, rows, P, 4, P) == native.TOPO_OK
    assert L.topo_rom_assemble_batch(T.h, -1, P, rows, P, 4, P) == native.TOPO_ERR_INVALID
    assert L.topo_rom_assemble_batch(T.h, 2, P, rows - 1, P, 4, P) == native.TOPO_ERR_INVALID
    assert L.topo_rom_assemble_batch(T.h, 2, P, rows, P, 0, P) == native.TOPO_ERR_INVALID
    assert L.topo_rom_assemble_batch(T.h, 2, P, rows, P, 129, P) == native.TOPO_ERR_INVALID
    assert L.topo_rom_assemble_batch(T.h, 2, None, rows, P, 4, P) == native.TOPO_ERR_INVALID
    for bad in (2, -1):
        with pytest.raises(native.TopoError):
            T.topo_set_param(native.TOPO_PARAM_ROM_ASSEMBLY, bad)
    T.topo_check()
