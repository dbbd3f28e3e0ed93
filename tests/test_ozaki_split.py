"""The arithmetic of the tensor-core reduced assembly (the Ozaki scheme of Ozaki, Ogita, Oishi and
Rump, 2012, with BF16 digits and FP32 sums as in Mukunoki, Ozaki, Ogita and Imamura, 2020),
restated in numpy integers so that its exactness claims can be checked without a GPU:

- the 8 balanced base-128 digits of q = trunc(|x| 2^off / 2^(mx - 1022) * 2^55) rebuild q exactly,
  with |d| <= 64 (so each digit is exact in BF16);
- over 512 element rows the sum of |digit products| of one level stays <= 2^24, so every FP32
  partial sum of the MMAs is an exact integer, in any order;
- on SIMP moduli against the element matrices of a snapshot basis (whose soft elements carry the
  largest entries), the per-element power-of-two balancing taken from Hel keeps the result at
  FP64 size relative to H, where one scale for all elements loses about 2^-42 of it.

The GPU kernel itself is tested against exact sums in tests/test_gpu_assembly_tc.py."""
import math

import numpy as np

from oracle import element, fem, hatfilter, rom
from paper_2004_05756_gb300 import workloads as w

D = 8  # digits per operand


def exponent(x):
    return ((np.asarray(x, np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)


def digits(x, mx, off):
    """Balanced base-128 digits, most significant first: shape x.shape + (8,)."""
    x = np.asarray(x, np.float64)
    b = x.view(np.uint64)
    ex = exponent(x)
    sh = mx - ex - off
    ok = (ex != 0) & (sh >= 0) & (sh < 55)
    m53 = (b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    q = np.where(ok, (m53 << np.uint64(2)) >> np.clip(sh, 0, 63).astype(np.uint64), np.uint64(0))
    d = np.zeros(x.shape + (D,), np.int64)
    carry = np.zeros(x.shape, np.int64)
    for i in range(D - 1, 0, -1):
        u = ((q >> np.uint64(7 * (D - 1 - i))) & np.uint64(127)).astype(np.int64) + carry
        carry = (u >= 64).astype(np.int64)
        d[..., i] = u - 128 * carry
    d[..., 0] = (q >> np.uint64(49)).astype(np.int64) + carry
    sign = np.where((b >> np.uint64(63)) == 1, -1, 1)
    return d * sign[..., None], q


def assemble(E, H, balance=True, drain=512):
    """C = E @ H the way the kernel forms it over one range of element rows (one CTA, one tile)."""
    R, n = E.shape
    if balance:
        se = np.max(np.where(H != 0, exponent(H), 0), axis=1)  # per element row, over the columns
    else:
        se = np.full(n, 1023)
    se = np.where(se == 0, 1023, se)
    offE = se - 1023
    exE = exponent(E)
    rexp = np.max(np.where(exE != 0, exE + offE[None, :], 0), axis=1)
    exH = exponent(H)
    cexp = np.max(np.where(exH != 0, exH - offE[:, None], 0), axis=0)
    dE, _ = digits(E, rexp[:, None], offE[None, :])
    dH, _ = digits(H, cexp[None, :], -offE[:, None])
    acc = np.zeros((R, H.shape[1]))
    worst = 0
    for e0 in range(0, n, drain):
        sl = slice(e0, min(n, e0 + drain))
        V = np.zeros((D, R, H.shape[1]), np.int64)
        A = np.zeros((D, R, H.shape[1]), np.int64)
        for i in range(D):
            for j in range(D - i):
                V[i + j] += dE[:, sl, i] @ dH[sl, :, j]
                A[i + j] += np.abs(dE[:, sl, i]) @ np.abs(dH[sl, :, j])
        worst = max(worst, int(A.max()))
        t = V[D - 1].astype(np.float64)
        for lv in range(D - 2, -1, -1):
            t = t * 2.0 ** -7 + V[lv]
        acc += t
    scale = np.ldexp(1.0, (rexp[:, None] - 1022) + (cexp[None, :] - 1022) - 12)
    return acc * scale, worst


def exact_dot(a, b):
    def split(x):
        c = 134217729.0 * x
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    return math.fsum(np.concatenate([p, ((ah * bh - p) + ah * bl + al * bh) + al * bl]))


def test_digits_rebuild_q_exactly():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-40, 40, 20000))
    x[:5] = [0.0, 1.0, -1.0, 2.0 ** -1074, np.nextafter(2.0, 0)]
    mx = np.full(x.shape, int(exponent(np.abs(x)).max()))
    d, q = digits(x, mx, 0)
    assert np.abs(d).max() <= 64
    rebuilt = np.zeros(x.shape, dtype=object)
    for i in range(D):
        rebuilt = rebuilt + d[:, i].astype(object) * (128 ** (D - 1 - i))
    sgn = np.where(x < 0, -1, 1)
    assert all(int(r) == int(s) * int(qq) for r, s, qq in zip(rebuilt, sgn, q))
    # the truncation: |x| / tau * 2^55 - q in [0, 1)
    tau = np.ldexp(1.0, mx - 1022)
    frac = np.abs(x) / tau * 2.0 ** 55 - q.astype(np.float64)
    assert np.all((frac > -1e-3) & (frac < 1.0 + 1e-3))


def _snapshot_case():
    p = w.mbb_2d(40, 14)
    k = 6
    psi0 = w.design_field(p, 5)
    snaps = w.perturbed_designs(p, psi0, k, amplitude=0.1, first_seed=12)
    Phi = rom.basis(np.stack([fem.solve(p, hatfilter.filter_fwd(p, snaps[:, i]))[:, 0] for i in range(k)], 1))
    kk = Phi.shape[1]
    Ke = element.ke(p.dim, p.nu)
    ed = fem.edof(p)
    iu = np.triu_indices(kk)
    Hel = np.stack([(Phi[ed[e]].T @ Ke @ Phi[ed[e]])[iu] for e in range(p.nel)])
    cands = w.perturbed_designs(p, psi0, 3, amplitude=0.02, first_seed=400)
    E = np.stack([fem.young(hatfilter.filter_fwd(p, cands[:, r]), p.E0, p.Emin, p.penal) for r in range(3)])
    return E, Hel


def test_level_sums_stay_exact_in_fp32():
    E, Hel = _snapshot_case()
    _, worst = assemble(E, Hel)
    assert worst <= 2 ** 24


def test_balancing_keeps_fp64_accuracy():
    E, Hel = _snapshot_case()
    ex = np.array([[exact_dot(E[r], Hel[:, q]) for q in range(Hel.shape[1])] for r in range(E.shape[0])])
    hmax = np.abs(ex).max(1, keepdims=True)
    bal, _ = assemble(E, Hel, balance=True)
    unb, _ = assemble(E, Hel, balance=False)
    err_bal = (np.abs(bal - ex) / hmax).max()
    err_unb = (np.abs(unb - ex) / hmax).max()
    assert err_bal <= 2.0 ** -46, err_bal
    assert err_unb > 10 * err_bal  # the scale common to all elements loses bits on soft elements


def test_integer_inputs_exact():
    rng = np.random.default_rng(2)
    E = rng.integers(1, 65, (3, 1300)) / 64.0
    H = rng.integers(-4096, 4097, (1300, 10)).astype(float)
    got, _ = assemble(E, H)
    assert np.array_equal(got, E @ H)
