"""Linear ("hat", cone) density filter rho = rho*(psi) and its adjoint, in plain FP64.

The paper filters with a Helmholtz PDE (Section 2.2, Eq. helm-soln .. cdens-star). The
benchmark replaces it with the linear density filter of the paper's references on
density-based topology optimisation: for element centres c_e, c_i,
    w_ei = max(0, r - ||c_e - c_i||),   Hs_e = sum_i w_ei,
    rho_e = sum_i w_ei psi_i / Hs_e.
Only neighbours with ||c_e - c_i|| < r contribute; boundary rows keep fewer neighbours and
are renormalised by their own Hs_e. Its adjoint, the action of (d rho*/d psi)^T that
Eq. pap_sensitivity needs, is
    g_i = sum_e w_ei v_e / Hs_e.
W is built here as an explicit sparse matrix so that the adjoint is literally W^T.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp


def element_centres(p) -> np.ndarray:
    if p.dim == 2:
        jj, ii = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
        return np.stack([ii.ravel() + 0.5, jj.ravel() + 0.5], axis=1)
    kk, jj, ii = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    return np.stack([ii.ravel() + 0.5, jj.ravel() + 0.5, kk.ravel() + 0.5], axis=1)


def weight_matrix(p) -> sp.csr_matrix:
    """W[e, i] = max(0, r - dist(e, i)) for all element pairs closer than r."""
    r = p.rmin
    R = int(math.ceil(r))
    dims = (p.nx, p.ny) if p.dim == 2 else (p.nx, p.ny, p.nz)
    grids = np.meshgrid(*[np.arange(n) for n in reversed(dims)], indexing="ij")
    idx = [g.ravel() for g in reversed(grids)]  # idx[0] = i (x), idx[1] = j, ...
    rows, cols, vals = [], [], []
    for off in itertools.product(range(-R, R + 1), repeat=p.dim):
        dist = math.sqrt(sum(o * o for o in off))
        w = r - dist
        if w <= 0.0:
            continue
        nb = [idx[a] + off[a] for a in range(p.dim)]
        ok = np.ones_like(idx[0], dtype=bool)
        for a in range(p.dim):
            ok &= (nb[a] >= 0) & (nb[a] < dims[a])
        e = np.flatnonzero(ok)
        if p.dim == 2:
            i = nb[0][ok] + p.nx * nb[1][ok]
        else:
            i = nb[0][ok] + p.nx * (nb[1][ok] + p.ny * nb[2][ok])
        rows.append(e)
        cols.append(i)
        vals.append(np.full(e.shape, w))
    W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(p.nel, p.nel)).tocsr()
    return W


def filter_fwd(p, psi: np.ndarray) -> np.ndarray:
    W = weight_matrix(p)
    Hs = np.asarray(W.sum(axis=1)).ravel()
    return (W @ psi) / Hs


def filter_adj(p, v: np.ndarray) -> np.ndarray:
    W = weight_matrix(p)
    Hs = np.asarray(W.sum(axis=1)).ravel()
    return W.T @ (v / Hs)


def filter_bruteforce(p, psi: np.ndarray) -> np.ndarray:
    """O(N_e^2) double loop over all element pairs (small meshes only)."""
    c = element_centres(p)
    out = np.zeros(p.nel)
    for e in range(p.nel):
        num = 0.0
        den = 0.0
        for i in range(p.nel):
            w = p.rmin - math.sqrt(float(np.sum((c[e] - c[i]) ** 2)))
            if w > 0:
                num += w * psi[i]
                den += w
        out[e] = num / den
    return out
