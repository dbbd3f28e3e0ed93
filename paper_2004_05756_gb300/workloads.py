"""Seeded synthetic inputs: meshes, boundary conditions, loads and design fields.

This module is shared by the CUDA path, the oracle, the tests and the bench. It holds
problem *definitions* only (which DOFs are fixed, where unit loads sit, what the seeded
random design looks like) and none of the method's arithmetic: no stiffness, no filter
of the design, no solve, no reduced model.

Numbering convention (shared by every component):
  * node n = i + (nx+1) * (j + (ny+1) * k), x fastest;
  * DOF = dim * n + c (interleaved u_x, u_y[, u_z]);
  * element e = i + nx * (j + ny * k);
  * blocks of vectors are column-major N x m with leading dimension ld >= N.

The benchmark problems stand in for the paper's MBB-beam and cantilever workloads
(Section 5.1, 5.2): unit-size Q1 elements, point loads, Dirichlet DOFs kept in the vectors.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """One linear-elasticity design problem on a structured grid of unit Q1 elements."""

    dim: int
    nx: int
    ny: int
    nz: int
    fixed: np.ndarray  # uint8[N], 1 = homogeneous Dirichlet DOF
    F: np.ndarray  # float64[N, nlc], column-major load cases (zero on fixed DOFs)
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal: float = 3.0
    rmin: float = 1.5
    name: str = ""

    @property
    def nnodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * ((self.nz + 1) if self.dim == 3 else 1)

    @property
    def ndof(self) -> int:
        return self.dim * self.nnodes

    @property
    def nel(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def shape_el(self) -> tuple:
        """Element grid shape in C order (slowest first): (ny, nx) or (nz, ny, nx)."""
        return (self.ny, self.nx) if self.dim == 2 else (self.nz, self.ny, self.nx)


def node_id(p: Problem, i, j, k=0):
    return i + (p.nx + 1) * (j + (p.ny + 1) * k)


def mbb_2d(nx: int, ny: int, rmin: float = 1.5, **material) -> Problem:
    """MBB half-beam: u_x = 0 on the left edge (symmetry), u_y = 0 at the bottom-right
    node (roller), unit downward point load at the top-left node. y points up."""
    p = Problem(2, nx, ny, 0, None, None, rmin=rmin, name=f"mbb{nx}x{ny}", **material)
    N = p.ndof
    fixed = np.zeros(N, np.uint8)
    for j in range(ny + 1):
        fixed[2 * node_id(p, 0, j) + 0] = 1
    fixed[2 * node_id(p, nx, 0) + 1] = 1
    F = np.zeros((N, 1))
    F[2 * node_id(p, 0, ny) + 1, 0] = -1.0
    p.fixed, p.F = fixed, F
    return p


def mbb_2d_multiload(nx: int, ny: int, nlc: int, seed: int, rmin: float = 1.5, **material) -> Problem:
    """MBB supports with nlc unit downward point loads at seeded top-edge nodes."""
    p = mbb_2d(nx, ny, rmin=rmin, **material)
    rng = np.random.default_rng(seed)
    cols = rng.choice(nx + 1, size=nlc, replace=(nlc > nx + 1))
    F = np.zeros((p.ndof, nlc))
    for c, i in enumerate(cols):
        F[2 * node_id(p, int(i), ny) + 1, c] = -1.0
    p.F = F
    p.name = f"mbb{nx}x{ny}_lc{nlc}"
    return p


def cantilever_3d(nx: int, ny: int, nz: int, rmin: float = 2.0, total_force_one: bool = False,
                  **material) -> Problem:
    """3D cantilever: every DOF on the face i = 0 clamped; a downward (-y) line load of
    unit intensity along the bottom edge of the right face (nodes (nx, 0, k), k = 0..nz).
    Consistent nodal forces of a unit line load on unit edges: -1 at interior nodes and
    -1/2 at the two end nodes (total -nz). With total_force_one the total is -1 instead."""
    p = Problem(3, nx, ny, nz, None, None, rmin=rmin, name=f"cant{nx}x{ny}x{nz}", **material)
    N = p.ndof
    fixed = np.zeros(N, np.uint8)
    for k in range(nz + 1):
        for j in range(ny + 1):
            n = node_id(p, 0, j, k)
            fixed[3 * n:3 * n + 3] = 1
    F = np.zeros((N, 1))
    for k in range(nz + 1):
        w = 0.5 if (k == 0 or k == nz) else 1.0
        F[3 * node_id(p, nx, 0, k) + 1, 0] = -w
    if total_force_one:
        F /= nz
    p.fixed, p.F = fixed, F
    return p


def seed_for(config_id: str, index: int) -> int:
    """Stable per-instance seed: hash of (config id, index)."""
    h = hashlib.sha256(f"{config_id}:{index}".encode()).digest()
    return int.from_bytes(h[:4], "little")


def _hat_smooth_noise(g: np.ndarray, radius: float) -> np.ndarray:
    """Input recipe only: smooth white noise g (element grid, C order) with cone weights
    max(0, radius - distance) between element centres, renormalised at the boundary.
    Written as shifted-slice sums so that it shares nothing with either filter code."""
    R = int(math.ceil(radius)) - 1
    acc = np.zeros_like(g)
    wsum = np.zeros_like(g)
    ones = np.ones_like(g)
    offs = range(-R, R + 1)
    grids = [offs] * g.ndim
    for off in np.array(np.meshgrid(*grids, indexing="ij")).reshape(g.ndim, -1).T:
        w = radius - math.sqrt(float(np.sum(off.astype(float) ** 2)))
        if w <= 0:
            continue
        src = []
        dst = []
        for ax, o in enumerate(off):
            n = g.shape[ax]
            if o >= 0:
                src.append(slice(o, n))
                dst.append(slice(0, n - o))
            else:
                src.append(slice(0, n + o))
                dst.append(slice(-o, n))
        acc[tuple(dst)] += w * g[tuple(src)]
        wsum[tuple(dst)] += w * ones[tuple(src)]
    return acc / wsum


def design_field(p: Problem, seed: int, smooth_radius: float = 3.0) -> np.ndarray:
    """Seeded smoothed-random design psi in [1e-3, 1] (float64[N_e], element order).

    g ~ N(0,1) per element (default_rng(seed).standard_normal, element order), smoothed
    with radius-3 cone weights, shifted to zero mean and scaled to unit population std;
    psi = clip(0.5 + 0.3 g, 1e-3, 1)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(p.nel).reshape(p.shape_el)
    s = _hat_smooth_noise(g, smooth_radius).ravel()
    s = s - s.mean()
    sd = s.std()
    if sd > 0:
        s = s / sd
    return np.clip(0.5 + 0.3 * s, 1e-3, 1.0)


def perturbed_designs(p: Problem, psi: np.ndarray, count: int, amplitude: float = 0.1,
                      first_seed: int = 1) -> np.ndarray:
    """Snapshot designs psi_i = clip(psi + amplitude * g_i, 1e-3, 1), g_i from seeds
    first_seed .. first_seed + count - 1 with the same smoothed recipe. Returns N_e x count."""
    out = np.empty((p.nel, count))
    for i in range(count):
        rng = np.random.default_rng(first_seed + i)
        g = rng.standard_normal(p.nel).reshape(p.shape_el)
        s = _hat_smooth_noise(g, 3.0).ravel()
        s = s - s.mean()
        sd = s.std()
        if sd > 0:
            s = s / sd
        out[:, i] = np.clip(psi + amplitude * s, 1e-3, 1.0)
    return out


# ---------------------------------------------------------------------------------------
# Named workloads (the five benchmark configurations, by what they are)
# ---------------------------------------------------------------------------------------

def mbb_60x20() -> Problem:
    return mbb_2d(60, 20, rmin=1.5)


def mbb_600x200() -> Problem:
    return mbb_2d(600, 200, rmin=1.5)


def cantilever_96x48x48() -> Problem:
    return cantilever_3d(96, 48, 48, rmin=2.0)


def batch_instances(count: int = 256, seed_base: int = 1000, nx_lo: int = 40, nx_hi: int = 400):
    """Uneven batch of 2D MBB instances: nx log-uniform in [nx_lo, nx_hi], ny = nx/2,
    1..8 seeded top-edge load cases, a basis size k in {8, 16, 32}, own seeded design."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed_base + i)
        nx = int(round(math.exp(rng.uniform(math.log(nx_lo), math.log(nx_hi)))))
        nx = max(nx_lo, min(nx_hi, nx))
        ny = max(1, nx // 2)
        nlc = int(rng.integers(1, 9))
        k = int(rng.choice([8, 16, 32]))
        p = mbb_2d_multiload(nx, ny, nlc, seed=seed_base + i)
        out.append(dict(problem=p, k=k, design_seed=seed_base + i))
    return out


def serving_stream(count: int = 2000, rate_per_s: float = 100.0, seed: int = 7,
                   q4_range=((100, 50), (800, 400)), h8_range=((32, 32, 32), (96, 48, 48))):
    """Poisson arrival stream of design-evaluation requests, 50/50 2D Q4 and 3D H8, sizes
    log-uniform between the given corners. Returns a list of dicts with arrival time,
    problem shape and seeds (problems are built lazily by the caller)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        is3d = bool(rng.integers(0, 2))
        u = rng.uniform()
        if is3d:
            lo, hi = h8_range
            shape = tuple(int(round(math.exp(math.log(a) + u * (math.log(b) - math.log(a))))) for a, b in zip(lo, hi))
        else:
            lo, hi = q4_range
            shape = tuple(int(round(math.exp(math.log(a) + u * (math.log(b) - math.log(a))))) for a, b in zip(lo, hi))
        out.append(dict(arrival=t, dim=3 if is3d else 2, shape=shape, seed=seed_for("serving", r)))
    return out


def session_stream(count: int, rate_per_s: float, sessions: int = 8, seed: int = 7,
                   q4_range=((100, 50), (800, 400)), h8_range=((32, 32, 32), (96, 48, 48))):
    """Poisson stream of requests that belong to `sessions` concurrent optimisation runs (half
    2D Q4, half 3D H8, sizes log-uniform between the corners): each request is the next
    trust-region evaluation of a session picked at random. Returns dicts with arrival time,
    session id, step within the session, last-request flag, problem shape and the session's
    seed."""
    rng = np.random.default_rng(seed)
    shapes = []
    for s in range(sessions):
        is3d = s % 2 == 1
        lo, hi = h8_range if is3d else q4_range
        u = rng.uniform()
        shapes.append((3 if is3d else 2,
                       tuple(int(round(math.exp(math.log(a) + u * (math.log(b) - math.log(a))))) for a, b in zip(lo, hi))))
    t = 0.0
    steps = [0] * sessions
    out = []
    for r in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        s = int(rng.integers(0, sessions))
        dim, shape = shapes[s]
        out.append(dict(arrival=t, session=s, step=steps[s], dim=dim, shape=shape, seed=seed_for("session", s)))
        steps[s] += 1
    seen = set()
    for d in reversed(out):  # mark each session's last request
        d["last"] = d["session"] not in seen
        seen.add(d["session"])
    return out


def build_problem(dim: int, shape) -> Problem:
    if dim == 2:
        return mbb_2d(shape[0], shape[1], rmin=1.5)
    return cantilever_3d(shape[0], shape[1], shape[2], rmin=2.0)
