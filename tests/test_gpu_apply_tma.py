"""GPU parity of the TMA-staged 2D FP32 block apply (chosen when the leading dimension is a
multiple of 4 and V is 16-byte aligned).

- Against the FP64 oracle's K(rho) V within the FP32 tolerance of the other apply tests
  (2e-6 max-normalised).
- Bit for bit against the cp.async-staged form (TOPO_PARAM_APPLY_STAGES = 0), which forms the
  same stencil rows and the same products in the same order.
- The cases cover column counts that leave ragged 8-column batches, node rows of odd and even
  length (the aligned boxes then start one node early on alternate rows or on none), meshes of
  one tile and of ragged tiles, every ring depth, and non-finite values next to the grid edges:
  a halo position outside the grid must not carry the neighbouring grid row into a product.
"""
import numpy as np
import pytest

from oracle import fem
from paper_2004_05756_gb300 import workloads as w
from tests.gpu_util import dev, relerr, require_cuda

pytestmark = pytest.mark.gpu

SHAPES = {
    "q4_60x20": (60, 20),   # 61 nodes per row: alternate rows start one node early
    "q4_63x10": (63, 10),   # 64 nodes per row: every row aligned
    "q4_37x13": (37, 13),   # ragged tiles in x and y
    "q4_5x40": (5, 40),     # one tile wide, five tall
    "q4_1x1": (1, 1),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _ctx(p, stages):
    from paper_2004_05756_gb300.native import TOPO_PARAM_APPLY_STAGES, Topo
    T = Topo(p)
    T.topo_set_param(TOPO_PARAM_APPLY_STAGES, stages)
    return T


def _block(torch, M, ld):
    """N x m numpy block -> (m, ld)-strided float32 view of its first N entries per column."""
    N, m = M.shape
    buf = torch.full((m, ld), float("nan"), dtype=torch.float32, device="cuda")
    buf[:, :N] = torch.as_tensor(np.ascontiguousarray(M.T), dtype=torch.float32).cuda()
    return buf[:, :N]


def _apply(torch, T, p, rho, V, stages=None, pad=4, extra=0):
    """Y = K(rho) V in FP32 with the column pitch N rounded up to a multiple of pad, plus extra;
    returns Y (N x m) and the whole output buffer (padding initialised to 7)."""
    from paper_2004_05756_gb300.native import TOPO_PARAM_APPLY_STAGES
    if stages is not None:
        T.topo_set_param(TOPO_PARAM_APPLY_STAGES, stages)
    N, m = V.shape
    ld = -(-N // pad) * pad + extra
    Vd = _block(torch, V, ld)
    Yb = torch.full((m, ld), 7.0, dtype=torch.float32, device="cuda")
    Yd = Yb[:, :N]
    T.topo_apply_K(dev(rho), Vd, Yd, "fp32")
    T.topo_check()
    return Yd.cpu().numpy().T.copy(), Yb


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("m", [1, 3, 8, 13])
@pytest.mark.parametrize("stages", [3])
def test_tma_apply_matches_oracle(torch, shape, m, stages):
    p = w.mbb_2d(*SHAPES[shape])
    T = _ctx(p, stages)
    rng = np.random.default_rng(11)
    rho = rng.uniform(1e-3, 1, p.nel)
    V = rng.standard_normal((p.ndof, m)).astype(np.float32)
    Y, _ = _apply(torch, T, p, rho, V)
    assert relerr(Y, fem.apply_K(p, rho, V.astype(float))) < 2e-6


@pytest.mark.parametrize("shape", ["q4_60x20", "q4_63x10", "q4_37x13", "q4_5x40"])
@pytest.mark.parametrize("stages", [2, 3, 4])
def test_tma_apply_bitwise_equals_cpasync(torch, shape, stages):
    p = w.mbb_2d(*SHAPES[shape])
    T = _ctx(p, stages)
    rng = np.random.default_rng(12)
    rho = rng.uniform(1e-3, 1, p.nel)
    V = rng.standard_normal((p.ndof, 21)).astype(np.float32)
    Yt, _ = _apply(torch, T, p, rho, V, stages)
    Yc, _ = _apply(torch, T, p, rho, V, 0)
    assert np.array_equal(Yt, Yc)


def test_tma_apply_leaves_padding_untouched(torch):
    p = w.mbb_2d(37, 13)
    T = _ctx(p, 3)
    rng = np.random.default_rng(13)
    rho = rng.uniform(1e-3, 1, p.nel)
    V = rng.standard_normal((p.ndof, 9)).astype(np.float32)
    Y, Yb = _apply(torch, T, p, rho, V, extra=8)
    assert relerr(Y, fem.apply_K(p, rho, V.astype(float))) < 2e-6
    assert np.all(Yb[:, p.ndof:].cpu().numpy() == 7.0)


def test_tma_apply_nonfinite_beside_row_ends(torch):
    """NaN at the last node of grid row j and Inf at the first node of row j + 3: in the flat
    DOF order these lie where the halo positions outside the grid of edge nodes in nearby rows
    fall. Results must match the cp.async form (which zero-fills those positions) bit for bit,
    including which entries are non-finite, and edge nodes whose grid neighbours are all finite
    stay finite."""
    nx, ny = 60, 20
    p = w.mbb_2d(nx, ny)
    nnx = nx + 1
    T = _ctx(p, 3)
    rng = np.random.default_rng(14)
    rho = rng.uniform(1e-3, 1, p.nel)
    V = rng.standard_normal((p.ndof, 8)).astype(np.float32)
    j = 9
    a = nnx - 1 + nnx * j          # last node of row j
    b = nnx * (j + 3)              # first node of row j + 3
    V[2 * a:2 * a + 2, :] = np.nan
    V[2 * b:2 * b + 2, :] = np.inf
    Yc, _ = _apply(torch, T, p, rho, V, 0)
    for st in (2, 3):
        _nonfinite_same(*_apply(torch, T, p, rho, V, st)[:1], Yc, nnx, j)


def _nonfinite_same(Yt, Yc, nnx, j):
    assert np.array_equal(np.isnan(Yt), np.isnan(Yc))
    fin = np.isfinite(Yc)
    assert np.array_equal(np.isfinite(Yt), fin)
    assert np.array_equal(Yt[fin], Yc[fin])
    # (0, j), (0, j + 1): their halo position left of the grid in row j + 1 holds node a;
    # (nnx - 1, j + 2), (nnx - 1, j + 3): their halo position right of the grid in row j + 2
    # holds node b. None of them has a non-finite grid neighbour.
    for node in (nnx * j, nnx * (j + 1), nnx - 1 + nnx * (j + 2), nnx - 1 + nnx * (j + 3)):
        assert np.all(np.isfinite(Yt[2 * node:2 * node + 2, :])), node


def test_tma_apply_full_size_600x200(torch):
    """The benchmark's mesh and launch (m = 64, column pitch rounded up to a multiple of 4):
    against the oracle and bit for bit against the cp.async form."""
    p = w.mbb_600x200()
    T = _ctx(p, 3)
    rho = np.clip(w.design_field(p, 0), 1e-3, 1.0)
    V = np.random.default_rng(15).standard_normal((p.ndof, 64)).astype(np.float32)
    Yc, _ = _apply(torch, T, p, rho, V, 0)
    assert relerr(Yc, fem.apply_K(p, rho, V.astype(float))) < 2e-6
    for st in (3, 4):
        Yt, _ = _apply(torch, T, p, rho, V, st)
        assert np.array_equal(Yt, Yc), st


def test_apply_stages_parameter_range(torch):
    from paper_2004_05756_gb300.native import TOPO_PARAM_APPLY_STAGES, TopoError
    T = _ctx(w.mbb_2d(4, 2), 3)
    for v in (0, 2, 3, 4):
        T.topo_set_param(TOPO_PARAM_APPLY_STAGES, v)
    for v in (1, 5, -1, 2.5):
        with pytest.raises(TopoError):
            T.topo_set_param(TOPO_PARAM_APPLY_STAGES, v)
