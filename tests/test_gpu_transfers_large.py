"""The FP64 transfer kernels on grids that span several thread blocks with ragged last ones,
against the oracle's P (point evaluation of the coarse hats at the fine nodes):
* 2D, 320 -> 160 cells: the restriction takes two coarse nodes per thread (blocks of 64
  coarse columns: 2 full + 1 partial), the prolongation one coarse cell per thread (5 blocks
  of 32 cells), both 8 rows per block (20 blocks of 159 or 160 rows, ragged);
* 3D, 96 -> 48 cells: prolongation per coarse cell (2 blocks of 32 cells, the second
  partial), restriction by coarse pairs, 6 blocks of rows and 47 or 48 planes.
The restriction is checked through residual_restrict with x = 0 (so r = f exactly), which
needs no fine-level operator on the oracle's side, at the tolerance of the small-grid
transfer test (1e-13: sums of seven terms in an order of their own)."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import _fmg, _pair, dev, host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "2d_320": (dict(dim=2, coarse_cells=5, levels=7, w_quad=(1.0, 2.0, 0.0), zeta=3.0), 7),
    "3d_96": (dict(dim=3, coarse_cells=3, levels=6, w_quad=(1.0, 2.0, 1.5), zeta=3.0), 6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_transfers_span_blocks(name):
    kw, k = CASES[name]
    op, gp = _pair(**kw)
    fine = O.Mesh(op.dim, op.cells(k), op.box_len)
    coarse = O.Mesh(op.dim, op.cells(k - 1), op.box_len)
    p = O.prolongation(coarse, fine)
    rng = np.random.default_rng(2100 + k)
    f = rng.normal(size=gp.size(k))
    with _fmg().Solver(gp) as s:
        rc = torch.empty(gp.size(k - 1), dtype=torch.float64, device="cuda")
        s.residual_restrict(k, dev(f), dev(np.zeros(gp.size(k))), rc)
        # seven-term sums in another order than the sparse product's: a few ulps per entry
        assert rel(host(rc), p.T @ f) <= 1e-13
        ec = rng.normal(size=gp.size(k - 1))
        x = rng.normal(size=gp.size(k))
        xd = dev(x)
        s.prolong_add(k, dev(ec), xd)
        assert rel(host(xd), x + p @ ec) <= 1e-14
