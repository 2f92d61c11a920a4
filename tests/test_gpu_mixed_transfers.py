"""The single-precision restriction and prolongation of the mixed modes on grids that span
several thread blocks (four coarse nodes or four fine columns per thread, 32 threads per block
row): 2D 640 cells (restriction 320 -> 80 threads, 3 blocks, ragged; prolongation 160
threads, 5 blocks) and 3D 384 cells (restriction 48 threads, 2 blocks, ragged; prolongation
96 threads, 3 blocks).

The component multigrid call of a mixed handle runs FP64 defect correction around
single-precision V-cycles; from the same start and right-hand side its result must agree with
the FP64 handle's m V-cycles to single-precision accuracy of the correction.  A wrong
coupling in either transfer leaves the V-cycle a much poorer preconditioner, and the two
results then differ by a sizeable fraction of the correction."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "2d_640": (dict(dim=2, coarse_cells=5, levels=8, w_quad=(1.0, 2.0, 0.0), zeta=3.0), 8),
    "3d_384": (dict(dim=3, coarse_cells=3, levels=8, w_quad=(1.0, 2.0, 1.5), zeta=3.0), 8),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_vcycles_match_fp64_on_multiblock_grids(name):
    fmg = _fmg()
    kw, k = CASES[name]
    out = {}
    rng = np.random.default_rng(2300 + k)
    p = fmg.Problem(**kw, flags=fmg.FMG_FLAG_NO_AUTOTUNE)
    f, x0 = rng.normal(size=(2, p.size(k)))
    for prec in (fmg.FMG_FP64, fmg.FMG_MIXED_FP32):
        q = fmg.Problem(**kw, precision=prec, flags=fmg.FMG_FLAG_NO_AUTOTUNE)
        with fmg.Solver(q) as s:
            x = dev(x0)
            s.multigrid(k, dev(f), x)
            out[prec] = host(x)
        torch.cuda.empty_cache()
    x64, x32 = out[fmg.FMG_FP64], out[fmg.FMG_MIXED_FP32]
    corr = np.linalg.norm(x64 - x0)
    assert corr > 0.0
    rel = np.linalg.norm(x32 - x64) / corr
    print(f"{name}: |x_mixed - x_fp64| / |x_fp64 - x0| = {rel:.2e}")
    assert rel <= 1e-5  # measured 6.7e-8 (2D), 1.9e-7 (3D)
