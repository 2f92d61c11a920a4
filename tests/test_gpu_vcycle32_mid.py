"""In the mixed modes the 2D levels of a single-precision V-cycle below the TMA-fed ones (at most
256 cells per side) run as two kernels per level, a down leg (pre-smoothing from zero,
residual, restriction) and an up leg (prolongation, post-smoothing), on 32 x 32 tiles with
recomputed halos.  They evaluate the separate kernels' expressions in the same order and store
in the same precision where those do, so FP32 and BF16-storage results must be bit-identical
to FMG_FLAG_SEPARATE_VCYCLE: for the component multigrid call (which always runs the
single-precision V-cycles) entered at several levels and on odd coarse sizes, whose interiors
span several tiles with a ragged last one (191 = 5 x 32 + 31 nodes per side at 192 cells), for
sweep counts that the fused legs take (up to 4) and that they leave to the separate kernels,
for whole solves whose large stages use the TMA-fed sweeps above the fused levels, and for a
batch of uneven instances.

The 3D levels of up to 32 cells per side (8 x 8 x 8 tiles, up to 2 + 2 sweeps) are checked
the same way: component calls on coarse sizes 3 and 4 (23 = 2 x 8 + 7 interior nodes per side
at 24 cells), sweep counts in and out of the fused range, solves whose 128-cell stage uses
the TMA-fed sweep (and 64- and 96-cell stages that use the separate kernels) above the fused
levels, and a batch."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(**kw):
    fmg = _fmg()
    base = dict(dim=2, coarse_cells=8, levels=4, w_const=0.2, w_quad=(1.0, 2.0, 0.0), zeta=9.0,
                precision=fmg.FMG_MIXED_FP32)
    return fmg.Problem(**{**base, **kw})


def _separate(p):
    fmg = _fmg()
    q = fmg.Problem(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.flags = p.flags | fmg.FMG_FLAG_SEPARATE_VCYCLE
    return q


def _precisions():
    fmg = _fmg()
    return [("fp32", fmg.FMG_MIXED_FP32), ("bf16", fmg.FMG_MIXED_BF16)]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("k,cells", [(2, 8), (4, 8), (6, 8), (6, 6), (7, 6), (6, 5), (5, 3)])
def test_component_vcycles_bit_identical(k, cells, prec):
    p = _problem(coarse_cells=cells, levels=7, precision=_precisions()[prec][1])
    rng = np.random.default_rng(1700 + 10 * k + cells)
    f, x0 = rng.normal(size=(2, p.size(k)))
    out = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            x = dev(x0)
            s.multigrid(k, dev(f), x)
            out.append(host(x))
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (0, 1), (3, 0), (4, 4), (5, 1)],
                         ids=lambda t: f"nu{t[0]}{t[1]}")
def test_component_sweep_counts_bit_identical(nu):
    p = _problem(coarse_cells=6, levels=6, nu_pre=nu[0], nu_post=nu[1])
    rng = np.random.default_rng(1800 + 10 * nu[0] + nu[1])
    f, x0 = rng.normal(size=(2, p.size(6)))
    out = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            x = dev(x0)
            s.multigrid(6, dev(f), x)
            out.append(host(x))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("cells,levels", [(8, 7), (6, 8)])
def test_mixed_solves_bit_identical(cells, levels, prec):
    """512 and 768 cells per side: the stages from 512 up run FP32 V-cycles whose top levels
    use the TMA-fed sweeps and whose levels from 256 down the fused legs."""
    p = _problem(coarse_cells=cells, levels=levels, precision=_precisions()[prec][1])
    res = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            u = np.empty(q.size(q.levels))
            lam, _, rc = s.solve(u)
            assert rc == 0
            res.append((lam, u))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_mixed_batch_bit_identical():
    fmg = _fmg()
    probs = [_problem(coarse_cells=8, levels=lv, zeta=z, w_quad=(1.0, g * g, 0.0))
             for lv, z, g in ((7, 3.0, 1.0), (6, 40.0, 2.0), (7, 100.0, 1.5), (5, 7.0, 3.0))]
    lams = []
    for ps in (probs, [_separate(p) for p in probs]):
        b = fmg.BatchSolver(ps)
        lam = torch.empty(len(ps), dtype=torch.float64, device="cuda")
        b.solve_dev_all(lam)
        lams.append(host(lam))
        b.close()
    assert np.array_equal(lams[0], lams[1])


def _problem3(**kw):
    base = dict(dim=3, coarse_cells=4, levels=5, w_const=0.2, w_quad=(1.0, 2.0, 4.0),
                zeta=30.0)
    return _problem(**{**base, **kw})


def _component_pair(p, k, seed):
    rng = np.random.default_rng(seed)
    f, x0 = rng.normal(size=(2, p.size(k)))
    out = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            x = dev(x0)
            s.multigrid(k, dev(f), x)
            out.append(host(x))
    return out


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("k,cells", [(2, 4), (3, 3), (5, 3), (4, 4), (5, 4), (6, 4)])
def test_component_vcycles_bit_identical_3d(k, cells, prec):
    p = _problem3(coarse_cells=cells, levels=6, precision=_precisions()[prec][1])
    out = _component_pair(p, k, 2700 + 10 * k + cells)
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nu", [(2, 2), (1, 2), (0, 1), (2, 0), (3, 1), (1, 3)],
                         ids=lambda t: f"nu{t[0]}{t[1]}")
def test_component_sweep_counts_bit_identical_3d(nu):
    p = _problem3(coarse_cells=3, levels=5, nu_pre=nu[0], nu_post=nu[1])
    out = _component_pair(p, 5, 2800 + 10 * nu[0] + nu[1])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("cells,levels", [(4, 6), (3, 6)])
def test_mixed_solves_bit_identical_3d(cells, levels, prec):
    p = _problem3(coarse_cells=cells, levels=levels, precision=_precisions()[prec][1])
    res = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            u = np.empty(q.size(q.levels))
            lam, _, rc = s.solve(u)
            assert rc == 0
            res.append((lam, u))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_mixed_batch_bit_identical_3d():
    fmg = _fmg()
    probs = [_problem3(coarse_cells=c, levels=lv, zeta=z, w_quad=(1.0, 2.0, g * g))
             for c, lv, z, g in ((4, 5, 3.0, 1.0), (4, 4, 40.0, 2.0), (4, 5, 100.0, 1.5))]
    lams = []
    for ps in (probs, [_separate(p) for p in probs]):
        b = fmg.BatchSolver(ps)
        lam = torch.empty(len(ps), dtype=torch.float64, device="cuda")
        b.solve_dev_all(lam)
        lams.append(host(lam))
        b.close()
    assert np.array_equal(lams[0], lams[1])
