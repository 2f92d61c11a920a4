"""The small levels of a 2D V-cycle (at most 32 cells per side) run as one fused kernel per
V-cycle.  It evaluates the same expressions in the same order as the separate sweep and
transfer kernels, so results must be bit-identical to FMG_FLAG_SEPARATE_VCYCLE: for the
component V-cycles (entered at the fused levels and above them, on even and odd coarse
sizes), for whole solves with even and odd sweep counts (which decide the ping-pong buffer of
the result) up to 4 + 4 and beyond, on hierarchies up to 256 cells per side, and for a batch
of uneven instances."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(**kw):
    fmg = _fmg()
    base = dict(dim=2, coarse_cells=8, levels=4, w_const=0.2, w_quad=(1.0, 2.0, 0.0), zeta=9.0)
    return fmg.Problem(**{**base, **kw})


def _separate(p):
    fmg = _fmg()
    q = fmg.Problem(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.flags = p.flags | fmg.FMG_FLAG_SEPARATE_VCYCLE
    return q


@pytest.mark.parametrize("k,cells", [(2, 8), (3, 8), (4, 8), (5, 6), (6, 8)])
def test_component_vcycles_bit_identical(k, cells):
    p = _problem(coarse_cells=cells, levels=6)
    rng = np.random.default_rng(1500 + k)
    f, x0 = rng.normal(size=(2, p.size(k)))
    out = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            x = dev(x0)
            s.multigrid(k, dev(f), x)
            out.append(host(x))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (0, 1), (3, 0), (4, 4), (5, 1)],
                         ids=lambda t: f"nu{t[0]}{t[1]}")
@pytest.mark.parametrize("cells,levels", [(8, 5), (4, 4), (6, 3), (6, 6), (8, 6)])
def test_solves_bit_identical(nu, cells, levels):
    p = _problem(coarse_cells=cells, levels=levels, nu_pre=nu[0], nu_post=nu[1])
    res = []
    for q in (p, _separate(p)):
        with _fmg().Solver(q) as s:
            u = np.empty(q.size(q.levels))
            lam, stats, rc = s.solve(u, stats=True)
            assert rc == 0
            res.append((lam, u))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_batch_bit_identical():
    fmg = _fmg()
    probs = [_problem(levels=lv, zeta=z, w_quad=(1.0, g * g, 0.0))
             for lv, z, g in ((4, 3.0, 1.0), (3, 40.0, 2.0), (5, 100.0, 1.5), (2, 7.0, 3.0))]
    lams = []
    for ps in (probs, [_separate(p) for p in probs]):
        b = fmg.BatchSolver(ps)
        lam = torch.empty(len(ps), dtype=torch.float64, device="cuda")
        b.solve_dev_all(lam)
        lams.append(host(lam))
        b.close()
    assert np.array_equal(lams[0], lams[1])
