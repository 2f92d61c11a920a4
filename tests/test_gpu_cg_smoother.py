"""The conjugate-gradient smoother (FMG_SMOOTH_CG, the paper's Section 4 setting of 3 + 3
steps) against the oracle's cg_steps: multigrid iterations step by step, whole FMG solves in
2D and 3D, and a batch whose instances each carry their own CG scalars."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import LAM_TOL, U_TOL, _fmg, dev, host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(**kw):
    fmg = _fmg()
    kw = {"nu_pre": 3, "nu_post": 3, **kw}
    op = O.Problem(smoother=O.SMOOTH_CG, **kw)
    gp = fmg.Problem(dim=op.dim, coarse_cells=op.coarse_cells, levels=op.levels, nu_pre=op.nu_pre,
                     nu_post=op.nu_post, vcycles=op.vcycles, corrections=op.corrections,
                     box_len=op.box_len, w_const=op.w_const, w_quad=tuple(op.w_quad), zeta=op.zeta,
                     omega=op.omega, scf_tol=op.scf_tol, scf_max_iter=100,
                     smoother=fmg.FMG_SMOOTH_CG)
    return op, gp


@pytest.mark.parametrize("kw", [
    dict(dim=2, coarse_cells=4, levels=4, w_const=0.2, w_quad=(3.0, 1.0, 0.0), zeta=5.0),
    dict(dim=2, coarse_cells=4, levels=3, w_quad=(1.0, 1.0, 0.0), zeta=5.0, nu_pre=2, nu_post=1),
    dict(dim=3, coarse_cells=2, levels=3, w_quad=(1.0, 2.0, 3.0), zeta=5.0),
], ids=["2d", "2d-2+1", "3d"])
def test_cg_multigrid_matches_oracle(kw):
    op, gp = _pair(**kw)
    lv = O.build_hierarchy(op)
    k = gp.levels
    rng = np.random.default_rng(5)
    x, f = rng.normal(size=(2, gp.size(k)))
    with _fmg().Solver(gp) as s:
        xd = dev(x)
        s.multigrid(k, dev(f), xd)
        assert rel(host(xd), O.multigrid(lv, k, f, x, op.vcycles, op)) <= 1e-11


@pytest.mark.parametrize("kw", [
    dict(dim=2, coarse_cells=8, levels=4, w_quad=(1.0, 1.0, 0.0), zeta=10.0),
    dict(dim=3, coarse_cells=4, levels=3, w_quad=(1.0, 1.0, 1.0), zeta=100.0, vcycles=1),
], ids=["2d", "3d-paper"])
def test_cg_fmg_matches_oracle(kw):
    op, gp = _pair(**kw)
    ref = O.fmg_solve(op)
    assert ref.converged
    with _fmg().Solver(gp) as s:
        u = np.empty(gp.size(gp.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) <= LAM_TOL * ref.lam
    assert np.linalg.norm(u - ref.u) <= U_TOL * np.linalg.norm(ref.u)


def test_cg_batch_equals_single_solves():
    """Each instance of a batch runs its own CG scalars: bit-identical to its solve alone."""
    fmg = _fmg()
    probs = []
    for lv, z, g in ((4, 30.0, 2.0), (3, 5.0, 1.0), (4, 120.0, 3.0)):
        _, gp = _pair(dim=2, coarse_cells=8, levels=lv, w_quad=(1.0, g * g, 0.0), zeta=z)
        probs.append(gp)
    with fmg.BatchSolver(probs) as b:
        lams, us, _, codes = b.solve_all()
    for i, p in enumerate(probs):
        with fmg.Solver(p) as s:
            u = np.empty(p.size(p.levels))
            lam, _, rc = s.solve(u)
        assert codes[i] == rc == 0
        assert lams[i] == lam
        assert np.array_equal(us[i], u)


def test_cg_needs_fp64():
    fmg = _fmg()
    _, gp = _pair(dim=2, coarse_cells=4, levels=3)
    gp.precision = fmg.FMG_MIXED_FP32
    with pytest.raises(fmg.FmgError) as e:
        fmg.Solver(gp)
    assert e.value.code == fmg.FMG_ENOTSUP
