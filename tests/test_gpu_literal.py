"""The paper-literal form of the auxiliary problem (Algorithm 3.1 step 1 as the paper writes
it: only the stiffness A on the left, W u moved to the right-hand side) against the oracle,
step by step and for whole FMG solves, with the same tolerances as the default form."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import LAM_TOL, U_TOL, _fmg, dev, host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(**kw):
    fmg = _fmg()
    op = O.Problem(operator_form=O.PAPER_LITERAL, **kw)
    gp = fmg.Problem(dim=op.dim, coarse_cells=op.coarse_cells, levels=op.levels, nu_pre=op.nu_pre,
                     nu_post=op.nu_post, vcycles=op.vcycles, corrections=op.corrections,
                     box_len=op.box_len, w_const=op.w_const, w_quad=tuple(op.w_quad), zeta=op.zeta,
                     omega=op.omega, scf_tol=op.scf_tol, scf_max_iter=100,
                     operator_form=fmg.FMG_PAPER_LITERAL)
    return op, gp


@pytest.mark.parametrize("dim", [2, 3])
def test_literal_components(dim):
    kw = (dict(dim=2, coarse_cells=4, levels=3, w_const=0.3, w_quad=(2.0, 5.0, 0.0), zeta=7.0)
          if dim == 2 else
          dict(dim=3, coarse_cells=3, levels=2, w_const=0.3, w_quad=(2.0, 5.0, 1.0), zeta=7.0))
    op, gp = _pair(**kw)
    lv = O.build_hierarchy(op)
    k = gp.levels
    rng = np.random.default_rng(40 + dim)
    u, f = rng.uniform(0.1, 1.0, size=(2, gp.size(k)))
    with _fmg().Solver(gp) as s:
        y = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
        s.apply_operator(k, dev(u), y)  # the auxiliary operator: A only
        assert rel(host(y), lv[k - 1].A @ u) <= 1e-13
        s.aux_rhs(k, 17.0, dev(u), y)
        assert rel(host(y), O.aux_rhs(op, lv[k - 1], 17.0, u)) <= 1e-13
        xd = dev(u)
        s.multigrid(k, dev(f), xd)
        assert rel(host(xd), O.multigrid(lv, k, f, u, op.vcycles, op)) <= 1e-12
        psi, k0, mm = O.augmented_blocks(lv, k, u)
        c = rng.normal(size=psi.shape[1])
        K, M, _ = s.augmented_system(k, dev(u), c)
        assert rel(K, k0) <= 1e-12  # the augmented problem keeps A + W
        assert rel(M, mm) <= 1e-12


CASES = [
    dict(dim=2, coarse_cells=4, levels=4, w_const=0.5, w_quad=(1.0, 3.0, 0.0), zeta=20.0),
    dict(dim=2, coarse_cells=8, levels=3, w_quad=(1.0, 1.0, 0.0), zeta=1.0, corrections=2),
    dict(dim=3, coarse_cells=3, levels=3, w_quad=(4.0, 1.0, 2.0), zeta=10.0),
]


@pytest.mark.parametrize("kw", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_literal_fmg_matches_oracle(kw):
    op, gp = _pair(**kw)
    ref = O.fmg_solve(op)
    assert ref.converged
    with _fmg().Solver(gp) as s:
        u = np.empty(gp.size(gp.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) <= LAM_TOL * ref.lam
    assert np.linalg.norm(u - ref.u) <= U_TOL * np.linalg.norm(ref.u)
    assert abs(st.identity_defect) < 1e-10 * lam


def test_literal_and_default_forms_share_the_fixed_point():
    """Both forms converge to the same discrete ground state (many corrections on a small
    mesh); the default form's iterate is the reference."""
    fmg = _fmg()
    kw = dict(dim=2, coarse_cells=4, levels=3, w_quad=(1.0, 2.0, 0.0), zeta=5.0, corrections=12)
    _, gp = _pair(**kw)
    with fmg.Solver(gp) as s:
        lam_lit, _, rc1 = s.solve()
    gp.operator_form = fmg.FMG_W_LEFT
    with fmg.Solver(gp) as s:
        lam_left, _, rc2 = s.solve()
    assert rc1 == rc2 == 0
    assert abs(lam_lit - lam_left) <= 1e-11 * lam_left
