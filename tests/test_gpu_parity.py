"""GPU parity: every step of the hot path through the C ABI against the FP64 oracle.

Tolerances (FP64 everywhere; the two sides differ only in rounding order, FMA contraction and
the nonlinear solver's path to the same fixed point):
  * linear stencil / transfer / load steps: max |gpu - oracle| <= 1e-13 * max |oracle|;
  * V-cycles: 1e-12 relative (a few sweeps compound rounding);
  * eigenpairs: |lambda rel| <= 1e-11 and ||u_gpu - u_oracle||_2 / ||u_oracle||_2 <= 1e-9,
    the bound the solver is specified to meet."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from workloads import seeded_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM_TOL = 1e-11
U_TOL = 1e-9


def _fmg():
    from paper_1502_04657_gb300 import fmg
    return fmg


def _pair(**kw):
    """Oracle problem and GPU problem with identical parameters."""
    fmg = _fmg()
    op = O.Problem(**kw)
    gp = fmg.Problem(dim=op.dim, coarse_cells=op.coarse_cells, levels=op.levels, nu_pre=op.nu_pre,
                     nu_post=op.nu_post, vcycles=op.vcycles, corrections=op.corrections,
                     box_len=op.box_len, w_const=op.w_const, w_quad=tuple(op.w_quad), zeta=op.zeta,
                     omega=op.omega, scf_tol=op.scf_tol, scf_max_iter=100)
    return op, gp


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


KW = dict(dim=2, coarse_cells=4, levels=4, w_const=0.3, w_quad=(1.0, 2.5, 0.0), zeta=7.0)


@pytest.fixture(scope="module")
def setup():
    op, gp = _pair(**KW)
    levels = O.build_hierarchy(op)
    solver = _fmg().Solver(gp)
    yield op, gp, levels, solver
    solver.close()


@pytest.mark.parametrize("k", [1, 2, 4])
def test_operator_and_mass(setup, k):
    op, gp, lv, s = setup
    rng = np.random.default_rng(100 + k)
    x = rng.normal(size=gp.size(k))
    y = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.apply_operator(k, dev(x), y)
    assert rel(host(y), lv[k - 1].L @ x) <= 1e-13
    s.apply_mass(k, dev(x), y)
    assert rel(host(y), lv[k - 1].M @ x) <= 1e-13


@pytest.mark.parametrize("k", [2, 4])
def test_jacobi_sweep(setup, k):
    op, gp, lv, s = setup
    rng = np.random.default_rng(200 + k)
    x, f = rng.normal(size=(2, gp.size(k)))
    out = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.jacobi(k, dev(f), dev(x), out)
    assert rel(host(out), O.jacobi(lv[k - 1], f, x, op.omega)) <= 1e-13


@pytest.mark.parametrize("k", [2, 3, 4])
def test_residual_restrict_and_prolong(setup, k):
    op, gp, lv, s = setup
    rng = np.random.default_rng(300 + k)
    x, f = rng.normal(size=(2, gp.size(k)))
    rc = torch.empty(gp.size(k - 1), dtype=torch.float64, device="cuda")
    s.residual_restrict(k, dev(f), dev(x), rc)
    ref = lv[k - 1].P.T @ (f - lv[k - 1].L @ x)
    assert rel(host(rc), ref) <= 1e-13
    ec = rng.normal(size=gp.size(k - 1))
    xd = dev(x)
    s.prolong_add(k, dev(ec), xd)
    assert rel(host(xd), x + lv[k - 1].P @ ec) <= 1e-14


@pytest.mark.parametrize("k", [1, 3, 4])
def test_nonlinear_load_and_rhs(setup, k):
    op, gp, lv, s = setup
    rng = np.random.default_rng(400 + k)
    u = rng.normal(size=gp.size(k))
    out = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.nonlinear_load(k, dev(u), out)
    assert rel(host(out), O.nonlinear_load(lv[k - 1].mesh, u, 1.0)) <= 1e-13
    s.aux_rhs(k, 23.5, dev(u), out)
    assert rel(host(out), O.aux_rhs(op, lv[k - 1], 23.5, u)) <= 1e-13


@pytest.mark.parametrize("k", [2, 4])
def test_multigrid_vcycles(setup, k):
    op, gp, lv, s = setup
    rng = np.random.default_rng(500 + k)
    x, f = rng.normal(size=(2, gp.size(k)))
    xd = dev(x)
    s.multigrid(k, dev(f), xd)
    assert rel(host(xd), O.multigrid(lv, k, f, x, op.vcycles, op)) <= 1e-12


@pytest.mark.parametrize("k", [2, 3, 4])
def test_augmented_system(setup, k):
    """Algorithm 3.1 step 2's small system from one fine pass (restricted loads, coarsened
    density stencil, per-triangle moments) against its definition Psi^T A Psi, Psi^T M Psi,
    Psi^T B(Psi c) Psi assembled on the fine grid by the oracle."""
    op, gp, lv, s = setup
    rng = np.random.default_rng(600 + k)
    ut = rng.uniform(0.2, 1.0, size=gp.size(k))
    psi, k0, mm = O.augmented_blocks(lv, k, ut)
    c = rng.normal(size=psi.shape[1])
    g_ref = (psi.T @ O.density_matrix(lv[k - 1].mesh, psi @ c) @ psi).toarray()
    K, M, G = s.augmented_system(k, dev(ut), c)
    assert rel(K, k0) <= 1e-12
    assert rel(M, mm) <= 1e-12
    assert rel(G, g_ref) <= 1e-12


def test_coarse_solve(setup):
    op, gp, lv, s = setup
    lam_o, u_o, res = O.coarse_solve(op, lv[0])
    u = torch.empty(gp.size(1), dtype=torch.float64, device="cuda")
    lam, iters, rc = s.coarse_solve(u)
    assert rc == 0 and res.converged
    assert abs(lam - lam_o) <= LAM_TOL * lam_o
    u = host(u)
    assert np.linalg.norm(u - u_o) <= U_TOL * np.linalg.norm(u_o)


@pytest.mark.parametrize("k", [2, 4])
def test_correction_step(setup, k):
    """Algorithm 3.1 from the same (lambda, u): GPU (moments + Newton) vs oracle (fine-grid
    assembly per SCF iteration + dense eigh)."""
    op, gp, lv, s = setup
    r = O.fmg_solve(O.Problem(**{**KW, "levels": k - 1}))
    lam0, u0 = r.lam, lv[k - 1].P @ r.u
    info = O.eigen_mg(op, lv, k, lam0, u0)
    u_out = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    ut = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    lam, iters, rc = s.correction(k, lam0, dev(u0), u_out, ut)
    assert rc == 0
    assert rel(host(ut), info.u_tilde) <= 1e-12
    assert abs(lam - info.lam) <= LAM_TOL * info.lam
    assert np.linalg.norm(host(u_out) - info.u) <= U_TOL * np.linalg.norm(info.u)


CASES = [
    dict(dim=2, coarse_cells=8, levels=4, w_quad=(1.0, 1.0, 0.0), zeta=1.0),
    dict(dim=2, coarse_cells=8, levels=3, w_quad=(1.0, 1.0, 0.0), zeta=10.0),
    dict(dim=2, coarse_cells=5, levels=4, w_const=2.0, w_quad=(3.0, 1.0, 0.0), zeta=150.0),
    dict(dim=2, coarse_cells=3, levels=5, w_quad=(0.0, 0.0, 0.0), zeta=0.0),
    dict(dim=2, coarse_cells=2, levels=4, w_quad=(1.0, 4.0, 0.0), zeta=5.0),
    dict(dim=2, coarse_cells=6, levels=3, box_len=2.0, w_quad=(1.0, 1.0, 0.0), zeta=20.0,
         nu_pre=0, nu_post=3, vcycles=3, corrections=2),
    dict(dim=2, coarse_cells=4, levels=1, zeta=3.0),
]


@pytest.mark.parametrize("kw", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_fmg_solve_matches_oracle(kw):
    op, gp = _pair(**kw)
    ref = O.fmg_solve(op)
    assert ref.converged
    fmg = _fmg()
    with fmg.Solver(gp) as s:
        u = np.empty(gp.size(gp.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) <= LAM_TOL * ref.lam
    assert np.linalg.norm(u - ref.u) <= U_TOL * np.linalg.norm(ref.u)
    for k in range(gp.levels):
        assert abs(st.lambda_levels[k] - ref.lam_levels[k]) <= LAM_TOL * ref.lam_levels[k]
    assert abs(st.norm_defect) < 1e-12
    assert abs(st.identity_defect) < 1e-10 * lam


def test_fmg_config1_seeded_parity():
    """The 2D benchmark discretisation at full size of its first configuration (h = 1/256)."""
    kw = seeded_problem("config1")
    op, gp = _pair(**kw)
    ref = O.fmg_solve(op)
    with _fmg().Solver(gp) as s:
        u = np.empty(gp.size(gp.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) <= LAM_TOL * ref.lam
    assert np.linalg.norm(u - ref.u) <= U_TOL * np.linalg.norm(ref.u)


def test_solve_is_deterministic_and_dev_path_agrees():
    op, gp = _pair(**CASES[0])
    with _fmg().Solver(gp) as s:
        u1 = np.empty(gp.size(gp.levels))
        lam1, _, _ = s.solve(u1)
        lam_d = torch.empty(1, dtype=torch.float64, device="cuda")
        u_d = torch.empty(gp.size(gp.levels), dtype=torch.float64, device="cuda")
        s.solve_dev(lam_d, u_d)
        assert host(lam_d)[0] == lam1
        assert np.array_equal(host(u_d), u1)


def test_invalid_arguments_are_rejected():
    fmg = _fmg()
    bad = [dict(levels=0), dict(coarse_cells=1), dict(zeta=-1.0), dict(omega=0.0), dict(vcycles=0)]
    for b in bad:
        p = fmg.Problem(**{**dict(coarse_cells=4, levels=2), **b})
        with pytest.raises(fmg.FmgError) as e:
            fmg.Solver(p)
        assert e.value.code == fmg.FMG_EINVAL
    with fmg.Solver(fmg.Problem(coarse_cells=4, levels=2)) as s:
        with pytest.raises(fmg.FmgError):
            s.solve(np.empty(5))


@pytest.mark.parametrize("kw", [dict(dim=2, coarse_cells=4, levels=5, w_quad=(1.0, 2.0, 0.0)),
                                dict(dim=2, coarse_cells=5, levels=4, w_quad=(1.0, 2.0, 0.0)),
                                dict(dim=3, coarse_cells=3, levels=4, w_quad=(1.0, 2.0, 3.0))],
                         ids=["2d_64", "2d_40", "3d_24"])
def test_pinned_and_pageable_outputs_agree(kw):
    """fmg_eig_solve copies the interior of u into a pinned host buffer by one strided
    transfer from the padded finest level and stages a pageable one through a packing kernel:
    both give the same u (odd interior widths included: 39 and 23 nodes per row)."""
    fmg = _fmg()
    _, gp = _pair(**kw, zeta=6.0)
    n = gp.size(gp.levels)
    with fmg.Solver(gp) as s:
        pageable = np.empty(n)
        lam1, _, rc1 = s.solve(pageable)
        pinned = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pinned[:] = np.nan
        lam2, _, rc2 = s.solve(pinned)
    assert rc1 == rc2 == 0 and lam1 == lam2
    assert np.array_equal(pageable, pinned)
