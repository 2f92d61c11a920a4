"""GPU parity on the 3D Kuhn mesh: every step through the C ABI against the FP64 oracle
(same tolerances as the 2D tests)."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import LAM_TOL, U_TOL, _fmg, _pair, dev, host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW3 = dict(dim=3, coarse_cells=3, levels=3, w_const=0.4, w_quad=(1.0, 2.0, 3.0), zeta=9.0)


@pytest.fixture(scope="module")
def setup3():
    op, gp = _pair(**KW3)
    levels = O.build_hierarchy(op)
    solver = _fmg().Solver(gp)
    yield op, gp, levels, solver
    solver.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_operator_mass_jacobi_3d(setup3, k):
    op, gp, lv, s = setup3
    rng = np.random.default_rng(700 + k)
    x, f = rng.normal(size=(2, gp.size(k)))
    y = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.apply_operator(k, dev(x), y)
    assert rel(host(y), lv[k - 1].L @ x) <= 1e-13
    s.apply_mass(k, dev(x), y)
    assert rel(host(y), lv[k - 1].M @ x) <= 1e-13
    if k >= 2:
        s.jacobi(k, dev(f), dev(x), y)
        assert rel(host(y), O.jacobi(lv[k - 1], f, x, op.omega)) <= 1e-13


@pytest.mark.parametrize("k", [2, 3])
def test_transfers_3d(setup3, k):
    op, gp, lv, s = setup3
    rng = np.random.default_rng(800 + k)
    x, f = rng.normal(size=(2, gp.size(k)))
    rc = torch.empty(gp.size(k - 1), dtype=torch.float64, device="cuda")
    s.residual_restrict(k, dev(f), dev(x), rc)
    assert rel(host(rc), lv[k - 1].P.T @ (f - lv[k - 1].L @ x)) <= 1e-13
    ec = rng.normal(size=gp.size(k - 1))
    xd = dev(x)
    s.prolong_add(k, dev(ec), xd)
    assert rel(host(xd), x + lv[k - 1].P @ ec) <= 1e-14


@pytest.mark.parametrize("k", [1, 3])
def test_nonlinear_load_rhs_multigrid_3d(setup3, k):
    op, gp, lv, s = setup3
    rng = np.random.default_rng(900 + k)
    u = rng.normal(size=gp.size(k))
    out = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.nonlinear_load(k, dev(u), out)
    assert rel(host(out), O.nonlinear_load(lv[k - 1].mesh, u, 1.0)) <= 1e-13
    s.aux_rhs(k, 31.0, dev(u), out)
    assert rel(host(out), O.aux_rhs(op, lv[k - 1], 31.0, u)) <= 1e-13
    if k >= 2:
        f = rng.normal(size=gp.size(k))
        xd = dev(u)
        s.multigrid(k, dev(f), xd)
        assert rel(host(xd), O.multigrid(lv, k, f, u, op.vcycles, op)) <= 1e-12


@pytest.mark.parametrize("k", [2, 3])
def test_augmented_system_3d(setup3, k):
    op, gp, lv, s = setup3
    rng = np.random.default_rng(1000 + k)
    ut = rng.uniform(0.2, 1.0, size=gp.size(k))
    psi, k0, mm = O.augmented_blocks(lv, k, ut)
    c = rng.normal(size=psi.shape[1])
    g_ref = (psi.T @ O.density_matrix(lv[k - 1].mesh, psi @ c) @ psi).toarray()
    K, M, G = s.augmented_system(k, dev(ut), c)
    assert rel(K, k0) <= 1e-12
    assert rel(M, mm) <= 1e-12
    assert rel(G, g_ref) <= 1e-12


def test_augmented_system_3d_deep_level():
    """T3 / T2 on a level 3 refinements below the coarse mesh (r = 8 fine cells per coarse
    cell), where every class of fine node inside a coarse tetrahedron is populated."""
    op, gp = _pair(dim=3, coarse_cells=3, levels=4, w_const=0.2, w_quad=(1.0, 3.0, 2.0), zeta=4.0)
    lv = O.build_hierarchy(op)
    rng = np.random.default_rng(1100)
    ut = rng.uniform(0.2, 1.0, size=gp.size(4))
    psi, k0, mm = O.augmented_blocks(lv, 4, ut)
    c = rng.normal(size=psi.shape[1])
    g_ref = (psi.T @ O.density_matrix(lv[3].mesh, psi @ c) @ psi).toarray()
    with _fmg().Solver(gp) as s:
        K, M, G = s.augmented_system(4, dev(ut), c)
    assert rel(K, k0) <= 1e-12
    assert rel(M, mm) <= 1e-12
    assert rel(G, g_ref) <= 1e-12


def test_coarse_solve_3d(setup3):
    op, gp, lv, s = setup3
    lam_o, u_o, res = O.coarse_solve(op, lv[0])
    u = torch.empty(gp.size(1), dtype=torch.float64, device="cuda")
    lam, iters, rc = s.coarse_solve(u)
    assert rc == 0 and res.converged
    assert abs(lam - lam_o) <= LAM_TOL * lam_o
    assert np.linalg.norm(host(u) - u_o) <= U_TOL * np.linalg.norm(u_o)


CASES3 = [
    dict(dim=3, coarse_cells=2, levels=3, w_quad=(1.0, 1.0, 1.0), zeta=1.0),
    dict(dim=3, coarse_cells=4, levels=2, w_quad=(100.0, 100.0, 400.0), zeta=100.0),
    dict(dim=3, coarse_cells=3, levels=3, w_const=1.0, w_quad=(2.0, 1.0, 3.0), zeta=30.0,
         vcycles=1, corrections=2),
]


@pytest.mark.parametrize("kw", CASES3, ids=[f"case{i}" for i in range(len(CASES3))])
def test_fmg_solve_3d_matches_oracle(kw):
    op, gp = _pair(**kw)
    ref = O.fmg_solve(op)
    assert ref.converged
    with _fmg().Solver(gp) as s:
        u = np.empty(gp.size(gp.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) <= LAM_TOL * ref.lam
    assert np.linalg.norm(u - ref.u) <= U_TOL * np.linalg.norm(ref.u)
    assert abs(st.norm_defect) < 1e-12
    assert abs(st.identity_defect) < 1e-10 * lam
