"""Pins for the oracle's solver layer: V-cycle (Algorithm 3.1 step 1), SCF on small spaces,
one correction step (Algorithm 3.1) and the full multigrid scheme (Algorithm 3.2).

The references are: the exact linear solve (spsolve), continuum eigenvalues 2 pi^2 / 3 pi^2
with their O(h^2) rate (Assumption B1), brute-force minimisation of the Gross-Pitaevskii
energy with an independent quadrature for int u^4, fixed points implied by Theorem 3.1, and
symmetries of the model problem."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from scipy.optimize import minimize

from oracle import fmg_oracle as O
from tests.quadrature import p1_eval, simplex_points


def quartic_by_quadrature(mesh, u):
    full = mesh.to_full(u)
    tot = 0.0
    for el in mesh.elems:
        x, w = simplex_points(mesh.coords[el], mesh.dim)
        tot += np.sum(w * p1_eval(mesh.coords[el], full[el], x) ** 4)
    return tot


@pytest.mark.parametrize("dim,ns,limit", [(2, (8, 16, 32), 2 * np.pi ** 2), (3, (4, 8, 16), 3 * np.pi ** 2)])
def test_laplace_eigenvalue_converges_at_h_squared(dim, ns, limit):
    """W = 0, zeta = 0: lambda_h -> d pi^2 from above with error ratio ~4 per halving."""
    errs = []
    for n in ns:
        mesh = O.Mesh(dim, n, 1.0)
        lam = spla.eigsh(O.stiffness(mesh).tocsc(), k=1, M=O.mass(mesh).tocsc(), sigma=0.0, which="LM")[0][0]
        assert lam > limit
        errs.append(lam - limit)
    r = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < x < 4.4 for x in r), r


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("omega", [2.0 / 3.0, 0.8])
def test_jacobi_damps_each_sine_mode_by_its_closed_form_factor(dim, omega):
    """W = 0: the P1 stiffness is the (2d+1)-point Laplacian (diagonal 4 in 2D, 6h on the 3D Kuhn
    mesh), whose eigenvectors are the discrete sine modes, so one damped Jacobi sweep with
    f = 0 multiplies the mode (k_1 .. k_d) by 1 - omega (2d - 2 sum cos(k_i pi h)) / (2d).
    A wrong damping, diagonal, sign or operator changes that factor."""
    n = 8 if dim == 2 else 6
    prob = O.Problem(dim=dim, coarse_cells=n, levels=1, w_const=0.0, w_quad=(0.0, 0.0, 0.0),
                     omega=omega)
    lev = O.build_hierarchy(prob)[0]
    ijk = lev.mesh.ijk[lev.mesh.interior]
    h = 1.0 / n
    for ks in [(1, 1, 1), (3, 5, 2), (n - 1, n - 1, n - 1), (1, n - 1, 4)]:
        x = np.ones(len(ijk))
        for ax in range(dim):
            x *= np.sin(ks[ax] * np.pi * ijk[:, ax] * h)
        factor = 1.0 - omega * (2 * dim - 2 * sum(np.cos(ks[ax] * np.pi * h) for ax in range(dim))) / (2 * dim)
        y = O.jacobi(lev, np.zeros_like(x), x, omega)
        assert np.max(np.abs(y - factor * x)) <= 1e-14, (ks, factor)


def test_level_solve_minimises_gp_energy():
    """The SCF ground state equals the brute-force minimiser of
    E(u) = 1/2 u^T (A + W) u + zeta/4 int u^4 on u^T M u = 1 (int u^4 by independent quadrature)."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=1, w_quad=(1.0, 2.0, 0.0), zeta=5.0)
    lev = O.build_hierarchy(prob)[0]
    lam, u, res = O.discrete_ground_state(prob, lev)
    assert res.converged
    k = (lev.A + lev.Wm).toarray()
    mm = lev.M.toarray()

    def energy(v):
        v = v / np.sqrt(v @ mm @ v)
        return 0.5 * v @ k @ v + prob.zeta / 4 * quartic_by_quadrature(lev.mesh, v)

    best = minimize(energy, np.ones(lev.mesh.n_interior), method="BFGS", options={"gtol": 1e-11})
    v = best.x / np.sqrt(best.x @ mm @ best.x)
    v = v if v.sum() > 0 else -v
    assert np.abs(v - u).max() < 1e-5
    lam_bf = v @ k @ v + prob.zeta * quartic_by_quadrature(lev.mesh, v)
    assert abs(lam_bf - lam) < 1e-8 * lam


def test_lambda_identity_and_symmetry():
    """lambda = a^(u,u) + (W u,u) + zeta int u^4 with b(u,u) = 1 (Example 4.1 tested against u
    itself), and u(x,y) = u(y,x) when W is symmetric (the (1,1)-diagonal mesh is too)."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=3, zeta=3.0)
    lv = O.build_hierarchy(prob)
    r = O.fmg_solve(prob, lv)
    fine = lv[-1]
    au, q4, bu = O.gp_energy_parts(prob, fine, r.u)
    assert abs(bu - 1) < 1e-13
    q4_ind = quartic_by_quadrature(fine.mesh, r.u)
    assert abs(au + prob.zeta * q4_ind - r.lam) < 1e-11 * r.lam
    m = fine.mesh.n - 1
    grid = r.u.reshape(m, m)
    assert np.abs(grid - grid.T).max() < 1e-11
    assert np.all(r.u > 0)


def test_lambda_increases_with_zeta():
    lams = []
    for z in (0.0, 1.0, 10.0, 50.0):
        prob = O.Problem(dim=2, coarse_cells=4, levels=2, zeta=z)
        lams.append(O.fmg_solve(prob).lam)
    assert all(a < b for a, b in zip(lams, lams[1:]))


@pytest.mark.parametrize("dim,nc,levels", [(2, 4, 4), (3, 2, 3)])
def test_vcycle_converges_to_exact_solve(dim, nc, levels):
    prob = O.Problem(dim=dim, coarse_cells=nc, levels=levels, w_quad=(1.0, 1.0, 1.0))
    lv = O.build_hierarchy(prob)
    fine = lv[-1]
    rng = np.random.default_rng(5)
    f = rng.normal(size=fine.mesh.n_interior)
    exact = spla.spsolve(fine.L.tocsc(), f)
    x = np.zeros_like(f)
    errs = []
    for _ in range(16):
        x = O.vcycle(lv, levels, f, x, prob)
        errs.append(np.linalg.norm(x - exact))
    rate = (errs[10] / errs[2]) ** (1 / 8)
    assert rate < 0.35, rate
    assert errs[-1] < 1e-6 * np.linalg.norm(exact)


def test_two_level_cycle_with_exact_coarse_grid():
    """With levels = 2 the V-cycle is a two-grid cycle: zero smoothing leaves exactly the
    Galerkin coarse-grid correction, whose residual is orthogonal to range(P)."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=2, nu_pre=0, nu_post=0)
    lv = O.build_hierarchy(prob)
    fine = lv[-1]
    rng = np.random.default_rng(2)
    f = rng.normal(size=fine.mesh.n_interior)
    x = O.vcycle(lv, 2, f, np.zeros_like(f), prob)
    r = f - fine.L @ x
    assert np.abs(fine.P.T @ r).max() < 1e-12


@pytest.mark.parametrize("form", [O.W_LEFT, O.PAPER_LITERAL])
def test_correction_fixed_point(form):
    """Theorem 3.1 with u^(l) = the discrete solution: the auxiliary solution equals it, so it
    lies in V_{H,h_k} and EigenMG returns it unchanged."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=2, zeta=4.0, operator_form=form, vcycles=3)
    lv = O.build_hierarchy(prob)
    lam, u, res = O.discrete_ground_state(prob, lv[-1])
    info = O.eigen_mg(prob, lv, 2, lam, u)
    assert abs(info.lam - lam) < 1e-11 * lam
    assert np.abs(info.u - u).max() < 1e-9
    assert np.abs(info.u_tilde - u).max() < 1e-9


def test_correction_contracts_error():
    """Repeated corrections converge geometrically to the discrete solution (gamma < 1)."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=3, zeta=2.0, vcycles=1)
    lv = O.build_hierarchy(prob)
    lam_h, u_h, _ = O.discrete_ground_state(prob, lv[-1])
    a = (lv[-1].A).tocsr()
    r = O.fmg_solve(O.Problem(dim=2, coarse_cells=4, levels=2, zeta=2.0, vcycles=1))
    lam, u = r.lam, lv[-1].P @ r.u
    errs = []
    for _ in range(6):
        e = u - u_h
        errs.append(np.sqrt(e @ (a @ e)))
        info = O.eigen_mg(prob, lv, 3, lam, u)
        lam, u = info.lam, info.u
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1)]
    assert max(ratios) < 0.5, ratios


def test_augmented_solution_minimises_energy_on_augmented_space():
    """Step 2 of Algorithm 3.1 gives the GP ground state on V_H + span{u~}: it matches a
    brute-force energy minimisation over that space and lies between the energy bounds."""
    prob = O.Problem(dim=2, coarse_cells=2, levels=3, zeta=6.0, w_quad=(1.0, 3.0, 0.0))
    lv = O.build_hierarchy(prob)
    r2 = O.fmg_solve(O.Problem(dim=2, coarse_cells=2, levels=2, zeta=6.0, w_quad=(1.0, 3.0, 0.0)))
    lam0, u0 = r2.lam, lv[-1].P @ r2.u
    info = O.eigen_mg(prob, lv, 3, lam0, u0)
    psi, k0, mm = O.augmented_blocks(lv, 3, info.u_tilde)
    fine = lv[-1]

    def energy_c(c):
        c = c / np.sqrt(c @ mm @ c)
        v = psi @ c
        return 0.5 * c @ k0 @ c + prob.zeta / 4 * quartic_by_quadrature(fine.mesh, v)

    c0 = np.zeros(psi.shape[1])
    c0[-1] = 1.0
    best = minimize(energy_c, c0, method="BFGS", options={"gtol": 1e-12})
    c = best.x / np.sqrt(best.x @ mm @ best.x)
    c = c if c[-1] > 0 else -c
    assert np.abs(psi @ c - info.u).max() < 1e-5

    def energy(v):
        k = lv[-1].A + lv[-1].Wm
        return 0.5 * v @ (k @ v) + prob.zeta / 4 * O.quartic(fine.mesh, v)

    ut = info.u_tilde / np.sqrt(info.u_tilde @ (fine.M @ info.u_tilde))
    _, u_h, _ = O.discrete_ground_state(prob, fine)
    assert energy(u_h) - 1e-12 <= energy(info.u) <= energy(ut) + 1e-12


def test_fmg_converges_to_discrete_solution_with_many_corrections():
    prob = O.Problem(dim=2, coarse_cells=4, levels=3, zeta=8.0, corrections=12)
    lv = O.build_hierarchy(prob)
    lam_h, u_h, _ = O.discrete_ground_state(prob, lv[-1])
    r = O.fmg_solve(prob, lv)
    assert abs(r.lam - lam_h) < 1e-11 * lam_h
    assert np.abs(r.u - u_h).max() < 1e-8


def test_fmg_error_far_below_discretisation_error():
    """Theorem 3.2: with p = 1 the FMG eigenvalue is much closer to the discrete one than the
    discrete one is to the next coarser level's (the O(h^2) discretisation error)."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=4, zeta=1.0)
    lv = O.build_hierarchy(prob)
    r = O.fmg_solve(prob, lv)
    lam_h, _, _ = O.discrete_ground_state(prob, lv[-1])
    lam_2h, _, _ = O.discrete_ground_state(prob, lv[-2])
    assert abs(r.lam - lam_h) < 0.05 * abs(lam_2h - lam_h)


def test_fmg_3d_kuhn_small():
    prob = O.Problem(dim=3, coarse_cells=2, levels=3, zeta=2.0, w_quad=(1.0, 1.0, 4.0))
    lv = O.build_hierarchy(prob)
    r = O.fmg_solve(prob, lv)
    assert r.converged
    au, q4, bu = O.gp_energy_parts(prob, lv[-1], r.u)
    assert abs(bu - 1) < 1e-13 and abs(au + prob.zeta * q4 - r.lam) < 1e-11 * r.lam
    lam_h, _, _ = O.discrete_ground_state(prob, lv[-1])
    lam_2h, _, _ = O.discrete_ground_state(prob, lv[-2])
    assert abs(r.lam - lam_h) < 0.1 * abs(lam_2h - lam_h)



def _cheb_poly(t, degree, low=O.CHEB_LOW, high=O.CHEB_HIGH):
    """The closed-form residual polynomial T_k((theta - t) / delta) / T_k(theta / delta)."""
    theta, delta = 0.5 * (high + low), 0.5 * (high - low)
    tk = np.polynomial.chebyshev.Chebyshev.basis(degree)
    return tk((theta - t) / delta) / tk(theta / delta)


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_error_is_the_chebyshev_polynomial_of_the_spectrum(degree):
    """The error after the semi-iteration is p(D^-1 L) e0 with p the scaled Chebyshev
    polynomial: on each eigenvector of D^-1 L the error shrinks by p(its eigenvalue)."""
    prob = O.Problem(dim=2, coarse_cells=6, levels=1, w_const=0.5, w_quad=(2.0, 1.0, 0.0))
    lev = O.build_hierarchy(prob)[0]
    L = lev.L.toarray()
    Dm = np.diag(1.0 / lev.D)
    lam, V = np.linalg.eig(Dm @ L)
    lam, V = lam.real, V.real
    rng = np.random.default_rng(degree)
    x_true = rng.normal(size=L.shape[0])
    f = L @ x_true
    x0 = rng.normal(size=L.shape[0])
    x = O.chebyshev(lev, f, x0, degree)
    coef0 = np.linalg.solve(V, x0 - x_true)
    coef1 = np.linalg.solve(V, x - x_true)
    assert np.allclose(coef1, _cheb_poly(lam, degree) * coef0, rtol=1e-9, atol=1e-12)


def test_gershgorin_interval_contains_the_spectrum():
    for dim, nc in ((2, 8), (3, 4)):
        prob = O.Problem(dim=dim, coarse_cells=nc, levels=1, w_const=3.0, w_quad=(50.0, 20.0, 80.0))
        lev = O.build_hierarchy(prob)[0]
        lam = np.linalg.eigvals(np.diag(1.0 / lev.D) @ lev.L.toarray()).real
        assert lam.max() <= O.CHEB_HIGH and lam.min() > 0.0


def test_chebyshev_vcycle_converges_faster_than_jacobi():
    errs = {}
    for sm in (O.SMOOTH_JACOBI, O.SMOOTH_CHEBYSHEV):
        prob = O.Problem(dim=2, coarse_cells=4, levels=4, w_quad=(1.0, 1.0, 0.0), smoother=sm)
        lv = O.build_hierarchy(prob)
        lev = lv[-1]
        rng = np.random.default_rng(3)
        x_true = rng.normal(size=lev.L.shape[0])
        f = lev.L @ x_true
        x = O.multigrid(lv, 4, f, np.zeros_like(f), 4, prob)
        errs[sm] = np.linalg.norm(x - x_true) / np.linalg.norm(x_true)
    assert errs[O.SMOOTH_CHEBYSHEV] < 0.8 * errs[O.SMOOTH_JACOBI]


def test_cg_steps_terminate_at_the_exact_solution():
    """CG on an SPD system of N unknowns reaches the solution in N steps (finite
    termination, exact arithmetic): pinned on a 9-unknown level against a dense solve."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=1, w_const=0.5, w_quad=(2.0, 1.0, 0.0))
    lev = O.build_hierarchy(prob)[0]
    L = lev.L.toarray()
    rng = np.random.default_rng(17)
    f = rng.normal(size=L.shape[0])
    x0 = rng.normal(size=L.shape[0])
    x = O.cg_steps(lev, f, x0, L.shape[0])
    assert np.allclose(x, np.linalg.solve(L, f), rtol=1e-10, atol=1e-12)


def test_cg_first_step_is_steepest_descent_with_exact_line_search():
    prob = O.Problem(dim=3, coarse_cells=3, levels=1, w_quad=(1.0, 2.0, 3.0))
    lev = O.build_hierarchy(prob)[0]
    L = lev.L.toarray()
    rng = np.random.default_rng(5)
    f = rng.normal(size=L.shape[0])
    x0 = rng.normal(size=L.shape[0])
    r = f - L @ x0
    x1 = x0 + (r @ r) / (r @ L @ r) * r
    assert np.allclose(O.cg_steps(lev, f, x0, 1), x1, rtol=1e-13, atol=1e-14)


def test_cg_energy_error_decreases_and_minimises_over_the_krylov_space():
    """The k-th CG iterate minimises the L-energy error over x0 + K_k(L, r0): checked
    against the minimiser computed from an explicit Krylov basis."""
    prob = O.Problem(dim=2, coarse_cells=6, levels=1, w_const=1.0, w_quad=(3.0, 1.0, 0.0))
    lev = O.build_hierarchy(prob)[0]
    L = lev.L.toarray()
    rng = np.random.default_rng(9)
    x_true = rng.normal(size=L.shape[0])
    f = L @ x_true
    x0 = np.zeros_like(f)
    r0 = f - L @ x0
    prev = np.inf
    for k in (1, 2, 3):
        x = O.cg_steps(lev, f, x0, k)
        e = x - x_true
        en = e @ L @ e
        assert en < prev
        prev = en
        K = np.stack([np.linalg.matrix_power(L, i) @ r0 for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        c = np.linalg.solve(Q.T @ L @ Q, Q.T @ (f - L @ x0))
        assert np.allclose(x, x0 + Q @ c, rtol=1e-9, atol=1e-11)


def test_cg_smoothed_vcycle_converges():
    """The paper's setting (3 + 3 CG smoothing steps) gives a convergent V-cycle."""
    prob = O.Problem(dim=2, coarse_cells=4, levels=4, w_quad=(1.0, 1.0, 0.0),
                     smoother=O.SMOOTH_CG, nu_pre=3, nu_post=3)
    lv = O.build_hierarchy(prob)
    lev = lv[-1]
    rng = np.random.default_rng(3)
    x_true = rng.normal(size=lev.L.shape[0])
    f = lev.L @ x_true
    e = [np.linalg.norm(x_true)]
    x = np.zeros_like(f)
    for _ in range(4):
        x = O.vcycle(lv, 4, f, x, prob)
        e.append(np.linalg.norm(x - x_true))
    assert all(e[i + 1] < 0.5 * e[i] for i in range(4))
