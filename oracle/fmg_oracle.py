"""Plain FP64 CPU oracle for the full multigrid / multilevel-correction method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.  The
GPU library never calls it, and the two share no code, tables or constants.

What it computes (Jia, Xie, Xie, Xu, "A Full Multigrid Method for Nonlinear Eigenvalue
Problems", arXiv:1502.04657):

* the Gross-Pitaevskii eigenproblem of Example 4.1, -Lap u + W u + zeta u^3 = lambda u on
  [0, L]^d, u = 0 on the boundary, int u^2 = 1 (Section 2, the model problem; Example 4.1),
* discretised by linear finite elements (Section 2, the P1 space V_h) on nested, regularly
  refined structured meshes with refinement index beta = 2 (Section 3, the mesh sequence),
* solved by the full multigrid scheme (Algorithm 3.2), whose levels apply the one-correction
  step EigenMG (Algorithm 3.1): m multigrid iterations on the auxiliary linear problem, then
  the nonlinear eigenproblem on the augmented space V_H + span{u~}.

Everything is written from definitions, with no blocking, fusion or reordering:

* element matrices and nonlinear terms use the exact barycentric monomial rule
  int_K lambda^alpha = d! |K| alpha! / (|alpha| + d)!  (all integrands are polynomials of
  degree <= 4, so this is exact, and equals any exact degree-4 quadrature rule);
* global matrices are assembled element by element into scipy CSR matrices;
* the prolongation is the nested-space embedding, obtained by evaluating each coarse hat
  function at each fine node through point location and barycentric coordinates;
* the multigrid iteration is a V-cycle with damped Jacobi smoothing, rediscretised level
  operators, the FE restriction P^T and an exact (Cholesky) solve on the coarsest level;
* every nonlinear eigenproblem on a small space is solved by self-consistent-field (SCF)
  iteration, each step a dense generalised symmetric eigensolve (scipy.linalg.eigh) whose
  lowest eigenpair is taken (the paper names SCF, Section 3.2), with a fixed density-mixing
  rule.

Readings of the paper where it is silent:
* meshes: 2D squares split along their (1,1) diagonal, 3D cubes split into the 6 Kuhn
  tetrahedra;
* W sits on the left of the auxiliary problem, (A + W) u^ = lambda M u - N(u) (operator
  form "W_LEFT"); "PAPER_LITERAL" keeps only the stiffness on the left, as Algorithm 3.1
  writes it, and moves W u to the right-hand side;
* V_H = V_{h_1}: the coarse space of the correction is the first level;
* the sign of every eigenvector is fixed by sum(u) > 0 on level 1 and by a positive
  coefficient of u~ in the augmented space.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from math import factorial

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

W_LEFT = 0
PAPER_LITERAL = 1
SMOOTH_JACOBI = 0
SMOOTH_CHEBYSHEV = 1
SMOOTH_CG = 2  # Section 4: "3 conjugate gradient smooth steps" (plain CG on L_j x = f)
# Chebyshev smoothing interval [CHEB_LOW, CHEB_HIGH] for the spectrum of D^{-1} L: the upper
# end is Gershgorin's bound for these operators (the stiffness rows sum to zero and the
# potential mass has the P1 mass pattern, so every row of D^{-1} L has |off-diagonal| sum at
# most 1, and the spectrum does reach close to 2); the smoother damps the part above the
# lower end and leaves the smooth part to the coarse grid.  0.3 gave the fastest V-cycle
# among 0.1..0.7 on 2D and 3D model problems (0.21 / 0.24 per cycle with degree 2 + 2,
# against 0.27 / 0.38 for 2 + 2 damped Jacobi).
CHEB_LOW = 0.3
CHEB_HIGH = 2.0


# --------------------------------------------------------------------------------------
# Exact integration on a simplex (Section 2: P1 elements; all integrands are polynomials)
# --------------------------------------------------------------------------------------
def bary_monomial_integral(alpha, vol: float, d: int) -> float:
    """int_K prod_i lambda_i^alpha_i = d! |K| prod(alpha_i!) / (|alpha| + d)!."""
    num = factorial(d)
    for a in alpha:
        num *= factorial(a)
    return vol * num / factorial(sum(alpha) + d)


def bary_tensor(order: int, d: int) -> np.ndarray:
    """T[i1..i_order] = int_K lambda_i1 ... lambda_i_order / |K| on any d-simplex."""
    shape = (d + 1,) * order
    t = np.empty(shape)
    for idx in np.ndindex(*shape):
        alpha = [idx.count(v) for v in range(d + 1)]
        t[idx] = bary_monomial_integral(alpha, 1.0, d)
    return t


# --------------------------------------------------------------------------------------
# Structured nested meshes (Section 3: T_{h_k} from T_{h_{k-1}} by one regular refinement)
# --------------------------------------------------------------------------------------
_KUHN_PERMS = list(itertools.permutations(range(3)))


@dataclass
class Mesh:
    """Uniform P1 mesh of [0, L]^d with n cells per side.

    Nodes are numbered lexicographically over the (n+1)^d grid, x fastest.  ``interior``
    lists the interior nodes in that order, which is the vector layout of every oracle
    function (Dirichlet values are zero and are not stored)."""

    dim: int
    n: int
    L: float
    h: float = field(init=False)
    coords: np.ndarray = field(init=False)   # (n_nodes, dim)
    ijk: np.ndarray = field(init=False)      # integer grid index per node
    elems: np.ndarray = field(init=False)    # (n_elems, dim+1) node ids
    interior: np.ndarray = field(init=False)

    def __post_init__(self):
        d, n = self.dim, self.n
        self.h = self.L / n
        grids = np.meshgrid(*([np.arange(n + 1)] * d), indexing="ij")
        # lexicographic, x fastest: reverse the meshgrid axes
        ijk = np.stack([g.ravel() for g in grids[::-1]], axis=1)
        self.ijk = ijk
        self.coords = ijk * self.h
        stride = (n + 1) ** np.arange(d)
        cells = np.stack([g.ravel() for g in np.meshgrid(*([np.arange(n)] * d), indexing="ij")[::-1]], 1)
        base = cells @ stride
        if d == 2:
            e = np.array([1, 0]) @ stride, np.array([1, 1]) @ stride, np.array([0, 1]) @ stride
            t1 = np.stack([base, base + e[0], base + e[1]], 1)   # (i,j),(i+1,j),(i+1,j+1)
            t2 = np.stack([base, base + e[1], base + e[2]], 1)   # (i,j),(i+1,j+1),(i,j+1)
            self.elems = np.stack([t1, t2], 1).reshape(-1, 3)
        elif d == 3:
            tets = []
            for p in _KUHN_PERMS:
                v1 = np.zeros(3, int)
                v1[p[0]] = 1
                v2 = v1.copy()
                v2[p[1]] = 1
                tets.append(np.stack([base, base + v1 @ stride, base + v2 @ stride,
                                      base + np.ones(3, int) @ stride], 1))
            self.elems = np.stack(tets, 1).reshape(-1, 4)
        else:
            raise ValueError("dim must be 2 or 3")
        inner = np.all((ijk > 0) & (ijk < n), axis=1)
        self.interior = np.flatnonzero(inner)

    @property
    def n_nodes(self) -> int:
        return (self.n + 1) ** self.dim

    @property
    def n_interior(self) -> int:
        return (self.n - 1) ** self.dim

    def geometry(self):
        """Per element: volume |K| and barycentric gradients grad lambda_a, (E, d+1, d)."""
        x = self.coords[self.elems]                    # (E, d+1, d)
        b = x[:, 1:, :] - x[:, :1, :]                  # rows: edge vectors X_i - X_0
        vol = np.abs(np.linalg.det(b)) / factorial(self.dim)
        ginv = np.linalg.inv(b)                        # lambda_{1..d} = (x - X_0) @ ginv
        g = np.transpose(ginv, (0, 2, 1))              # g[:, i, :] = grad lambda_{i+1}
        g0 = -g.sum(axis=1, keepdims=True)
        return vol, np.concatenate([g0, g], axis=1)

    def to_full(self, u: np.ndarray) -> np.ndarray:
        full = np.zeros(self.n_nodes)
        full[self.interior] = u
        return full


def _assemble(mesh: Mesh, local: np.ndarray) -> sp.csr_matrix:
    """Sum element matrices (E, d+1, d+1) into a global matrix restricted to interior nodes."""
    e = mesh.elems
    k = e.shape[1]
    rows = np.repeat(e, k, axis=1).ravel()
    cols = np.tile(e, (1, k)).ravel()
    a = sp.coo_matrix((local.ravel(), (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes)).tocsr()
    idx = mesh.interior
    return a[idx][:, idx].tocsr()


def _assemble_vec(mesh: Mesh, local: np.ndarray) -> np.ndarray:
    v = np.zeros(mesh.n_nodes)
    np.add.at(v, mesh.elems.ravel(), local.ravel())
    return v[mesh.interior]


# --------------------------------------------------------------------------------------
# Bilinear forms (Section 2: a(u,v), b(u,v) and a^(w,v); Example 4.1: f(x,u) = W u + zeta u^3)
# --------------------------------------------------------------------------------------
def stiffness(mesh: Mesh) -> sp.csr_matrix:
    """A_ij = int grad phi_i . grad phi_j  (the form a^ of Section 2 with the identity matrix)."""
    vol, g = mesh.geometry()
    local = vol[:, None, None] * np.einsum("eai,ebi->eab", g, g)
    return _assemble(mesh, local)


def mass(mesh: Mesh) -> sp.csr_matrix:
    """M_ij = b(phi_i, phi_j) = int phi_i phi_j."""
    vol, _ = mesh.geometry()
    t2 = bary_tensor(2, mesh.dim)
    return _assemble(mesh, vol[:, None, None] * t2[None])


def potential_mass(mesh: Mesh, w_const: float, w_quad) -> sp.csr_matrix:
    """W_ij = int W phi_i phi_j with W(x) = w_const + sum_d w_quad[d] x_d^2 (exact).

    x_d = sum_v X_{v,d} lambda_v on each element, so x_d^2 phi_a phi_b is a degree-4
    barycentric polynomial integrated by the monomial rule."""
    vol, _ = mesh.geometry()
    t2 = bary_tensor(2, mesh.dim)
    t4 = bary_tensor(4, mesh.dim)
    x = mesh.coords[mesh.elems]
    local = w_const * t2[None] * np.ones((len(vol), 1, 1))
    for d in range(mesh.dim):
        if w_quad[d] != 0.0:
            xd = x[:, :, d]
            local = local + w_quad[d] * np.einsum("ev,ew,vwab->eab", xd, xd, t4)
    return _assemble(mesh, vol[:, None, None] * local)


def nonlinear_load(mesh: Mesh, u: np.ndarray, zeta: float) -> np.ndarray:
    """N(u)_i = zeta int u^3 phi_i (the zeta |u|^2 u part of f(x,u) in Example 4.1)."""
    vol, _ = mesh.geometry()
    t4 = bary_tensor(4, mesh.dim)
    ue = mesh.to_full(u)[mesh.elems]
    local = vol[:, None] * np.einsum("ev,ew,ez,vwza->ea", ue, ue, ue, t4)
    return zeta * _assemble_vec(mesh, local)


def density_matrix(mesh: Mesh, w: np.ndarray) -> sp.csr_matrix:
    """B(w)_ij = int w^2 phi_i phi_j, so that (B(w) u)_i = int w^2 u phi_i."""
    vol, _ = mesh.geometry()
    t4 = bary_tensor(4, mesh.dim)
    we = mesh.to_full(w)[mesh.elems]
    local = vol[:, None, None] * np.einsum("ev,ew,vwab->eab", we, we, t4)
    return _assemble(mesh, local)


def quartic(mesh: Mesh, u: np.ndarray) -> float:
    """int u^4."""
    vol, _ = mesh.geometry()
    t4 = bary_tensor(4, mesh.dim)
    ue = mesh.to_full(u)[mesh.elems]
    per = np.einsum("ea,eb,ec,ed,abcd->e", ue, ue, ue, ue, t4)
    return float(np.dot(vol, per))


# --------------------------------------------------------------------------------------
# Nested-space embedding V_{h_{k-1}} -> V_{h_k} (Section 3, the nested spaces)
# --------------------------------------------------------------------------------------
def locate(coarse: Mesh, ijk_fine: np.ndarray, ratio: int) -> np.ndarray:
    """Index of a coarse element that contains each fine node (given by its grid index)."""
    d, nc = coarse.dim, coarse.n
    cell = np.minimum(ijk_fine // ratio, nc - 1)
    rem = ijk_fine - cell * ratio                      # local position in units of h_fine
    stride = nc ** np.arange(d)
    c = cell @ stride
    if d == 2:
        upper = rem[:, 1] > rem[:, 0]                  # above the (1,1) diagonal -> 2nd triangle
        return 2 * c + upper.astype(int)
    order = np.argsort(-rem, axis=1, kind="stable")    # x_{s1} >= x_{s2} >= x_{s3}
    lookup = {p: i for i, p in enumerate(_KUHN_PERMS)}
    local = np.array([lookup[tuple(o)] for o in order])
    return 6 * c + local


def prolongation(coarse: Mesh, fine: Mesh) -> sp.csr_matrix:
    """P with (P v_c)(x_f) = v_c(x_f): P_fc = phi^coarse_c(x_f), interior rows and columns."""
    ratio = fine.n // coarse.n
    assert ratio * coarse.n == fine.n
    fidx = fine.interior
    el = locate(coarse, fine.ijk[fidx], ratio)
    verts = coarse.elems[el]                           # (F, d+1)
    x0 = coarse.coords[verts[:, 0]]
    b = coarse.coords[verts[:, 1:]] - x0[:, None, :]
    lam_rest = np.einsum("fi,fij->fj", fine.coords[fidx] - x0, np.linalg.inv(b))
    lam = np.concatenate([1.0 - lam_rest.sum(1, keepdims=True), lam_rest], axis=1)
    lam[np.abs(lam) < 1e-12] = 0.0                     # exact zeros on faces
    rows = np.repeat(np.arange(len(fidx)), verts.shape[1])
    p = sp.coo_matrix((lam.ravel(), (rows, verts.ravel())), shape=(len(fidx), coarse.n_nodes)).tocsr()
    return p[:, coarse.interior].tocsr()


# --------------------------------------------------------------------------------------
# Problem description and level hierarchy
# --------------------------------------------------------------------------------------
@dataclass
class Problem:
    """The parameters of the model problem (Example 4.1) and of Algorithms 3.1/3.2."""

    dim: int = 2
    box_len: float = 1.0
    coarse_cells: int = 8          # cells per side of T_{h_1} = T_H
    levels: int = 3                # n of Algorithm 3.2
    w_const: float = 0.0
    w_quad: tuple = (1.0, 1.0, 1.0)
    zeta: float = 1.0
    nu_pre: int = 2
    nu_post: int = 2
    omega: float = 2.0 / 3.0
    vcycles: int = 2               # m of Algorithm 3.1
    corrections: int = 1           # p of Algorithm 3.2
    operator_form: int = W_LEFT
    smoother: int = SMOOTH_JACOBI  # Chebyshev: degree nu_pre / nu_post on [CHEB_LOW, CHEB_HIGH];
    # CG: nu_pre / nu_post conjugate gradient steps
    scf_tol: float = 1e-13
    scf_max_iter: int = 500

    def cells(self, k: int) -> int:
        """Cells per side on level k = 1..levels (h_k = h_{k-1} / 2)."""
        return self.coarse_cells << (k - 1)


@dataclass
class Level:
    mesh: Mesh
    A: sp.csr_matrix
    M: sp.csr_matrix
    Wm: sp.csr_matrix
    L: sp.csr_matrix                 # operator of the auxiliary problem (A + W or A)
    D: np.ndarray                    # diagonal of L
    P: sp.csr_matrix | None          # prolongation from the level below (None on level 1)


def build_level(prob: Problem, k: int, coarse: Level | None) -> Level:
    mesh = Mesh(prob.dim, prob.cells(k), prob.box_len)
    a = stiffness(mesh)
    m = mass(mesh)
    wm = potential_mass(mesh, prob.w_const, prob.w_quad)
    lop = (a + wm).tocsr() if prob.operator_form == W_LEFT else a
    p = prolongation(coarse.mesh, mesh) if coarse is not None else None
    return Level(mesh, a, m, wm, lop, lop.diagonal().copy(), p)


def build_hierarchy(prob: Problem, upto: int | None = None) -> list[Level]:
    levels: list[Level] = []
    for k in range(1, (upto or prob.levels) + 1):
        levels.append(build_level(prob, k, levels[-1] if levels else None))
    return levels


# --------------------------------------------------------------------------------------
# Multigrid iteration MG(V, f, x0, m) (Algorithm 3.1, step 1)
# --------------------------------------------------------------------------------------
def jacobi(lev: Level, f: np.ndarray, x: np.ndarray, omega: float) -> np.ndarray:
    """One damped Jacobi sweep x <- x + omega D^{-1} (f - L x)."""
    return x + omega * (f - lev.L @ x) / lev.D


def chebyshev_coefficients(degree: int, low: float = CHEB_LOW, high: float = CHEB_HIGH):
    """(alpha_k, beta_k), k < degree, of the Chebyshev semi-iteration on [low, high]
    (the three-term recurrence of Chebyshev acceleration, e.g. Saad, Iterative Methods for
    Sparse Linear Systems, Sec. 12.3): with theta = (high + low)/2, delta = (high - low)/2,
    sigma = theta/delta, rho_0 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1}),
        d_0 = D^{-1} r_0 / theta,  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^{-1} r_k,
        x_{k+1} = x_k + d_k."""
    theta, delta = 0.5 * (high + low), 0.5 * (high - low)
    sigma = theta / delta
    out = [(0.0, 1.0 / theta)]
    rho = 1.0 / sigma
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        out.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return out


def chebyshev(lev: Level, f: np.ndarray, x: np.ndarray, degree: int) -> np.ndarray:
    """degree steps of the Chebyshev semi-iteration for L x = f preconditioned by D."""
    d = np.zeros_like(x)
    for alpha, beta in chebyshev_coefficients(degree):
        d = alpha * d + beta * (f - lev.L @ x) / lev.D
        x = x + d
    return x


def cg_steps(lev: Level, f: np.ndarray, x: np.ndarray, steps: int) -> np.ndarray:
    """steps iterations of the conjugate gradient method (Hestenes-Stiefel, no
    preconditioner) for L x = f from x: the smoother of the paper's experiments (Section 4).
    A zero denominator (an exact x, or f = 0) ends the steps with a zero update."""
    r = f - lev.L @ x
    p = r.copy()
    rr = float(r @ r)
    for _ in range(steps):
        q = lev.L @ p
        pq = float(p @ q)
        alpha = rr / pq if pq > 0.0 else 0.0
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr if rr > 0.0 else 0.0
        p = r + beta * p
        rr = rr_new
    return x


def smooth(lev: Level, f: np.ndarray, x: np.ndarray, nu: int, prob: Problem) -> np.ndarray:
    if prob.smoother == SMOOTH_CHEBYSHEV:
        return chebyshev(lev, f, x, nu) if nu > 0 else x
    if prob.smoother == SMOOTH_CG:
        return cg_steps(lev, f, x, nu)
    for _ in range(nu):
        x = jacobi(lev, f, x, prob.omega)
    return x


def vcycle(levels: list[Level], j: int, f: np.ndarray, x: np.ndarray, prob: Problem) -> np.ndarray:
    """One V-cycle on level j (1-based) for L_j x = f."""
    lev = levels[j - 1]
    if j == 1:
        return sla.cho_solve(sla.cho_factor(lev.L.toarray()), f)
    x = smooth(lev, f, x, prob.nu_pre, prob)
    r = f - lev.L @ x
    rc = lev.P.T @ r
    ec = vcycle(levels, j - 1, rc, np.zeros_like(rc), prob)
    x = x + lev.P @ ec
    return smooth(lev, f, x, prob.nu_post, prob)


def multigrid(levels, j, f, x0, m, prob):
    x = x0
    for _ in range(m):
        x = vcycle(levels, j, f, x, prob)
    return x


# --------------------------------------------------------------------------------------
# Small nonlinear eigenproblems by SCF (Algorithm 3.1 step 2, Algorithm 3.2 step 1)
# --------------------------------------------------------------------------------------
@dataclass
class ScfResult:
    lam: float
    c: np.ndarray
    iters: int
    residual: float
    converged: bool


def scf(k0: np.ndarray, mm: np.ndarray, gfun, zeta: float, c0: np.ndarray, sign_fn,
        tol: float, max_iter: int, history: int = 6, beta: float = 0.5) -> ScfResult:
    """Lowest solution of (K0 + zeta G(c)) c = lambda M c, c^T M c = 1.

    Self-consistent field iteration: each step solves the linear eigenproblem
    (K0 + zeta X) c = mu M c for the lowest eigenpair (aufbau) and forms the density matrix
    G(c).  The input matrix X is updated by Anderson (Pulay) mixing of the residuals
    F = G(c(X)) - X over the last `history` steps with damping beta (plain damped SCF for the
    first step); the fixed point X = G(c) is the SCF solution.  lambda is reported as
    c^T (K0 + zeta G(c)) c, the nonlinear Rayleigh quotient, and the iteration stops when the
    relative residual of the nonlinear equation is below tol."""
    x = gfun(c0)
    xs, fs = [], []
    c, lam, res = c0, np.nan, np.inf
    for it in range(1, max_iter + 1):
        _, vecs = sla.eigh(k0 + zeta * x, mm)
        c = vecs[:, 0] / np.sqrt(vecs[:, 0] @ mm @ vecs[:, 0])
        if sign_fn(c) < 0:
            c = -c
        g_new = gfun(c)
        h = k0 + zeta * g_new
        lam = float(c @ h @ c)
        r = h @ c - lam * (mm @ c)
        res = float(np.linalg.norm(r) / (abs(lam) * np.linalg.norm(mm @ c)))
        if res <= tol:
            return ScfResult(lam, c, it, res, True)
        f = (g_new - x).ravel()
        xs.append(x.ravel().copy())
        fs.append(f)
        xs, fs = xs[-(history + 1):], fs[-(history + 1):]
        step = beta * f
        if len(fs) > 1:
            d_f = np.stack([fs[i + 1] - fs[i] for i in range(len(fs) - 1)], axis=1)
            d_x = np.stack([xs[i + 1] - xs[i] for i in range(len(xs) - 1)], axis=1)
            gamma = np.linalg.lstsq(d_f, f, rcond=None)[0]
            step = step - (d_x + beta * d_f) @ gamma
        x = x + step.reshape(x.shape)
        x = 0.5 * (x + x.T)
    return ScfResult(lam, c, max_iter, res, False)


def coarse_solve(prob: Problem, lev: Level) -> tuple[float, np.ndarray, ScfResult]:
    """Algorithm 3.2 step 1: the nonlinear eigenproblem directly on V_{h_1}.

    SCF starts from the lowest eigenvector of the linear problem zeta = 0."""
    k0 = (lev.A + lev.Wm).toarray()
    mm = lev.M.toarray()
    _, vecs = sla.eigh(k0, mm)
    c0 = vecs[:, 0] if vecs[:, 0].sum() > 0 else -vecs[:, 0]
    res = scf(k0, mm, lambda c: density_matrix(lev.mesh, c).toarray(), prob.zeta, c0,
              lambda c: c.sum(), prob.scf_tol, prob.scf_max_iter)
    return res.lam, res.c, res


def prolong_to(levels: list[Level], k: int) -> sp.csr_matrix:
    """P_{k <- 1} = P_k P_{k-1} ... P_2: coefficient vectors of the V_{h_1} basis on level k."""
    p = sp.identity(levels[0].mesh.n_interior, format="csr")
    for j in range(2, k + 1):
        p = (levels[j - 1].P @ p).tocsr()
    return p


@dataclass
class CorrectionInfo:
    lam: float
    u: np.ndarray
    u_tilde: np.ndarray
    scf: ScfResult


def aux_rhs(prob: Problem, lev: Level, lam: float, u: np.ndarray) -> np.ndarray:
    """Right-hand side of the auxiliary problem: lambda M u - f(x, u) tested on V_{h_k}.

    W_LEFT keeps W in the operator, so only the cubic term is moved right."""
    f = lam * (lev.M @ u) - nonlinear_load(lev.mesh, u, prob.zeta)
    if prob.operator_form == PAPER_LITERAL:
        f = f - lev.Wm @ u
    return f


def augmented_blocks(levels, k, u_tilde):
    """Basis psi = (phi^H_1..phi^H_N, u~) of V_{H,h_k} as fine coefficient vectors, and the
    matrices K0 = [a^(psi_i, psi_j) + (W psi_i, psi_j)] and M = [b(psi_i, psi_j)]."""
    lev = levels[k - 1]
    psi = sp.hstack([prolong_to(levels, k), sp.csr_matrix(u_tilde[:, None])]).tocsr()
    kfull = (lev.A + lev.Wm).tocsr()
    k0 = (psi.T @ kfull @ psi).toarray()
    mm = (psi.T @ lev.M @ psi).toarray()
    return psi, 0.5 * (k0 + k0.T), 0.5 * (mm + mm.T)


def eigen_mg(prob: Problem, levels: list[Level], k: int, lam: float, u: np.ndarray) -> CorrectionInfo:
    """One correction step EigenMG(V_H, lambda, u, V_{h_k}, m) (Algorithm 3.1)."""
    lev = levels[k - 1]
    f = aux_rhs(prob, lev, lam, u)
    u_tilde = multigrid(levels, k, f, u, prob.vcycles, prob)          # step 1
    psi, k0, mm = augmented_blocks(levels, k, u_tilde)                 # step 2
    n = psi.shape[1]
    c0 = np.zeros(n)
    c0[-1] = 1.0 / np.sqrt(u_tilde @ (lev.M @ u_tilde))

    def gfun(c):
        w = psi @ c
        return (psi.T @ density_matrix(lev.mesh, w) @ psi).toarray()

    res = scf(k0, mm, gfun, prob.zeta, c0, lambda c: c[-1], prob.scf_tol, prob.scf_max_iter)
    return CorrectionInfo(res.lam, psi @ res.c, u_tilde, res)


@dataclass
class FmgResult:
    lam: float
    u: np.ndarray
    lam_levels: list
    scf_iters: list
    converged: bool
    corrections: list


def fmg_solve(prob: Problem, levels: list[Level] | None = None) -> FmgResult:
    """Algorithm 3.2: direct nonlinear solve on V_{h_1}, then for k = 2..n prolong the
    previous level's pair and apply p correction steps."""
    levels = levels or build_hierarchy(prob)
    lam, u, r1 = coarse_solve(prob, levels[0])
    lams, iters, conv, corr = [lam], [r1.iters], r1.converged, []
    for k in range(2, prob.levels + 1):
        u = levels[k - 1].P @ u
        for _ in range(prob.corrections):
            info = eigen_mg(prob, levels, k, lam, u)
            lam, u = info.lam, info.u
            iters.append(info.scf.iters)
            conv = conv and info.scf.converged
            corr.append(info)
        lams.append(lam)
    return FmgResult(lam, u, lams, iters, conv, corr)


# --------------------------------------------------------------------------------------
# Reference quantities used by the pins
# --------------------------------------------------------------------------------------
def gp_energy_parts(prob: Problem, lev: Level, u: np.ndarray):
    """(a^(u,u) + (W u, u), int u^4, b(u,u)) on one level."""
    k = lev.A + lev.Wm
    return float(u @ (k @ u)), quartic(lev.mesh, u), float(u @ (lev.M @ u))


def discrete_ground_state(prob: Problem, lev: Level, tol: float = 1e-11) -> tuple[float, np.ndarray, ScfResult]:
    """The discrete problem of Section 2 on one level, solved directly by dense SCF (tiny
    meshes only).  Dense eigensolves of a few hundred unknowns floor the relative residual
    near 1e-12, hence the looser default tolerance."""
    k0 = (lev.A + lev.Wm).toarray()
    mm = lev.M.toarray()
    _, vecs = sla.eigh(k0, mm)
    c0 = vecs[:, 0] if vecs[:, 0].sum() > 0 else -vecs[:, 0]
    res = scf(k0, mm, lambda c: density_matrix(lev.mesh, c).toarray(), prob.zeta, c0,
              lambda c: c.sum(), tol, prob.scf_max_iter)
    return res.lam, res.c, res
