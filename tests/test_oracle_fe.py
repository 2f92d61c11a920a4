"""Pins for the oracle's finite-element layer (Section 2 forms, Section 3 nested spaces).

Each check compares the oracle with something it does not compute itself: closed-form
stencils and spectra, an independent collapsed-Gauss quadrature, point evaluation of hat
functions, or an identity the nested spaces force (Galerkin coarse operators)."""
from pathlib import Path

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fmg_oracle as O
from tests.quadrature import p1_eval, simplex_points


def _full_matrix(mesh, kind, **kw):
    """Global matrix over ALL nodes, to look at rows whose support misses the boundary."""
    vol, g = mesh.geometry()
    e = mesh.elems
    k = e.shape[1]
    if kind == "A":
        local = vol[:, None, None] * np.einsum("eai,ebi->eab", g, g)
    else:
        local = vol[:, None, None] * O.bary_tensor(2, mesh.dim)[None]
    rows = np.repeat(e, k, axis=1).ravel()
    cols = np.tile(e, (1, k)).ravel()
    return sp.coo_matrix((local.ravel(), (rows, cols)), shape=(mesh.n_nodes,) * 2).tocsr()


def test_bary_monomial_rule_against_quadrature():
    """int_K lambda^alpha on a skewed triangle and tetrahedron vs collapsed Gauss."""
    rng = np.random.default_rng(7)
    for d in (2, 3):
        verts = rng.normal(size=(d + 1, d))
        vol = abs(np.linalg.det(verts[1:] - verts[0])) / (2 if d == 2 else 6)
        x, w = simplex_points(verts, d)
        lam = np.stack([p1_eval(verts, np.eye(d + 1)[a], x) for a in range(d + 1)])
        for alpha in [(4, 0, 0, 0), (1, 1, 1, 1), (2, 1, 1, 0), (2, 2, 0, 0), (3, 1, 0, 0), (0, 0, 2, 0)]:
            alpha = alpha[: d + 1]
            ref = np.sum(w * np.prod([lam[a] ** alpha[a] for a in range(d + 1)], axis=0))
            assert abs(O.bary_monomial_integral(alpha, vol, d) - ref) <= 1e-13 * max(1, abs(ref))


def test_stiffness_2d_is_five_point_stencil():
    """Right angles sit opposite the (1,1) diagonals, so P1 stiffness is the 5-point Laplacian."""
    n = 6
    mesh = O.Mesh(2, n, 1.0)
    a = O.stiffness(mesh).toarray()
    m = n - 1
    t = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    ref = np.kron(np.eye(m), t) + np.kron(t, np.eye(m))
    assert np.abs(a - ref).max() < 1e-13


def test_stiffness_2d_spectrum_closed_form():
    n = 8
    a = O.stiffness(O.Mesh(2, n, 1.0)).toarray()
    p = np.arange(1, n)
    ref = np.sort((4 - 2 * np.cos(np.pi * p[:, None] / n) - 2 * np.cos(np.pi * p[None, :] / n)).ravel())
    assert np.abs(np.linalg.eigvalsh(a) - ref).max() < 1e-12


def test_stiffness_3d_kuhn_is_seven_point_times_h():
    n = 4
    mesh = O.Mesh(3, n, 2.0)
    a = O.stiffness(mesh).toarray()
    m = n - 1
    t = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    i = np.eye(m)
    ref = np.kron(np.kron(i, i), t) + np.kron(np.kron(i, t), i) + np.kron(np.kron(t, i), i)
    assert np.abs(a - mesh.h * ref).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_rows_and_total(dim):
    """Sum_j M_ij = int phi_i = h^d for a node whose hat misses the boundary; 1^T M 1 over all
    nodes is |Omega|."""
    n = 4
    mesh = O.Mesh(dim, n, 1.5)
    mfull = _full_matrix(mesh, "M")
    assert abs(mfull.sum() - 1.5 ** dim) < 1e-13
    centre = int(np.flatnonzero(np.all(mesh.ijk == n // 2, axis=1))[0])
    row = mfull.getrow(centre)
    assert abs(row.sum() - mesh.h ** dim) < 1e-14
    if dim == 2:
        vals = np.sort(row.data / mesh.h ** 2)
        assert np.allclose(vals, [1 / 12] * 6 + [1 / 2], atol=1e-14)
    else:
        assert row.nnz == 15


def _quadrature_matrix(mesh, fn, u=None, kind="W"):
    """Independent element loop with collapsed Gauss: W: int fn(x) phi_a phi_b;
    N: int u^3 phi_a; G: int u^2 phi_a phi_b."""
    d = mesh.dim
    nn = mesh.n_nodes
    out = np.zeros((nn, nn)) if kind != "N" else np.zeros(nn)
    ufull = None if u is None else mesh.to_full(u)
    eye = np.eye(d + 1)
    for el in mesh.elems:
        verts = mesh.coords[el]
        x, w = simplex_points(verts, d)
        phi = np.stack([p1_eval(verts, eye[a], x) for a in range(d + 1)])
        if kind == "W":
            wt = w * fn(x)
        else:
            uh = p1_eval(verts, ufull[el], x)
            wt = w * (uh ** 3 if kind == "N" else uh ** 2)
        if kind == "N":
            out[el] += phi @ wt
        else:
            out[np.ix_(el, el)] += (phi * wt) @ phi.T
    idx = mesh.interior
    return out[idx] if kind == "N" else out[np.ix_(idx, idx)]


@pytest.mark.parametrize("dim", [2, 3])
def test_potential_mass_against_quadrature(dim):
    mesh = O.Mesh(dim, 3 if dim == 3 else 4, 1.3)
    wq = (1.0, 2.5, 4.0)[:dim]
    wm = O.potential_mass(mesh, 0.7, tuple(wq) + (0.0,) * (3 - dim)).toarray()
    ref = _quadrature_matrix(mesh, lambda x: 0.7 + (wq * x ** 2).sum(1))
    assert np.abs(wm - ref).max() < 1e-14 * max(1, np.abs(ref).max())


def test_potential_constant_is_mass():
    mesh = O.Mesh(2, 5, 1.0)
    wm = O.potential_mass(mesh, 3.0, (0.0, 0.0, 0.0))
    assert abs(wm - 3.0 * O.mass(mesh)).max() < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_terms_against_quadrature(dim):
    rng = np.random.default_rng(11)
    mesh = O.Mesh(dim, 3 if dim == 3 else 4, 1.0)
    u = rng.normal(size=mesh.n_interior)
    n_ref = _quadrature_matrix(mesh, None, u, kind="N")
    assert np.abs(O.nonlinear_load(mesh, u, 2.0) - 2.0 * n_ref).max() < 1e-13
    g_ref = _quadrature_matrix(mesh, None, u, kind="G")
    assert np.abs(O.density_matrix(mesh, u).toarray() - g_ref).max() < 1e-13
    # int u^4 = u^T B(u) u
    assert abs(O.quartic(mesh, u) - u @ g_ref @ u) < 1e-12


def test_degree4_six_point_rule_equals_exact_integration():
    """A symmetric 6-point rule of degree 4 (two orbits (a,b,b)), with its points and weights
    solved from its own moment equations, integrates u^3 phi exactly, i.e. it agrees with the
    oracle's monomial rule."""
    from scipy.optimize import fsolve

    def orbit(a):
        b = (1 - a) / 2
        return np.array([[a, b, b], [b, a, b], [b, b, a]])

    mons = [(2, 0, 0), (4, 0, 0), (2, 2, 0), (2, 1, 1)]

    def eqs(p):
        a1, a2, w1 = p[:3]
        w2 = 0.5 - w1
        out = []
        for al in mons[:3]:
            q = sum(wt * np.prod(orbit(a) ** np.array(al), axis=1).sum() for a, wt in ((a1, w1 / 3), (a2, w2 / 3)))
            out.append(q - O.bary_monomial_integral(al, 0.5, 2) / 0.5 * 0.5)
        return out

    a1, a2, w1 = fsolve(eqs, [0.1, 0.45, 0.1], xtol=1e-14)
    w2 = 0.5 - w1
    pts = np.vstack([orbit(a1), orbit(a2)])
    wts = np.concatenate([np.full(3, w1 / 3), np.full(3, w2 / 3)])
    rng = np.random.default_rng(3)
    uv = rng.normal(size=3)
    for a in range(3):
        uq = pts @ uv
        quad = 2 * np.sum(wts * uq ** 3 * pts[:, a])          # |K| = 1 (reference area 1/2, x2)
        exact = 0.0
        for idx in np.ndindex(3, 3, 3):
            al = [list(idx).count(v) + (v == a) for v in range(3)]
            exact += uv[idx[0]] * uv[idx[1]] * uv[idx[2]] * O.bary_monomial_integral(al, 1.0, 2)
        assert abs(quad - exact) < 1e-13


@pytest.mark.parametrize("dim,nc", [(2, 4), (3, 2)])
def test_prolongation_is_hat_evaluation(dim, nc):
    """Column c of P holds phi^coarse_c at the fine nodes: 1 at the coincident node, 1/2 at
    fine nodes on coarse edges through c, 0 elsewhere; rows sum to <= 1."""
    coarse, fine = O.Mesh(dim, nc, 1.0), O.Mesh(dim, 2 * nc, 1.0)
    p = O.prolongation(coarse, fine).toarray()
    assert set(np.unique(p)) <= {0.0, 0.5, 1.0}
    fi = fine.ijk[fine.interior]
    ci = coarse.ijk[coarse.interior]
    for c in range(len(ci)):
        col = p[:, c]
        on = np.all(fi == 2 * ci[c], axis=1)
        assert col[on][0] == 1.0 and col.sum() == 1.0 + 0.5 * (np.count_nonzero(col) - 1)
        assert np.count_nonzero(col) == (7 if dim == 2 else 15)


@pytest.mark.parametrize("dim,nc,levels", [(2, 4, 3), (3, 2, 3)])
def test_galerkin_identity(dim, nc, levels):
    """Nested spaces with exact integration: P^T L_k P = L_{k-1} and P^T M_k P = M_{k-1}."""
    prob = O.Problem(dim=dim, coarse_cells=nc, levels=levels, w_const=0.3, w_quad=(1.0, 2.0, 3.0))
    lv = O.build_hierarchy(prob)
    for j in range(2, levels + 1):
        p = lv[j - 1].P
        assert abs(p.T @ lv[j - 1].L @ p - lv[j - 2].L).max() < 1e-12
        assert abs(p.T @ lv[j - 1].M @ p - lv[j - 2].M).max() < 1e-15


def test_vector_layout_is_lexicographic_x_fastest():
    mesh = O.Mesh(2, 4, 1.0)
    ij = mesh.ijk[mesh.interior]
    assert ij[0].tolist() == [1, 1] and ij[1].tolist() == [2, 1] and ij[3].tolist() == [1, 2]


def _golden_elements():
    path = Path(__file__).parent / "golden" / "paper_tables_elements.txt"
    rows = []
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            table, level, printed, read = line.split()
            rows.append((table, int(level), int(printed), int(read)))
    return rows


def test_kuhn_hierarchy_matches_paper_tables():
    """Tables 1-2 print the element counts of the 3D hierarchy: the oracle's Kuhn meshes of an
    8-cell initial mesh (Table 1) and of its first refinement (Table 2) reproduce them.  The
    mesh is built only for the two smallest levels; larger ones follow from the 8x rule that
    regular refinement gives (checked on the built ones)."""
    rows = _golden_elements()
    built = {n: len(O.Mesh(3, n, 1.0).elems) for n in (8, 16)}
    assert built[16] == 8 * built[8]
    for table, level, printed, read in rows:
        first = 8 if table == "table1" else 16
        n = first << (level - 1)
        assert 6 * n ** 3 == read
        if n in built:
            assert built[n] == read
        assert printed == read or sorted(str(printed)) == sorted(str(read))
