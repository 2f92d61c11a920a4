"""The FP64 cubic-load, right-hand-side and density kernels walk columns (2D) and planes
(3D) in tiles: 30 produced columns x 64 rows per 2D block, 32 x 8 columns x 16 planes per
3D block.  These cases put several tiles and a ragged tail in every direction (2D n = 80:
79 = 30 + 30 + 19 columns, 64 + 15 rows; 3D n = 48: 47 = 32 + 15 columns, 5 x 8 + 7 rows,
16 + 16 + 15 planes) and compare each kernel with the oracle, once with the walks forced
(FMG_FLAG_STAR_WALKS) and once with the default choice, which runs launches this small node
by node."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import _fmg, _pair, dev, host, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "2d_n80": (dict(dim=2, coarse_cells=5, levels=5, w_const=0.3, w_quad=(1.0, 2.0, 0.0),
                    zeta=6.0), 5),
    "3d_n48": (dict(dim=3, coarse_cells=3, levels=5, w_const=0.3, w_quad=(1.0, 2.0, 1.5),
                    zeta=6.0), 5),
}


@pytest.fixture(scope="module", params=[(c, w) for c in sorted(CASES) for w in ("walk", "node")],
                ids=lambda p: f"{p[0]}-{p[1]}")
def case(request):
    name, mode = request.param
    kw, k = CASES[name]
    op, gp = _pair(**kw)
    if mode == "walk":
        gp.flags = _fmg().FMG_FLAG_STAR_WALKS
    lv = O.build_hierarchy(op)
    with _fmg().Solver(gp) as s:
        yield op, gp, lv, s, k


def test_cubic_load_and_rhs_span_tiles(case):
    op, gp, lv, s, k = case
    rng = np.random.default_rng(1300 + k)
    u = rng.normal(size=gp.size(k))
    out = torch.empty(gp.size(k), dtype=torch.float64, device="cuda")
    s.nonlinear_load(k, dev(u), out)
    assert rel(host(out), O.nonlinear_load(lv[k - 1].mesh, u, 1.0)) <= 1e-13
    s.aux_rhs(k, 17.0, dev(u), out)
    assert rel(host(out), O.aux_rhs(op, lv[k - 1], 17.0, u)) <= 1e-13


def test_density_stencil_spans_tiles(case):
    """The density stencil of the walk, through its Galerkin coarsening to the augmented
    space (G) and the restricted cubic load (T1 inside G)."""
    op, gp, lv, s, k = case
    rng = np.random.default_rng(1400 + k)
    ut = rng.uniform(0.2, 1.0, size=gp.size(k))
    psi, k0, mm = O.augmented_blocks(lv, k, ut)
    c = rng.normal(size=psi.shape[1])
    g_ref = (psi.T @ O.density_matrix(lv[k - 1].mesh, psi @ c) @ psi).toarray()
    K, M, G = s.augmented_system(k, dev(ut), c)
    assert rel(K, k0) <= 1e-12
    assert rel(M, mm) <= 1e-12
    assert rel(G, g_ref) <= 1e-12


_SOLVED = {}


def test_fp64_solve_spans_tiles(case):
    op, gp, lv, s, k = case
    key = (op.dim, op.coarse_cells, op.levels)
    if key not in _SOLVED:  # one oracle solve per case, shared by both modes
        _SOLVED[key] = O.fmg_solve(op)
    ref = _SOLVED[key]
    u = np.empty(gp.size(gp.levels))
    lam, stats, rc = s.solve(u, stats=True)
    assert rc == 0
    assert abs(lam - ref.lam) / abs(ref.lam) <= 1e-11
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-9


def test_mixed_double_float_walks_match_node_by_node_and_oracle():
    """In the mixed modes the 3D cubic load, density stencil and right-hand side run in
    double-float arithmetic, as plane walks where the FP64 ones walk (forced here on every
    level) and node by node otherwise.  At this size every FMG stage keeps FP64 V-cycles, so
    both must give the FP64 oracle's eigenpair to double-float rounding, and agree closely
    with each other."""
    fmg = _fmg()
    kw, _ = CASES["3d_n48"]
    op, gp = _pair(**kw)
    key = (op.dim, op.coarse_cells, op.levels)
    if key not in _SOLVED:
        _SOLVED[key] = O.fmg_solve(op)
    ref = _SOLVED[key]
    out = {}
    for mode, flags in (("walk", fmg.FMG_FLAG_STAR_WALKS), ("node", 0)):
        gp.precision = fmg.FMG_MIXED_FP32
        gp.flags = flags
        with fmg.Solver(gp) as s:
            u = np.empty(gp.size(gp.levels))
            lam, _, rc = s.solve(u)
        assert rc == 0
        assert abs(lam - ref.lam) / ref.lam <= 1e-10
        assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-8
        out[mode] = (lam, u)
    (lw, uw), (ln, un) = out["walk"], out["node"]
    assert abs(lw - ln) / ln <= 1e-12
    assert np.linalg.norm(uw - un) / np.linalg.norm(un) <= 1e-10
