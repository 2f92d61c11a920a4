"""Batches (fmg_eig_batch_create / fmg_eig_batch_solve / fmg_eig_solve_batch): every instance of
a batch must give the result of its own single-instance solve.

Batching only changes which instances a launch covers: every node, reduction and dense solve
of an instance is computed by the same expressions in the same order, so the eigenvalues and
eigenvectors are compared bit for bit with the single-instance handles, and a sample against
the FP64 oracle with the eigenpair tolerances."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import LAM_TOL, U_TOL, _fmg
from workloads import METHOD, batch_instances

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems(kws, **over):
    fmg = _fmg()
    return [fmg.Problem(**{**{k: v for k, v in kw.items() if k != "arrival_s"}, **over,
                           "scf_max_iter": 100}) for kw in kws]


def _mixed_2d(count=9, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        g = rng.uniform(1.0, 4.0)
        out.append({**METHOD, "dim": 2, "coarse_cells": 4, "box_len": 1.0,
                    "levels": int(rng.integers(1, 6)), "w_const": float(rng.uniform(0, 1)),
                    "w_quad": (1.0, g * g, 0.0), "zeta": float(rng.uniform(0.0, 200.0))})
    out[0]["levels"] = 5  # at least one of the deepest size
    return out


def _single(p, with_u=True):
    fmg = _fmg()
    with fmg.Solver(p) as s:
        u = np.empty(p.size(p.levels)) if with_u else None
        lam, st, rc = s.solve(u, stats=True)
    return lam, u, st, rc


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_2d_equals_single_solves(precision):
    fmg = _fmg()
    probs = _problems(_mixed_2d(), precision=precision)
    with fmg.BatchSolver(probs) as b:
        assert b.count() == len(probs)
        lams, us, sts, codes = b.solve_all(with_u=True, stats=True)
    for i, p in enumerate(probs):
        lam1, u1, st1, rc1 = _single(p)
        assert codes[i] == rc1 == 0
        assert lams[i] == lam1, (i, lams[i], lam1)
        assert np.array_equal(us[i], u1), i
        assert sts[i].levels == p.levels
        assert list(sts[i].scf_iters)[:p.levels] == list(st1.scf_iters)[:p.levels]
        assert abs(sts[i].identity_defect) < 1e-10 * lams[i]
        assert abs(sts[i].norm_defect) < 1e-12


def test_batch_2d_against_oracle():
    fmg = _fmg()
    kws = _mixed_2d(count=5, seed=5)
    for kw in kws:
        kw["levels"] = min(kw["levels"], 4)
    probs = _problems(kws)
    with fmg.BatchSolver(probs) as b:
        lams, us, _, codes = b.solve_all()
    for i, kw in enumerate(kws):
        ref = O.fmg_solve(O.Problem(**kw))
        assert ref.converged and codes[i] == 0
        assert abs(lams[i] - ref.lam) <= LAM_TOL * ref.lam
        assert np.linalg.norm(us[i] - ref.u) <= U_TOL * np.linalg.norm(ref.u)


def test_batch_3d_equals_single_solves():
    fmg = _fmg()
    rng = np.random.default_rng(3)
    kws = []
    for lv in (3, 2, 3, 1, 2):
        g = rng.uniform(1.0, 4.0)
        kws.append({**METHOD, "dim": 3, "coarse_cells": 4, "box_len": 1.0, "levels": lv,
                    "w_const": 0.0, "w_quad": (1.0, 1.0, g * g),
                    "zeta": float(rng.uniform(0.0, 200.0))})
    probs = _problems(kws)
    with fmg.BatchSolver(probs) as b:
        lams, us, _, codes = b.solve_all()
    for i, p in enumerate(probs):
        lam1, u1, _, rc1 = _single(p)
        assert codes[i] == rc1 == 0
        assert lams[i] == lam1
        assert np.array_equal(us[i], u1)


def test_mixed_batch_meets_dlambda_against_fp64_singles():
    """The benchmark batch's acceptance: mixed-precision batch vs FP64 single solves,
    |delta lambda| <= 1e-8 relative (instances of the benchmark distribution, smaller sizes)."""
    kws = batch_instances(count=12, levels_choices=(3, 4, 5))
    mixed = _problems(kws, precision=1)
    fp64 = _problems(kws, precision=0)
    fmg = _fmg()
    with fmg.BatchSolver(mixed) as b:
        lams, _, _, codes = b.solve_all(with_u=False)
    for i, p in enumerate(fp64):
        lam1, _, _, rc1 = _single(p, with_u=False)
        assert codes[i] == rc1 == 0
        assert abs(lams[i] - lam1) <= 1e-8 * lam1


def test_one_shot_solve_batch_groups_settings():
    """fmg_eig_solve_batch splits 2D/3D and FP64/mixed into groups and keeps the order."""
    fmg = _fmg()
    kws = _mixed_2d(count=4, seed=21)
    probs = _problems(kws)
    probs[1].precision = 1
    p3 = fmg.Problem(dim=3, coarse_cells=2, levels=3, w_quad=(1.0, 1.0, 2.0), zeta=5.0)
    probs.insert(2, p3)
    lams, us, _, codes = fmg.solve_batch(probs)
    for i, p in enumerate(probs):
        lam1, u1, _, rc1 = _single(p)
        assert codes[i] == rc1 == 0
        assert lams[i] == lam1
        assert np.array_equal(us[i], u1)


def test_autotuned_tiles_do_not_change_results():
    fmg = _fmg()
    kws = _mixed_2d(count=6, seed=8)
    tuned = _problems(kws)
    fixed = _problems(kws, flags=fmg.FMG_FLAG_NO_AUTOTUNE)
    with fmg.BatchSolver(tuned) as b:
        tiles = [b.level_tile(k) for k in range(1, 6)]
        lt, ut, _, _ = b.solve_all()
    with fmg.BatchSolver(fixed) as b:
        assert all(b.level_tile(k) == (32, 8) for k in range(1, 6))
        lf, uf, _, _ = b.solve_all()
    for bx, by in tiles:
        assert bx * by <= 1024 and bx >= 1 and by >= 1
    assert lt == lf
    assert all(np.array_equal(a, c) for a, c in zip(ut, uf))


def test_batch_rejects_incompatible_settings():
    fmg = _fmg()
    probs = _problems(_mixed_2d(count=3))
    probs[1].vcycles = 3
    with pytest.raises(fmg.FmgError) as e:
        fmg.BatchSolver(probs)
    assert e.value.code == fmg.FMG_EINVAL
