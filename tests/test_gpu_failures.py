"""The ABI's failure codes, produced without any GPU fault or hang.

* FMG_ETIMEOUT: the TMA-fed sweeps bound every mbarrier wait.  FMG_FLAG_EXPIRE_WAITS makes
  those waits give up at once; the sweep then records its instance in the solve's status word,
  waits (with the normal bound) for its own loads in flight and returns, and the solve reports
  FMG_ETIMEOUT for exactly the instances whose levels use the TMA path.
* FMG_ENOCONV: a cap of one nonlinear iteration per small solve; the partial result is still
  written and the per-instance statuses say which instances hit the cap.
* FMG_ENOMEM: fmg_eig_inject_alloc_failure makes one device allocation of the library fail as
  if the device were full.  Creation then fails cleanly at every allocation point (nothing
  stays allocated), and the server reports the cohort that could not be admitted while it
  serves the other requests.
After each case a normal solve in the same process still works (the context stays usable)."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg
from workloads import METHOD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(p, with_u=True):
    fmg = _fmg()
    with fmg.Solver(p) as s:
        u = np.empty(p.size(p.levels)) if with_u else None
        lam, st, rc = s.solve(u, stats=True)
    return lam, u, st, rc


# ---- FMG_ETIMEOUT ------------------------------------------------------------------------
@pytest.mark.parametrize("kw", [dict(dim=2, coarse_cells=4, levels=8, w_quad=(1.0, 2.0, 0.0), zeta=20.0),
                                dict(dim=3, coarse_cells=2, levels=7, w_quad=(1.0, 1.0, 4.0), zeta=30.0)],
                         ids=["2d-n512", "3d-n128"])
def test_expired_waits_report_etimeout_and_the_context_stays_usable(kw):
    fmg = _fmg()
    p = fmg.Problem(**{**METHOD, **kw}, precision=fmg.FMG_MIXED_FP32,
                    flags=fmg.FMG_FLAG_EXPIRE_WAITS)
    with fmg.Solver(p) as s:
        with pytest.raises(fmg.FmgError) as e:
            s.solve(np.empty(p.size(p.levels)), stats=True)
    assert e.value.code == fmg.FMG_ETIMEOUT
    # the same problem without the hook: a normal, converged solve
    q = fmg.Problem(**{**METHOD, **kw}, precision=fmg.FMG_MIXED_FP32)
    lam, u, st, rc = _solve(q)
    assert rc == 0 and np.isfinite(lam) and np.all(np.isfinite(u))
    lam64, _, _, _ = _solve(fmg.Problem(**{**METHOD, **kw}), with_u=False)
    assert abs(lam - lam64) <= 1e-8 * lam64


def test_expired_waits_mark_only_the_instances_on_tma_levels():
    """In a batch, the sweeps of a level run only for the instances that have it: the one with
    a 512-cell level times out, the one whose finest level has 64 cells does not, and its
    result equals its solve alone."""
    fmg = _fmg()
    big = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 7, "w_quad": (1.0, 3.0, 0.0),
                         "zeta": 40.0}, precision=fmg.FMG_MIXED_FP32, flags=fmg.FMG_FLAG_EXPIRE_WAITS)
    small = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 4, "w_quad": (1.0, 2.0, 0.0),
                           "zeta": 15.0}, precision=fmg.FMG_MIXED_FP32, flags=fmg.FMG_FLAG_EXPIRE_WAITS)
    with fmg.BatchSolver([big, small]) as b:
        lams, us, _, codes = b.solve_all(allow=(fmg.FMG_ETIMEOUT,))
    assert codes == [fmg.FMG_ETIMEOUT, fmg.FMG_OK]
    lam_s, u_s, _, rc = _solve(small)
    assert rc == 0
    assert lams[1] == lam_s and np.array_equal(us[1], u_s)


def test_expired_waits_in_serving_mark_the_request():
    fmg = _fmg()
    base = dict(METHOD, dim=2, coarse_cells=8, w_quad=(1.0, 1.0, 0.0), zeta=10.0, scf_max_iter=100)
    probs = [fmg.Problem(**{**base, "levels": 7}, precision=fmg.FMG_MIXED_FP32,
                         flags=fmg.FMG_FLAG_EXPIRE_WAITS),
             fmg.Problem(**{**base, "levels": 4}, precision=fmg.FMG_MIXED_FP32)]
    res, st = fmg.serve(probs, [0.0, 0.0], max_batch=1, max_inflight=2,
                        allow=(fmg.FMG_ETIMEOUT,))
    assert res[0]["status"] == fmg.FMG_ETIMEOUT
    assert res[1]["status"] == fmg.FMG_OK
    lam, _, _, _ = _solve(probs[1], with_u=False)
    assert res[1]["lambda"] == lam


# ---- FMG_ENOCONV -------------------------------------------------------------------------
def test_iteration_cap_reports_enoconv_with_the_partial_result_written():
    fmg = _fmg()
    p = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 4, "w_quad": (1.0, 1.0, 0.0),
                       "zeta": 50.0}, scf_max_iter=1)
    lam, u, st, rc = _solve(p)
    assert rc == fmg.FMG_ENOCONV and st.status == fmg.FMG_ENOCONV
    assert list(st.scf_iters[: p.levels]) == [1] * p.levels
    assert np.isfinite(lam) and lam > 0 and np.all(np.isfinite(u)) and np.any(u != 0)
    q = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 4, "w_quad": (1.0, 1.0, 0.0),
                       "zeta": 50.0}, scf_max_iter=100)
    lam_c, _, st_c, rc_c = _solve(q)
    assert rc_c == 0 and st_c.status == 0
    assert abs(lam - lam_c) < 0.5 * lam_c  # one iteration per level: rough, but an eigenvalue


def test_iteration_cap_statuses_per_instance_in_a_batch():
    """fmg_eig_solve_batch groups the problems by their shared settings (the cap is one), so a
    capped group and a normal group run together; statuses come back in the caller's order."""
    fmg = _fmg()
    rng = np.random.default_rng(3)
    probs = []
    for i in range(6):
        probs.append(fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 3 + i % 3,
                                    "w_quad": (1.0, float(rng.uniform(1, 4)), 0.0),
                                    "zeta": float(rng.uniform(0, 100))},
                                 scf_max_iter=1 if i % 2 == 0 else 100))
    lams, us, stats, codes = fmg.solve_batch(probs, stats=True)
    assert codes == [fmg.FMG_ENOCONV if i % 2 == 0 else fmg.FMG_OK for i in range(6)]
    for i, p in enumerate(probs):
        assert stats[i].status == codes[i]
        assert np.isfinite(lams[i]) and np.all(np.isfinite(us[i]))
        if codes[i] == 0:
            lam, u, _, _ = _solve(p)
            assert lams[i] == lam and np.array_equal(us[i], u)


# ---- FMG_ENOMEM --------------------------------------------------------------------------
def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _fail_creates(fmg, p, points):
    """Inject an allocation failure at each point in turn and create a handle for p; returns
    (creations that failed with FMG_ENOMEM, the first point past the handle's allocations)."""
    failed = 0
    try:
        for after in points:
            fmg.inject_alloc_failure(after)
            try:
                s = fmg.Solver(p)
            except fmg.FmgError as e:
                assert e.code == fmg.FMG_ENOMEM
                failed += 1
                continue
            s.close()  # every allocation succeeded: the injection point is past the end
            return failed, after
    finally:
        fmg.inject_alloc_failure(-1)
    raise AssertionError("creation never got past the injection points")


def test_allocation_failure_at_every_point_of_create_reports_enomem():
    fmg = _fmg()
    for prec in (fmg.FMG_FP64, fmg.FMG_MIXED_FP32):
        p = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 4, "w_quad": (1.0, 1.0, 0.0),
                           "zeta": 5.0}, precision=prec)
        lam0, _, _, _ = _solve(p, with_u=False)
        failed, end = _fail_creates(fmg, p, range(0, 1000))
        assert failed == end and failed >= 20  # one failure per allocation of the handle
        lam1, _, _, rc = _solve(p, with_u=False)
        assert rc == 0 and lam1 == lam0


def test_failed_creates_leave_nothing_allocated():
    """A 1M-dof mixed-precision hierarchy (several hundred MB) whose creation fails at every
    third allocation point: were the buffers allocated before the failure kept, the device
    would lose hundreds of MB per failed creation."""
    fmg = _fmg()
    p = fmg.Problem(**{**METHOD, "dim": 2, "coarse_cells": 8, "levels": 8, "w_quad": (1.0, 4.0, 0.0),
                       "zeta": 30.0}, precision=fmg.FMG_MIXED_FP32)
    _solve(p, with_u=False)  # tiles tuned and cached, lazily loaded modules in place
    free0 = _free_bytes()
    failed, _ = _fail_creates(fmg, p, range(0, 3000, 3))
    assert failed >= 10
    assert _free_bytes() >= free0 - (256 << 20)


def test_allocation_failure_while_serving_fails_one_cohort_and_serves_the_rest():
    fmg = _fmg()
    base = dict(METHOD, dim=2, coarse_cells=8, w_quad=(1.0, 1.0, 0.0), scf_max_iter=100)
    probs = [fmg.Problem(**{**base, "levels": 3 + i % 2, "zeta": 5.0 + i}) for i in range(6)]
    arrivals = [0.0] + [0.05 + 0.002 * i for i in range(5)]
    fmg.inject_alloc_failure(0)  # the first cohort's first allocation fails
    try:
        res, st = fmg.serve(probs, arrivals, max_batch=1, max_inflight=1,
                            allow=(fmg.FMG_ENOMEM,))
    finally:
        fmg.inject_alloc_failure(-1)
    assert res[0]["status"] == fmg.FMG_ENOMEM
    assert st["completed"] == len(probs) - 1
    for p, r in list(zip(probs, res))[1:]:
        lam, _, _, rc = _solve(p, with_u=False)
        assert r["status"] == rc == 0 and r["lambda"] == lam
