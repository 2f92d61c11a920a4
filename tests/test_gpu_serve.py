"""fmg_eig_serve: continuous batching of a request stream.  Every request's result must be
its solve alone (bit for bit: a cohort only changes which launches an instance shares), the
requests must actually share cohorts and overlap on the GPU, and admission must respect the
device-memory budget."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg
from workloads import METHOD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stream(count=30, rate=3000.0, seed=7):
    """Small mixed 2D/3D stream with the serving workload's parameter distribution."""
    fmg = _fmg()
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    probs = []
    for _ in range(count):
        g = rng.uniform(1.0, 4.0)
        zeta = float(rng.uniform(0.0, 200.0))
        if rng.uniform() < 0.7:
            kw = dict(dim=2, coarse_cells=8, levels=int(rng.integers(2, 6)), w_quad=(1.0, g * g, 0.0))
        else:
            kw = dict(dim=3, coarse_cells=4, levels=int(rng.integers(1, 4)), w_quad=(1.0, 1.0, g * g))
        probs.append(fmg.Problem(**{**METHOD, **kw, "zeta": zeta, "scf_max_iter": 100}))
    return probs, list(t)


def _alone(p):
    fmg = _fmg()
    with fmg.Solver(p) as s:
        u = np.empty(p.size(p.levels))
        lam, _, rc = s.solve(u)
    return lam, u, rc


def test_served_results_equal_solves_alone():
    fmg = _fmg()
    probs, arrivals = _stream()
    res, st = fmg.serve(probs, arrivals, max_batch=8, max_inflight=3, batch_window_s=0.002,
                        with_u=True)
    assert st["completed"] == len(probs)
    for p, r in zip(probs, res):
        lam, u, rc = _alone(p)
        assert r["status"] == rc == 0
        assert r["lambda"] == lam
        assert np.array_equal(r["u"], u)
        assert r["latency_s"] > 0 and r["done_s"] >= r["admit_s"]
    # requests shared cohorts, and cohorts were resident together
    assert st["max_cohort"] > 1
    assert st["cohorts"] < len(probs)
    assert st["max_inflight_seen"] >= 2
    lat = sorted(r["latency_s"] for r in res)
    assert st["p50_s"] == lat[(len(lat) + 1) // 2 - 1]
    assert st["p99_s"] == lat[-1] or st["p99_s"] <= lat[-1]


def test_admission_respects_memory_budget():
    fmg = _fmg()
    probs, arrivals = _stream(count=16, rate=1e5, seed=9)
    # a budget just above the largest request: cohorts must wait for memory to be released
    res0, st0 = fmg.serve(probs, arrivals, max_batch=16, max_inflight=8)
    largest = max(fmg.estimate_bytes([p]) for p in probs)
    assert fmg.estimate_bytes(probs) <= sum(fmg.estimate_bytes([p]) for p in probs)
    budget = 1.05 * (largest + 65536)
    assert st0["peak_bytes"] > budget  # unconstrained, more than that was resident
    res, st = fmg.serve(probs, arrivals, budget_bytes=budget, max_batch=16, max_inflight=8)
    assert st["peak_bytes"] <= budget
    assert st["completed"] == len(probs)
    for r0, r in zip(res0, res):
        assert r["lambda"] == r0["lambda"]


def test_pooled_hierarchies_are_replayed():
    """Cohorts with the level counts of an earlier cohort replay its pooled hierarchy (and
    graph) with their own parameters: results still equal the solves alone."""
    fmg = _fmg()
    rng = np.random.default_rng(17)
    probs = []
    for i in range(12):
        g = rng.uniform(1.0, 4.0)
        probs.append(fmg.Problem(dim=2, coarse_cells=8, levels=3 + (i % 2), w_quad=(1.0, g * g, 0.0),
                                 zeta=float(rng.uniform(0, 200)), scf_max_iter=100))
    arrivals = [0.004 * i for i in range(12)]  # one at a time: single-instance cohorts
    res, st = fmg.serve(probs, arrivals, max_batch=1, max_inflight=2)
    assert st["cohorts"] == 12 and st["reused"] >= 8
    for p, r in zip(probs, res):
        lam, _, rc = _alone(p)
        assert r["status"] == rc == 0 and r["lambda"] == lam


def test_request_larger_than_budget_is_rejected():
    fmg = _fmg()
    probs, arrivals = _stream(count=3)
    with pytest.raises(fmg.FmgError) as e:
        fmg.serve(probs, arrivals, budget_bytes=1024.0)
    assert e.value.code == fmg.FMG_EINVAL
