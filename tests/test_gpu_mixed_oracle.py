"""Mixed precision against the FP64 oracle at the sizes where the single-precision path runs.

The mixed modes run FP32 V-cycles (through the TMA-fed sweeps) inside the FP64 defect
correction only on FMG stages whose level has at least 512 (2D) or 128 (3D) cells per side;
smaller stages keep the FP64 V-cycles.  So these cases are the smallest that exercise it:

* 2D, config 2 truncated to 7 levels (h = 1/512, 261,121 dofs) and a ragged case with 640
  cells per side (639 interior nodes per row: four full 128-column tiles and a 127-column
  tail), against live oracle runs;
* 3D, config 3 truncated to 6 levels (h = 1/128, 2,048,383 dofs), against the oracle's stored
  result (``tests/golden/oracle_config3_6levels.txt``, written by
  ``tests/golden/make_oracle_3d_golden.py``, which calls only the oracle): its eigenvalue per
  level, u at every 8th interior node per direction, and the norm of u.

Bounds.  FP64 mode: the solver's own bounds (lambda 1e-11 relative, u 1e-9 in relative L2).
Mixed modes: |d lambda| <= 1e-8 relative, the benchmark's acceptance bound, and u within
1e-8 relative (L2 and element-wise max).  The latter is derived from the arithmetic: each
of the m = 2 V-cycles of the finest stage adds a single-precision rounding of about 2^-24
(6e-8) of its correction, and the correction of the finest stage is about 1e-3 of u (the
prolonged iterate is already within the discretisation error of the coarser level), so the
change of u~ is about 1e-10 of u; the augmented solve then fixes u to the ground state on
V_H + span{u~}, which moves with u~ at first order, and the bound leaves two orders of
magnitude for the amplification by the small problems' conditioning.  The BF16-storage
ablation (8-bit mantissas) is held only to the accuracy class it reaches (1e-4)."""
import numpy as np
import pytest

from oracle import fmg_oracle as O
from tests.test_gpu_parity import _fmg
from workloads import seeded_problem

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

LAM64, U64 = 1e-11, 1e-9
LAM_MIXED, U_MIXED = 1e-8, 1e-8
LAM_BF16, U_BF16 = 1e-4, 1e-2

GOLDEN_3D = "tests/golden/oracle_config3_6levels.txt"


def _gpu(kw, precision=0, flags=0):
    fmg = _fmg()
    p = fmg.Problem(**{k: v for k, v in kw.items() if k in fmg.Problem.__dataclass_fields__},
                    precision=precision, flags=flags)
    with fmg.Solver(p) as s:
        u = np.empty(p.size(p.levels))
        lam, st, rc = s.solve(u, stats=True)
    assert rc == 0
    return lam, u, st


def _errors(lam, u, lam_ref, u_ref):
    return (abs(lam - lam_ref) / lam_ref, np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref),
            np.abs(u - u_ref).max() / np.abs(u_ref).max())


CASES_2D = {
    "config2-h512": seeded_problem("config2", levels=7),
    "ragged-h640": dict(seeded_problem("config2", levels=8, coarse_cells=5),
                        w_quad=(1.0, 2.25, 0.0), zeta=60.0),
}


@pytest.fixture(scope="module", params=sorted(CASES_2D))
def oracle_2d(request):
    kw = CASES_2D[request.param]
    r = O.fmg_solve(O.Problem(**kw))
    assert r.converged
    return request.param, kw, r


MODES = [("fp64", 0, 0, LAM64, U64), ("fp32", 1, 0, LAM_MIXED, U_MIXED),
         ("fp32-rhs32", 1, 2, LAM_MIXED, None), ("bf16", 2, 0, LAM_BF16, U_BF16)]


@pytest.mark.parametrize("mode", MODES, ids=[m[0] for m in MODES])
def test_mixed_2d_against_oracle(oracle_2d, mode):
    name, kw, ref = oracle_2d
    key, prec, flags, lam_tol, u_tol = mode
    lam, u, st = _gpu(kw, prec, flags)
    dl, du, dmax = _errors(lam, u, ref.lam, ref.u)
    print(f"{name} {key}: dlambda {dl:.2e}  du_l2 {du:.2e}  du_max {dmax:.2e}")
    assert dl <= lam_tol
    if u_tol is not None:  # the FP32 right-hand side moves u~ by ~1e-7 of f: lambda only
        assert du <= u_tol and dmax <= 10 * u_tol
    else:
        assert du <= 1e-6
    assert abs(st.identity_defect) <= 1e-10 * lam


@pytest.fixture(scope="module")
def golden_3d():
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), GOLDEN_3D)
    d, samples = {}, []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 1:
                samples.append(float(parts[0]))
            elif parts[0] == "lambda_levels":
                d["lambda_levels"] = [float(v) for v in parts[1:]]
            else:
                d[parts[0]] = float(parts[1])
    assert len(samples) == int(d["u_samples"])
    n, step = int(d["cells"]), int(d["step"])
    g = np.arange(step, n, step) - 1
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    d["idx"] = (i + (n - 1) * (j + (n - 1) * k)).ravel()
    d["u"] = np.array(samples)
    return d


MODES_3D = [("fp64", 0, LAM64, U64), ("fp32", 1, LAM_MIXED, U_MIXED), ("bf16", 2, 1e-3, 1e-1)]


@pytest.mark.parametrize("mode", MODES_3D, ids=[m[0] for m in MODES_3D])
def test_mixed_3d_against_stored_oracle(golden_3d, mode):
    key, prec, lam_tol, u_tol = mode
    kw = seeded_problem("config3", levels=6)
    lam, u, st = _gpu(kw, prec)
    ref = golden_3d["lambda_levels"]
    lam_levels = list(st.lambda_levels)[:6]
    dl = abs(lam - ref[-1]) / ref[-1]
    us = u[golden_3d["idx"]]
    du = np.linalg.norm(us - golden_3d["u"]) / np.linalg.norm(golden_3d["u"])
    dmax = np.abs(us - golden_3d["u"]).max() / np.abs(golden_3d["u"]).max()
    dn = abs(np.linalg.norm(u) - golden_3d["u_norm2"]) / golden_3d["u_norm2"]
    ds = abs(u.sum() - golden_3d["u_sum"]) / abs(golden_3d["u_sum"])
    print(f"3d {key}: dlambda {dl:.2e}  du_l2(sampled) {du:.2e}  du_max {dmax:.2e}  "
          f"dnorm {dn:.2e}  dsum {ds:.2e}")
    assert dl <= lam_tol
    assert du <= u_tol and dmax <= 10 * u_tol
    assert dn <= u_tol and ds <= u_tol
    if prec == 0:  # FP64: every level's eigenvalue is the oracle's
        for a, b in zip(lam_levels, ref):
            assert abs(a - b) <= LAM64 * b
