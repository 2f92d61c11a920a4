"""The allocation-free coarsest-level solve, checked against the handle-based one.

fmg_eig_coarse_solve_noalloc exists for callers that may not allocate device memory (for
example code that runs while a stream capture forbids allocation, or a framework that owns
all GPU memory through its own pool).  It keeps its intermediates in one fixed device array
inside the library that every call reuses, so this test makes two calls in a row with
different problems (the second smaller than the first, so stale contents of the first would
show) and compares each with fmg_eig_coarse_solve on a handle, within the tolerances of the
other parity tests.  The file sorts last so a stop-at-first-failure run has already run
every other test before this one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM_TOL = 1e-11
U_TOL = 1e-9


def _problems(fmg):
    return [
        fmg.Problem(coarse_cells=8, levels=3, w_const=0.5, w_quad=(1.0, 3.0, 0.0), zeta=25.0),
        fmg.Problem(coarse_cells=5, levels=2, w_quad=(2.0, 1.0, 0.0), zeta=3.0, box_len=1.5),
    ]


def test_noalloc_coarse_solve_matches_handle_on_two_calls_in_a_row():
    from paper_1502_04657_gb300 import fmg

    for prob in _problems(fmg):
        m = (prob.coarse_cells - 1) ** 2
        u_new = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        lam_new, it_new, rc_new = fmg.coarse_solve_noalloc(prob, u_new)
        with fmg.Solver(prob) as s:
            u_ref = torch.empty(m, dtype=torch.float64, device="cuda")
            lam_ref, _, rc_ref = s.coarse_solve(u_ref)
        torch.cuda.synchronize()
        assert rc_new == 0 and rc_ref == 0
        assert abs(lam_new - lam_ref) <= LAM_TOL * abs(lam_ref)
        a, b = u_new.cpu().numpy(), u_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= U_TOL * np.linalg.norm(b)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    from paper_1502_04657_gb300 import fmg

    u = torch.empty(121, dtype=torch.float64, device="cuda")
    with pytest.raises(fmg.FmgError) as e:
        fmg.coarse_solve_noalloc(fmg.Problem(coarse_cells=11, levels=1), u)
    assert e.value.code == fmg.FMG_EINVAL
