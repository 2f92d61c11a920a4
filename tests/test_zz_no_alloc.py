"""The allocation-free coarsest-level solve, checked against the handle-based one.

fmg_eig_coarse_solve_noalloc exists for callers that may not allocate device memory (for
example a framework that owns all GPU memory through its own pool, or a service that must
not allocate while it serves, since an allocation can synchronise the device).  It keeps its
intermediates in one fixed device array inside the library that every call reuses, so these
tests make calls in a row with different problems (each smaller than the one before, so stale
contents of an earlier call would show) and compare each with fmg_eig_coarse_solve on a
handle, within the tolerances of the other parity tests.  The sizes span the accepted range:
the largest (9 coarse cells per side, where the array's layout and the dense solve's shared
memory are largest) down to the smallest (2 cells, one unknown).  The file sorts last so a
stop-at-first-failure run has already run every other test before this one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM_TOL = 1e-11
U_TOL = 1e-9


def _problems(fmg):
    return [
        fmg.Problem(coarse_cells=9, levels=2, w_const=0.25, w_quad=(3.0, 1.0, 0.0), zeta=60.0),
        fmg.Problem(coarse_cells=8, levels=3, w_const=0.5, w_quad=(1.0, 3.0, 0.0), zeta=25.0),
        fmg.Problem(coarse_cells=5, levels=2, w_quad=(2.0, 1.0, 0.0), zeta=3.0, box_len=1.5),
        fmg.Problem(coarse_cells=2, levels=2, w_quad=(1.0, 1.0, 0.0), zeta=7.0),
    ]


def _check_against_handle(fmg, prob, stream=None):
    m = (prob.coarse_cells - 1) ** 2
    u_new = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    lam_new, _, rc_new = fmg.coarse_solve_noalloc(prob, u_new, stream)
    with fmg.Solver(prob) as s:
        u_ref = torch.empty(m, dtype=torch.float64, device="cuda")
        lam_ref, _, rc_ref = s.coarse_solve(u_ref)
    torch.cuda.synchronize()
    assert rc_new == 0 and rc_ref == 0
    assert abs(lam_new - lam_ref) <= LAM_TOL * abs(lam_ref)
    a, b = u_new.cpu().numpy(), u_ref.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= U_TOL * np.linalg.norm(b)


def test_noalloc_coarse_solve_matches_handle_on_calls_in_a_row():
    from paper_1502_04657_gb300 import fmg

    for prob in _problems(fmg):
        _check_against_handle(fmg, prob)


def test_noalloc_coarse_solve_on_a_side_stream():
    """The call runs on the stream it is given and synchronises it before returning."""
    from paper_1502_04657_gb300 import fmg

    side = torch.cuda.Stream()
    for prob in _problems(fmg)[:2]:
        _check_against_handle(fmg, prob, side.cuda_stream)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    from paper_1502_04657_gb300 import fmg

    for cells in (10, 11):
        u = torch.empty((cells - 1) ** 2, dtype=torch.float64, device="cuda")
        with pytest.raises(fmg.FmgError) as e:
            fmg.coarse_solve_noalloc(fmg.Problem(coarse_cells=cells, levels=1), u)
        assert e.value.code == fmg.FMG_EINVAL
