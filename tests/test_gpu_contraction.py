"""Per-correction contraction of Algorithm 3.1 (Theorem 3.1) on the GPU, for both operator
forms and several coarse spaces V_H on a fixed fine level.

gamma = ||u^(l+1) - u_h||_2 / ||u^(l) - u_h||_2, u_h the discrete ground state of the
fine level (from many corrections).  Theorem 3.1 bounds the error after a correction by
C (theta^m + eta_a(V_H)) times the error before it, so gamma must be below 1 and shrink as H
does.  Run with -s to print the table."""
import numpy as np
import pytest

from tests.test_gpu_parity import _fmg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FINE_N = 128


def _gamma(form: int, coarse: int, vcycles: int = 1, steps: int = 3):
    fmg = _fmg()
    levels = int(np.log2(FINE_N // coarse)) + 1
    base = dict(dim=2, coarse_cells=coarse, levels=levels, w_quad=(1.0, 2.0, 0.0), zeta=10.0,
                vcycles=vcycles, operator_form=form, scf_max_iter=100)
    n = (FINE_N - 1) ** 2
    with fmg.Solver(fmg.Problem(**base, corrections=40)) as s:  # the discrete ground state
        ref = np.empty(n)
        lam_ref, _, rc = s.solve(ref)
    assert rc == 0
    with fmg.Solver(fmg.Problem(**base, corrections=1)) as s:
        u = np.empty(n)
        lam, _, rc = s.solve(u)
        assert rc == 0
        errs = [np.linalg.norm(u - ref)]
        ud = torch.from_numpy(u).cuda()
        uo = torch.empty_like(ud)
        for _ in range(steps):
            lam, _, rc = s.correction(levels, lam, ud, uo)
            assert rc == 0
            ud, uo = uo, ud
            errs.append(float(torch.linalg.norm(ud - torch.from_numpy(ref).cuda())))
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1) if errs[i] > 1e-11]
    return ratios, errs


@pytest.mark.parametrize("form", [0, 1], ids=["W_LEFT", "PAPER_LITERAL"])
def test_contraction_below_one_and_shrinks_with_H(form):
    table = {}
    for coarse in (2, 4, 8):
        ratios, errs = _gamma(form, coarse)
        assert ratios and all(r < 1.0 for r in ratios), (coarse, ratios)
        table[coarse] = ratios[0]
        print(f"form={form} H=1/{coarse}: gamma = {', '.join(f'{r:.3e}' for r in ratios)}"
              f"  (errors {', '.join(f'{e:.2e}' for e in errs)})")
    assert table[8] < table[2]
