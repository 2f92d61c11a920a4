"""Write the oracle's full multigrid result for the 3D trap at h = 1/128 to a text fixture.

The 3D problem (Kuhn P1 mesh on the unit cube, coarsest h = 1/4, 6 levels = 127^3 = 2,048,383
interior dofs, W = 100 (x^2 + y^2 + 4 z^2), zeta = 100, m = 2, p = 1, 2 + 2 damped Jacobi)
is the smallest 3D size whose finest FMG stage runs single-precision V-cycles in the mixed
modes, and far too large for the plain oracle to solve inside a test (minutes and several GB).
This script calls only the oracle (Algorithm 3.2 as written in ``oracle/fmg_oracle.py``) and
stores what the GPU tests compare against:

* lambda_{h_k} after every level k (the last is the final eigenvalue);
* u at every 8th interior node per direction (i, j, k in 8, 16, ..., 120), x fastest;
* the sum and the Euclidean norm of the whole interior vector u.

Run from the repository root:  python tests/golden/make_oracle_3d_golden.py
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fmg_oracle as O  # noqa: E402
from workloads import seeded_problem  # noqa: E402

OUT = os.path.join(HERE, "oracle_config3_6levels.txt")
LEVELS = 6
STEP = 8


def sample_indices(n: int, step: int = STEP) -> np.ndarray:
    """Positions in the interior vector (x fastest) of the nodes whose grid indices are all
    multiples of `step` (grid index i = 1..n-1 is interior position i - 1)."""
    m = n - 1
    g = np.arange(step, n, step) - 1
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    return (i + m * (j + m * k)).ravel()


def main() -> None:
    kw = seeded_problem("config3", levels=LEVELS)
    prob = O.Problem(**kw)
    t = time.time()
    r = O.fmg_solve(prob)
    dt = time.time() - t
    n = prob.cells(LEVELS)
    idx = sample_indices(n)
    with open(OUT, "w") as f:
        f.write("# oracle fmg_solve (Algorithm 3.2), written by tests/golden/make_oracle_3d_golden.py\n")
        f.write(f"# problem {sorted(kw.items())}\n")
        f.write(f"# oracle time {dt:.0f} s, converged {r.converged}, scf iterations {r.scf_iters}\n")
        f.write(f"cells {n}\n")
        f.write(f"step {STEP}\n")
        f.write("lambda_levels " + " ".join(repr(float(x)) for x in r.lam_levels) + "\n")
        f.write(f"u_sum {float(np.sum(r.u))!r}\n")
        f.write(f"u_norm2 {float(np.linalg.norm(r.u))!r}\n")
        f.write(f"u_samples {len(idx)}\n")
        for v in r.u[idx]:
            f.write(f"{float(v)!r}\n")
    print(f"wrote {OUT} in {dt:.0f} s: lambda = {r.lam!r}")


if __name__ == "__main__":
    main()
