"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle runs.

Only parameter generation lives here (no arithmetic of the method), so both the CUDA path and
the oracle can take the same instances.  The shapes follow the paper's workload (Example 4.1:
harmonic trap W, repulsive cubic term, unit box, P1 meshes refined by beta = 2) at the sizes
of the benchmark configurations:

  config1  2D, coarsest h = 1/8, 6 levels (h = 1/256, 65,025 dofs), W = x^2 + y^2, zeta = 1
  config2  2D, coarsest h = 1/8, 10 levels (h = 1/4096, 16,769,025 dofs), W = x^2 + y^2,
           zeta = 10
  config3  3D Kuhn, coarsest h = 1/4, 7 levels (h = 1/256, 16,581,375 dofs),
           W = 100 (x^2 + y^2 + 4 z^2), zeta = 100
  batch    256 2D instances, finest n uniform on {64, ..., 1024}, W = x^2 + g^2 y^2 with
           g ~ U[1, 4], zeta ~ U[0, 200]
  serve    Poisson arrivals (rate 200/s) of 70% 2D (n 64..2048) / 30% 3D (n 16..128)
           requests with zeta ~ U[0, 200] and an anisotropic trap g ~ U[1, 4]

Every parameter set uses 2 V-cycles per level (m), one correction per level (p), 2 + 2
damped-Jacobi sweeps with omega = 2/3."""
from __future__ import annotations

import numpy as np

SEED = 150204657
METHOD = dict(nu_pre=2, nu_post=2, omega=2.0 / 3.0, vcycles=2, corrections=1)

CONFIGS = {
    "config1": dict(dim=2, coarse_cells=8, levels=6, w_const=0.0, w_quad=(1.0, 1.0, 0.0), zeta=1.0),
    "config2": dict(dim=2, coarse_cells=8, levels=10, w_const=0.0, w_quad=(1.0, 1.0, 0.0), zeta=10.0),
    "config3": dict(dim=3, coarse_cells=4, levels=7, w_const=0.0, w_quad=(100.0, 100.0, 400.0), zeta=100.0),
}


def seeded_problem(name: str, **over) -> dict:
    """Keyword arguments of a problem (oracle Problem / library Problem field names)."""
    kw = {**CONFIGS[name], **METHOD, "box_len": 1.0}
    kw.update(over)
    return kw


def batch_instances(count: int = 256, seed: int = SEED, levels_choices=(4, 5, 6, 7, 8)) -> list[dict]:
    """The 256-instance 2D batch: n_1 = 8 and finest n in {64..1024} (4..8 levels)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        g = rng.uniform(1.0, 4.0)
        out.append({**METHOD, "dim": 2, "coarse_cells": 8, "box_len": 1.0,
                    "levels": int(rng.choice(levels_choices)), "w_const": 0.0,
                    "w_quad": (1.0, g * g, 0.0), "zeta": float(rng.uniform(0.0, 200.0))})
    return out


def serve_stream(count: int = 10000, rate: float = 200.0, seed: int = SEED + 1) -> list[dict]:
    """Poisson request stream: arrival time plus problem keywords."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = []
    for i in range(count):
        g = rng.uniform(1.0, 4.0)
        zeta = float(rng.uniform(0.0, 200.0))
        if rng.uniform() < 0.7:
            kw = {"dim": 2, "coarse_cells": 8, "levels": int(rng.integers(4, 10)),
                  "w_quad": (1.0, g * g, 0.0)}
        else:
            kw = {"dim": 3, "coarse_cells": 4, "levels": int(rng.integers(3, 7)),
                  "w_quad": (1.0, 1.0, g * g)}
        reqs.append({**METHOD, **kw, "box_len": 1.0, "w_const": 0.0, "zeta": zeta,
                     "arrival_s": float(t[i])})
    return reqs
