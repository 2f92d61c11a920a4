#!/usr/bin/env python3
"""Benchmark of the full multigrid GP ground-state solver (one JSON line on rank 0).

Default workload (N = 1): the 16.8M-dof 2D configuration - unit square, P1 mesh with (1,1)
diagonals, coarsest h = 1/8 refined 9 times to h = 1/4096 (16,769,025 interior dofs),
W = x^2 + y^2, zeta = 10, 2 V-cycles of 2 + 2 damped Jacobi (omega = 2/3) per level, one
correction per level, FP64 throughout.  A step is one complete solve (Algorithm 3.2,
including the per-solve operator setup and the upload of the problem parameters); inputs are
resident and the per-solve working set (>2 GB) is far larger than the 129 MB L2, so no flush
is needed between steps.  --workload selects another configuration (config1, config3, or a
"-mixed" variant with FP32 V-cycles inside the FP64 defect correction).

--impl ours (default): the CUDA library.  value = solves/s over the timed steps (CUDA events
on the launch stream), max over ranks; e2e = the same metric through fmg_eig_solve with a
pinned host output buffer (parameter upload and the D2H copy of lambda and u inside).
--impl reference: the FP64 CPU oracle on this host's cores (rank 0 only), each step a bounded
sample of the workload, scaled to the full size by the method's linear work (Theorem 3.3).
Multi-GPU: replicas only (instances are independent; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import batch_instances, seeded_problem, serve_stream  # noqa: E402

METRIC = "GP ground-state solves/s and fine-grid MDOF/s at |Δλ|≤1e-8; p50/p99 latency"
WORKLOADS = {
    "config2": ("config2", False,
                "2D unit square, P1 right-triangle mesh, coarsest h=1/8 refined to h=1/4096 "
                "(10 levels, 16,769,025 dofs), W=x^2+y^2, zeta=10, m=2 V-cycles, p=1, 2+2 damped "
                "Jacobi omega=2/3, FP64 plain per-instance solve"),
    "config2-mixed": ("config2", True,
                      "config2 with FP32 V-cycles inside the FP64 defect correction"),
    "config1": ("config1", False,
                "2D unit square, h=1/8 refined to h=1/256 (6 levels, 65,025 dofs), W=x^2+y^2, "
                "zeta=1, m=2, p=1, 2+2 Jacobi, FP64"),
    "config3": ("config3", False,
                "3D unit cube, Kuhn 6-tet mesh, h=1/4 refined to h=1/256 (7 levels, 16,581,375 "
                "dofs), W=100(x^2+y^2+4z^2), zeta=100, m=2, p=1, 2+2 Jacobi, FP64"),
    "config3-mixed": ("config3", True,
                      "config3 with FP32 V-cycles inside the FP64 defect correction"),
    "config2-bf16": ("config2", "bf16",
                     "config2 with bfloat16-stored (FP32-computed) V-cycles inside the FP64 "
                     "defect correction (storage ablation)"),
    "config3-bf16": ("config3", "bf16",
                     "config3 with bfloat16-stored (FP32-computed) V-cycles inside the FP64 "
                     "defect correction (storage ablation)"),
    "config4": ("config4", True,
                "batch of 256 seeded 2D instances, coarsest h=1/8, finest h uniform on "
                "{1/64..1/1024}, W=x^2+g^2 y^2 with g~U[1,4], zeta~U[0,200], FP32 V-cycles in "
                "FP64 defect correction, one launch per step and level for the batch, one CUDA "
                "graph, autotuned tiles; vs 256 sequential FP64 single solves"),
    "paper-examples": ("paper-examples", False,
                       "the paper's Examples 4.1 / 4.2 (Section 4): [0,1]^3, Kuhn P1 meshes, "
                       "W = x1^2 + x2^2 + x3^2, zeta = 1 and 100, finest h = 1/8 .. 1/128 (the "
                       "element counts of Tables 1-2); coarse space h = 1/4 (the paper's is its "
                       "h = 1/8 initial mesh, solved with ARPACK); m = 1, p = 1; 3 + 3 "
                       "conjugate-gradient smoothing steps as in the paper (3 + 3 Chebyshev "
                       "timed beside); FP64"),
    "config5": ("config5", True,
                "serving: seeded Poisson stream, 200 req/s, 10,000 requests, 70% 2D (h 1/64..1/2048, "
                "coarsest 1/8) / 30% 3D (h 1/16..1/128, coarsest 1/4), zeta~U[0,200], anisotropic "
                "trap g~U[1,4]; FP32 V-cycles in FP64 defect correction; continuous batching with "
                "free-HBM admission, resident hierarchies, per-level batched launches"),
}
FP64_FLOP_PER_CLK_SM = 4      # 2 DFMA per clock per SM (1.25 TFLOP/s nominal at 2070 MHz)
N_SM = 152
# Algorithmic FP64 flops and bytes per node of the finest-level launch:
#   Jacobi 2D: the defect f - L x as 7 multiply-adds + the update x + (omega/D) r = 16 flop;
#     24 B (x, f, x') + 40 B (4 couplings + omega/D)
#   cubic load + density stencil 2D (closed forms over the 6 star triangles from per-edge
#     numbers: 3 own edges x 5 + square 1 + 3 six-term sums 15 + cubic bracket 8 + diagonal 6
#     + 3 off-diagonal entries x 8): 69 flop; 8 B read + 40 B written
#   Jacobi 3D: 15 multiply-adds + update = 32 flop; 24 B + 72 B
#   cubic load + density stencil 3D (symmetric sums of the 6 tetrahedra of a cube formed once,
#     the power sums of the base vertices and the first middle vertex shared by two tetrahedra:
#     90 flop with u^2, 2 u^3; star and edge sums 73; N, diagonal and 7 edge entries 86):
#     249 flop; 8 B + 72 B
# The third number counts FP64 instructions (DADD, DMUL and DFMA alike take one issue slot of
# the FP64 pipe, 2 per SM per clock): the unit these kernels are bound by.  The Jacobi update
# forms f - L x as one chain of fused multiply-adds from f, then x + (omega/D) r: 8 in 2D,
# 16 in 3D.
KERNELS = {
    2: {"nload_density": (69.0, 48.0, 55.0), "jacobi": (16.0, 64.0, 8.0)},
    3: {"nload_density": (249.0, 80.0, 198.0), "jacobi": (32.0, 96.0, 16.0)},
}
# Launches too small to fill the GPU as walks run node by node, each node forming the sums of
# its own star: 2D 106 flop in 82 FP64 instructions (pair sums n_k + n_{k+1}), 3D 659 flop in
# about 490 (sums over the link of the 24-tetrahedron star).
NODE_KERNELS = {2: {"nload_density": (106.0, 48.0, 82.0)}, 3: {"nload_density": (659.0, 80.0, 490.0)}}


def star_walks(dim: int, n: int, nb: int) -> bool:
    """Whether the library runs a level of n cells per side (nb instances) as a column / plane
    walk: when the walk's grid has at least two blocks per SM (30 x 64-node 2D blocks,
    32 x 8 x 16-node 3D blocks)."""
    m = n - 1
    if dim == 2:
        blocks = -(-m // 30) * -(-m // 64)
    else:
        blocks = -(-m // 32) * -(-m // 8) * -(-m // 16)
    return blocks * nb >= 2 * N_SM
# the kernel with the largest share of the solve in the ncu launch lists (2D FP64 solve:
# k_jacobi2d 21 %; 3D FP64 solve: k_nload_density3d 35 %)
DOMINANT = {2: "jacobi", 3: "nload_density"}
# The single-precision V-cycle (mixed modes) is HBM-bound: a Jacobi sweep or residual reads x
# and f and writes one vector, 3 x 4 bytes per node (3 x 2 with BF16 storage); the
# coefficients are rebuilt from per-axis tables that stay in L1.
MIXED_HBM_KERNELS = ("jacobi", "residual")
# The mixed modes evaluate the cubic load + density stencil in double-float arithmetic on the
# FP32 pipes: the kernel is bound by instruction issue (4 warp instructions per SM per clock).
# Thread instructions per node (smsp__inst_executed.sum x 32 / nodes) and DRAM bytes per node
# from one ncu capture of each kernel: 2D the finest launch of the 10-level mixed solve
# (node by node, 16,769,025 nodes); 3D the plane walk at h = 1/128 (2,048,383 nodes; the walk
# runs every 3D level with n >= 128, so its per-node figures hold at h = 1/256).
ISSUE_PER_CLK_SM = 4 * 32
DF_INSTR_PER_NODE = {2: 618510721 * 32 / 16769025, 3: 200397029 * 32 / 2048383}
DF_TRAFFIC_PER_NODE = {2: (136027392 + 609443328) / 16769025,
                       3: (24750336 + 83417856) / 2048383}


def hbm_peak() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"
# DRAM bytes per node of a finest-level launch from one ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of the level-9 launch of the 9-level 2D
# solve, 4,190,209 nodes), scaled by the nodes a launch processes.
TRAFFIC_PER_NODE = {(2, "nload_density"): (34.109952e6 + 106.015232e6) / 4190209,
                    # the first level-9 sweep of the 9-level 2D solve, 4,190,209 nodes
                    (2, "jacobi"): (235144960 + 24157184) / 4190209,
                    # 3D: the level-6 launch of the 6-level solve, 2,048,383 nodes
                    (3, "nload_density"): (22.779648e6 + 83.184128e6) / 2048383}


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# Multi-GPU is replicas only: instances are independent, so each rank solves its own share
# and the only collectives are the barrier around the timed region and the max over ranks of
# its duration (no collective on the data path).
def shard(items, rank: int, world: int):
    """Rank r's share of independent instances: every world-th one, starting at r."""
    return items[rank::world]


def max_over_ranks(dist, value: float, device) -> float:
    """The slowest rank's time (the whole job's time); value itself with one rank."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3] not in ("[N/A]", "")]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def problem_kwargs(config: str, levels=None) -> dict:
    kw = seeded_problem(config)
    if levels is not None:
        kw["levels"] = levels
    return kw


ORACLE_SNIPPET = r"""
import hashlib, json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import fmg_oracle as O
from workloads import seeded_problem
kw = seeded_problem({cfg!r}, levels={levels})
times = []
for _ in range({reps}):
    t = time.perf_counter()
    prob = O.Problem(**kw)
    r = O.fmg_solve(prob)
    times.append(time.perf_counter() - t)
if {u_path!r}:
    np.save({u_path!r}, r.u)
print(json.dumps({{"times": times, "lam": r.lam, "dofs": (prob.cells(prob.levels) - 1) ** prob.dim,
                  "digest": hashlib.sha256(np.float64(r.lam).tobytes() + r.u.tobytes()).hexdigest()}}))
"""
ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def run_oracle(config: str, levels: int, reps: int, u_path: str = "") -> dict:
    """The oracle in a fresh single-threaded interpreter (exec'd, never forked from CUDA);
    u_path: where to save its final u (numpy .npy), if given."""
    env = {**os.environ, **ONE_THREAD}
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=config, levels=levels, reps=reps, u_path=u_path)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_all_cores(config: str, levels: int, procs: int | None = None) -> dict:
    """`procs` (default: every host core) single-threaded oracle interpreters, each solving the
    same sample at once: the oracle's throughput on all cores, in solves of the sample per
    second of wall time.  Independent solves need no communication, and each one's result is
    the single-threaded result bit for bit (checked by digest)."""
    procs = procs or os.cpu_count() or 1
    env = {**os.environ, **ONE_THREAD}
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=config, levels=levels, reps=1, u_path="")
    t = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    outs = [json.loads(p.communicate()[0].strip().splitlines()[-1]) for p in ps]
    wall = time.perf_counter() - t
    if any(p.returncode != 0 for p in ps):
        raise RuntimeError("an oracle process failed")
    return {"procs": procs, "wall_s": wall, "per_sample_s": wall / procs,
            "digests": sorted({o["digest"] for o in outs}), "dofs": outs[0]["dofs"]}


def dofs_of(kw: dict) -> int:
    return ((kw["coarse_cells"] << (kw["levels"] - 1)) - 1) ** kw["dim"]


# oracle samples sized for ~10-30 s (cpu_baseline) and a few s per step (reference arm)
ORACLE_SAMPLE = {"config1": (6, 5), "config2": (7, 6), "config3": (4, 3)}


def reference_arm(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    config, mixed, desc = WORKLOADS[args.workload]
    if config == "paper-examples":
        print(json.dumps({"impl": "reference", "unavailable": "context workload (the paper's "
                          "examples beside its Tables 1-2); the oracle is timed on configs 1-5"}),
              flush=True)
        return
    if config in ("config4", "config5"):
        vals = []
        for i in range(args.warmup + args.steps):
            r = (batch_cpu_baseline(count=2, cap=6) if config == "config4"
                 else serve_cpu_baseline(count=2))
            if i >= args.warmup:
                vals.append(r["value"])
        value = statistics.mean(vals)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "parallelism": "replicas"},
            "cpu_baseline": {**r, "value": value},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    levels = ORACLE_SAMPLE[config][1]
    walls, r = [], None
    for i in range(args.warmup + args.steps):
        r = run_oracle_all_cores(config, levels)
        if i >= args.warmup:
            walls.append(r["wall_s"])
    full = dofs_of(problem_kwargs(config))
    scale = full / r["dofs"]
    wall = statistics.mean(walls)
    per_solve = wall / r["procs"] * scale  # projected seconds per full-size solve
    value = 1.0 / per_solve
    sample = (f"each step: {r['procs']} single-threaded oracle solves (one per host core, at "
              f"once) of the same discretisation truncated to {levels} levels ({r['dofs']} "
              f"dofs); solves/s of the sample scaled x{scale:.1f} to {full} dofs by the "
              f"method's linear work (Theorem 3.3)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
        "ms_per_step_note": "measured wall time of one step (the sample on all cores)",
        "projected_ms_per_full_solve": per_solve * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": r["procs"], "kind": "oracle",
                         "sample": sample, "bitwise_equal_across_cores": len(r["digests"]) == 1},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


GOLDEN_3D = os.path.join(ROOT, "tests", "golden", "oracle_config3_6levels.txt")
# precision modes whose eigenpair is compared with the oracle: (key, precision, flags)
ACCURACY_MODES = (("fp64", 0, 0), ("mixed_fp32", 1, 0), ("mixed_fp32_rhs32", 1, 2),
                  ("mixed_bf16_storage", 2, 0))


def read_golden_3d(path: str = GOLDEN_3D) -> dict | None:
    """The oracle's stored result for the 3D trap at h = 1/128 (config 3 truncated to 6 levels;
    written by tests/golden/make_oracle_3d_golden.py, which calls only the oracle): lambda per
    level, u at every `step`-th interior node per direction, and the sum and norm of u."""
    import numpy as np

    if not os.path.exists(path):
        return None
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
    d["u"] = np.array(samples)
    n, step = int(d["cells"]), int(d["step"])
    g = np.arange(step, n, step) - 1
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    d["idx"] = (i + (n - 1) * (j + (n - 1) * k)).ravel()
    return d


def gpu_solve_u(kw: dict, precision: int, flags: int = 0):
    """(lambda, u) of one solve through the C ABI with a host output buffer."""
    import numpy as np

    from paper_1502_04657_gb300 import fmg

    p = fmg.Problem(**{k: v for k, v in kw.items() if k in fmg.Problem.__dataclass_fields__},
                    precision=precision, flags=flags)
    with fmg.Solver(p) as s:
        u = np.empty(p.size(p.levels))
        lam, _, rc = s.solve(u)
    return lam, u, rc


def accuracy_vs_oracle(lam2: float, u2, levels2: int, gold3: dict | None) -> dict:
    """Eigenvalue and eigenvector error of every precision mode against the oracle, at sizes
    whose finest FMG stage runs the single-precision V-cycles through the TMA-fed sweeps:
    config 2 truncated to `levels2` levels (h = 1/512 at 7) against a live oracle run, and
    config 3 truncated to 6 levels (h = 1/128) against the stored oracle result (u compared on
    its sampled nodes)."""
    import numpy as np

    out = {}
    kw2 = problem_kwargs("config2", levels2)
    kw3 = problem_kwargs("config3", 6)
    for key, prec, flags in ACCURACY_MODES:
        lam, u, rc = gpu_solve_u(kw2, prec, flags)
        row = {"config2_%dlevels" % levels2: {
            "dlambda_rel": abs(lam - lam2) / lam2,
            "du_rel_l2": float(np.linalg.norm(u - u2) / np.linalg.norm(u2)), "status": rc}}
        if gold3 is not None:
            lam, u, rc = gpu_solve_u(kw3, prec, flags)
            ref = gold3["lambda_levels"][-1]
            us = u[gold3["idx"]]
            row["config3_6levels"] = {
                "dlambda_rel": abs(lam - ref) / ref,
                "du_rel_l2_sampled": float(np.linalg.norm(us - gold3["u"]) / np.linalg.norm(gold3["u"])),
                "du_norm2_rel": abs(float(np.linalg.norm(u)) - gold3["u_norm2"]) / gold3["u_norm2"],
                "status": rc}
        out[key] = row
    return out


def measure(workload: str, steps: int, warmup: int, world: int, local: int, dist=None,
            with_e2e: bool = True, clocks: bool = True, levels: int | None = None,
            autotune: bool = True, flags: int = 0) -> dict:
    import torch

    from paper_1502_04657_gb300 import fmg

    config, mixed, desc = WORKLOADS[workload]
    kw = problem_kwargs(config, levels)
    if levels is not None:
        desc = f"{desc} [truncated to {levels} levels for profiling]"
    gp = fmg.Problem(**{k: v for k, v in kw.items() if k in fmg.Problem.__dataclass_fields__})
    if mixed:
        gp.precision = fmg.FMG_MIXED_BF16 if mixed == "bf16" else fmg.FMG_MIXED_FP32
    gp.flags = flags | (0 if autotune else fmg.FMG_FLAG_NO_AUTOTUNE)
    n = gp.size(gp.levels)
    solver = fmg.Solver(gp)
    stream = torch.cuda.Stream()
    lam_d = torch.empty(1, dtype=torch.float64, device="cuda")
    u_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            solver.solve_dev(lam_d, u_d, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk_s = Clocks(local) if clocks else None
        if clk_s:
            clk_s.start()
            time.sleep(0.25)
        evs[0].record(stream)
        for i in range(steps):
            solver.solve_dev(lam_d, u_d, stream=stream.cuda_stream)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        clk = clk_s.stop() if clk_s else None
        if dist:
            dist.barrier()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    out = {"value": world * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
           "step_ms": step_ms, "lambda": float(lam_d.item()), "dofs": n, "desc": desc,
           "profile": solver.profile(), "kernels": solver.kernel_count(), "clocks": clk,
           "dim": gp.dim, "mixed": mixed, "n_finest": gp.coarse_cells << (gp.levels - 1),
           "nb_finest": 1}
    if with_e2e:
        u_host = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        e2e_steps = max(3, min(steps, 10))
        solver.solve(u_host)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            lam_e2e, _, _ = solver.solve(u_host)
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(dist, e2e_s, "cuda")
        out["e2e"] = {"value": world * e2e_steps / e2e_s, "unit": "solves/s",
                      "h2d_bytes_per_step": 112, "d2h_bytes_per_step": 8 + 8 * n + 4 * 16}
        out["lambda_e2e"] = lam_e2e
        _, st, _ = solver.solve(u_host, stats=True)
        out["scf_iters"] = list(st.scf_iters)[:gp.levels]
        out["identity_defect"] = st.identity_defect
    solver.close()
    return out


def measure_batch(steps: int, warmup: int, world: int, local: int, dist=None) -> dict:
    """config4: the 256-instance batch, mixed precision, one batch handle; beside it the same
    instances as 256 sequential FP64 single-instance solves (the plain per-instance path)."""
    import numpy as np
    import torch

    from paper_1502_04657_gb300 import fmg

    kws = batch_instances(256)
    fields = fmg.Problem.__dataclass_fields__
    mixed = [fmg.Problem(**{k: v for k, v in kw.items() if k in fields}, precision=fmg.FMG_MIXED_FP32)
             for kw in kws]
    plain = [fmg.Problem(**{k: v for k, v in kw.items() if k in fields}) for kw in kws]
    t0 = time.perf_counter()
    batch = fmg.BatchSolver(mixed)
    create_s = time.perf_counter() - t0
    nb = len(mixed)
    dofs = sum(p.size(p.levels) for p in mixed)
    stream = torch.cuda.Stream()
    lams = torch.empty(nb, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            batch.solve_dev_all(lams, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if dist:
            dist.barrier()
        clk_s = Clocks(local)
        clk_s.start()
        time.sleep(0.25)
        evs[0].record(stream)
        for i in range(steps):
            batch.solve_dev_all(lams, stream=stream.cuda_stream)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        clk = clk_s.stop()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    lam_batch = lams.cpu().numpy()
    prof = batch.profile()
    kernels = batch.kernel_count()
    levels = [p.levels for p in mixed]
    finest = max(levels)
    at_finest = sum(1 for v in levels if v == finest)
    tiles = {k: list(batch.level_tile(k)) for k in range(1, finest + 1)}
    # end to end: fmg_eig_batch_solve with host outputs (every u copied back)
    e2e_steps = 3
    batch.solve_all(with_u=True)
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        lam_e2e, _, _, codes = batch.solve_all(with_u=True)
    e2e_s = time.perf_counter() - t1
    batch.close()
    # 256 sequential FP64 single-instance solves of the same instances
    singles = [fmg.Solver(p) for p in plain]
    lam_seq = torch.empty(nb, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for i, s in enumerate(singles):  # warm-up pass
            s.solve_dev(lam_seq[i:i + 1], stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, s in enumerate(singles):
            s.solve_dev(lam_seq[i:i + 1], stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    lam_seq = lam_seq.cpu().numpy()
    for s in singles:
        s.close()
    dlam = float(np.max(np.abs(lam_batch - lam_seq) / lam_seq))
    return {"value": world * nb * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
            "step_ms": step_ms, "dofs": dofs, "dofs_finest_launch": at_finest * ((8 << (finest - 1)) - 1) ** 2,
            "profile": prof, "kernels": kernels, "clocks": clk, "dim": 2, "mixed": True,
            "n_finest": 8 << (finest - 1), "nb_finest": at_finest, "nb": nb, "tiles": tiles, "create_s": create_s,
            "e2e": {"value": world * nb * e2e_steps / e2e_s, "unit": "solves/s",
                    "h2d_bytes_per_step": nb * 112,
                    "d2h_bytes_per_step": 8 * dofs + nb * (8 + 4 + 16 * 12)},
            "sequential_fp64": {"value": nb / (seq_ms / 1e3), "unit": "solves/s", "ms": seq_ms},
            "max_dlambda_rel_vs_sequential_fp64": dlam,
            "all_converged": all(c == 0 for c in codes), "levels_histogram":
                {str(v): levels.count(v) for v in sorted(set(levels))}}


# Tables 1 and 2 of the paper (Section 4): seconds of Algorithm 3.2 per finest mesh on a
# PowerEdge R720 with ARPACK, by number of elements (context only: other hardware and coarse
# space).  The tables print 1572846 for 8 x 196608 = 1572864.
PAPER_TABLE = {1.0: {3072: 0.45, 24576: 1.55, 196608: 8.08, 1572864: 63.01, 12582912: 519.86},
               100.0: {24576: 4.32, 196608: 11.43, 1572864: 70.88, 12582912: 577.52}}


def paper_examples_arm(args, world, local, dist):
    """The paper's two examples on its meshes (context run beside Tables 1-2)."""
    import torch

    from paper_1502_04657_gb300 import fmg

    rank = rank_info()[0]
    rows = []
    stream = torch.cuda.Stream()
    def timed(p):
        with fmg.Solver(p) as s:
            lam = torch.empty(1, dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    s.solve_dev(lam, stream=stream.cuda_stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    s.solve_dev(lam, stream=stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize()
            _, st, rc = s.solve(stats=True)
        return e0.elapsed_time(e1) / args.steps, lam, st, rc

    for zeta in (1.0, 100.0):
        for levels in range(2, 7):  # finest h = 1/8 .. 1/128 from the h = 1/4 coarse space
            p = fmg.Problem(dim=3, coarse_cells=4, levels=levels, w_const=0.0,
                            w_quad=(1.0, 1.0, 1.0), zeta=zeta, vcycles=1, corrections=1,
                            nu_pre=3, nu_post=3, smoother=fmg.FMG_SMOOTH_CG)
            elements = 6 * (4 << (levels - 1)) ** 3
            ms, lam, st, rc = timed(p)
            p.smoother = fmg.FMG_SMOOTH_CHEBYSHEV
            ms_cheb, lam_cheb, _, _ = timed(p)
            p.smoother = fmg.FMG_SMOOTH_CG
            # the discrete eigenvalue of the same mesh: 10 corrections per level
            p.corrections = 10
            with fmg.Solver(p) as s:
                lam_ref, _, _ = s.solve()
            lam1 = float(lam.item())
            rows.append({"zeta": zeta, "h": f"1/{4 << (levels - 1)}", "elements": elements,
                         "dofs": p.size(levels), "ms": ms, "lambda": lam1,
                         "lambda_p10": lam_ref, "fmg_error_rel": abs(lam1 - lam_ref) / lam_ref,
                         "identity_defect": st.identity_defect, "status": rc,
                         "ms_chebyshev": ms_cheb, "lambda_chebyshev": float(lam_cheb.item()),
                         "paper_s": PAPER_TABLE[zeta].get(elements)})
    big = [r for r in rows if r["zeta"] == 1.0][-1]
    line = {
        "metric": METRIC, "value": 1e3 / big["ms"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": big["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS["paper-examples"][2],
                                        "parallelism": "replicas"},
        "rows": rows,
        "note": "paper_s: seconds the paper reports for the same element count (PowerEdge R720, "
                "ARPACK, coarse space h = 1/8); context, not a target",
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_serve(nreq: int, max_batch: int, max_inflight: int, window: float, world: int,
                  local: int, dist=None, sample: int = 48) -> dict:
    """fmg_eig_serve over the first nreq requests of the config-5 stream (rank r serves every
    world-th one), after a short warm-up stream; accuracy on a seeded sample of requests
    solved alone in FP64."""
    import numpy as np
    import torch

    from paper_1502_04657_gb300 import fmg

    rank = rank_info()[0]
    reqs = shard(serve_stream(nreq), rank, world)
    fields = fmg.Problem.__dataclass_fields__
    probs = [fmg.Problem(**{k: v for k, v in r.items() if k in fields},
                         precision=fmg.FMG_MIXED_FP32) for r in reqs]
    t0 = reqs[0]["arrival_s"]
    arrivals = [r["arrival_s"] - t0 for r in reqs]
    # warm-up: a short stream of the same kinds (first cohort builds, memory pool growth)
    fmg.serve(probs[:48], [0.0] * 48, max_batch=16, max_inflight=4)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_s = Clocks(local)
    clk_s.start()
    res, st = fmg.serve(probs, arrivals, max_batch=max_batch, max_inflight=max_inflight,
                        batch_window_s=window)
    clk = clk_s.stop()
    rng = np.random.default_rng(4657)
    idx = rng.choice(len(probs), size=min(sample, len(probs)), replace=False)
    worst = 0.0
    for i in idx:
        p = fmg.Problem(**{k: v for k, v in reqs[i].items() if k in fields})
        with fmg.Solver(p) as s:
            lam, _, _ = s.solve()
        worst = max(worst, abs(res[i]["lambda"] - lam) / lam)
    value = st["solves_per_s"]
    if dist:
        value = nreq / max_over_ranks(dist, st["makespan_s"], "cuda")
    return {"value": value, "st": st, "res": res, "probs": probs, "arrivals": arrivals,
            "clocks": clk, "worst": worst, "sample": int(len(idx))}


def serve_summary(m: dict) -> dict:
    st = m["st"]
    dofs = sum(p.size(p.levels) for p in m["probs"])
    return {
        "latency_ms": {"p50": st["p50_s"] * 1e3, "p99": st["p99_s"] * 1e3,
                       "mean": st["mean_s"] * 1e3, "max": st["max_s"] * 1e3},
        "mdof_per_s": dofs / st["makespan_s"] / 1e6,
        "peak_hbm_gb": st["peak_bytes"] / 1e9, "hbm_budget_gb": st["budget_bytes"] / 1e9,
        "peak_hbm_note": "in-flight and pooled (reusable) hierarchies",
        "cohorts": st["cohorts"], "max_cohort": st["max_cohort"],
        "cohorts_replaying_pooled_graph": st["reused"], "pooled_evicted": st["evicted"],
        "max_inflight_seen": st["max_inflight_seen"], "completed": st["completed"],
        "max_dlambda_rel_vs_fp64_alone": m["worst"], "dlambda_sample": m["sample"],
        "all_converged": all(r["status"] == 0 for r in m["res"]),
    }


def serve_arm(args, world, local, dist):
    """config5: fmg_eig_serve over the request stream (rank r serves every world-th request)."""
    rank = rank_info()[0]
    m = measure_serve(args.serve_requests, args.serve_batch, args.serve_inflight,
                      args.serve_window, world, local, dist)
    probs, arrivals, value, st = m["probs"], m["arrivals"], m["value"], m["st"]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": st["makespan_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["config5"][2], "requests": len(probs),
                   "offered_rate_per_s": len(probs) / max(arrivals[-1], 1e-9),
                   "max_batch": args.serve_batch, "max_inflight": args.serve_inflight,
                   "batch_window_s": args.serve_window, "parallelism": "replicas",
                   "l2": "resident hierarchies of GBs >> 129 MB L2; no flush"},
        **serve_summary(m),
        "clocks": m["clocks"],
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 112 * len(probs),
                "d2h_bytes_per_step": 8 * len(probs),
                "note": "the serve call is the end-to-end path: requests in host memory, "
                        "lambdas copied to host inside each request's latency"},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serve_cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


SERVE_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import fmg_oracle as O
from workloads import serve_stream
reqs = serve_stream(10000)[:{count}]
t = time.perf_counter()
dofs = 0
for r in reqs:
    kw = {{k: v for k, v in r.items() if k != "arrival_s"}}
    kw["levels"] = min(kw["levels"], {cap2} if kw["dim"] == 2 else {cap3})
    p = O.Problem(**kw)
    O.fmg_solve(p)
    dofs += (p.cells(p.levels) - 1) ** p.dim
print(json.dumps({{"time": time.perf_counter() - t, "dofs": dofs}}))
"""


def serve_cpu_baseline(count: int = 6, cap2: int = 6, cap3: int = 4) -> dict:
    """The oracle on the stream's first requests (levels capped), scaled by dofs."""
    env = {**os.environ, "OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    code = SERVE_ORACLE_SNIPPET.format(root=ROOT, count=count, cap2=cap2, cap3=cap3)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    reqs = serve_stream(10000)
    full = sum(((q["coarse_cells"] << (q["levels"] - 1)) - 1) ** q["dim"] for q in reqs)
    value = len(reqs) / (r["time"] / r["dofs"] * full)
    return {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle solves of the stream's first {count} requests with levels capped "
                       f"(2D {cap2}, 3D {cap3}; {r['dofs']} dofs, {r['time']:.1f} s on 1 host "
                       f"core), scaled by total dofs to the 10,000 requests ({full} dofs)")}


def roofline(m: dict, clk: dict, fp64_peak: dict | None = None) -> tuple[dict, dict]:
    """Roofline of the dominant kernel (and the others): FP64 kernels against the measured
    FP64 multiply-add rate of this run's probe when given (fp64_peak), else the nominal rate
    from unit counts and clock; the nominal fraction is kept beside the measured one."""
    sm_max = (clk or {}).get("sm_max_mhz") or 2070
    nominal = FP64_FLOP_PER_CLK_SM * N_SM * sm_max * 1e6 / 1e12
    peak = fp64_peak["tflops"] if fp64_peak else nominal
    roof = {}
    nodes = m.get("dofs_finest_launch", m["dofs"])  # nodes one finest-level launch processes
    mixed = m.get("mixed")
    if mixed:  # FP32 / BF16 V-cycle kernels against the HBM peak
        bpn = 6.0 if mixed == "bf16" else 12.0
        hpeak, hsrc = hbm_peak()
        for name in MIXED_HBM_KERNELS:
            ms = m["profile"].get(name, -1.0)
            if ms and ms > 0:
                ach = bpn * nodes / (ms * 1e-3) / 1e9
                roof[name + "32"] = {"bound": "hbm", "achieved": ach, "peak": hpeak, "unit": "GB/s",
                                     "frac": ach / hpeak, "traffic": None, "launch_ms": ms,
                                     "bytes_per_node": bpn, "peak_source": hsrc}
    ops_peak = peak / 2  # one FP64 instruction per multiply-add lane of the probe
    table = dict(KERNELS[m["dim"]])
    node_run = "n_finest" in m and not star_walks(m["dim"], m["n_finest"], m.get("nb_finest", 1))
    if node_run:
        table.update(NODE_KERNELS[m["dim"]])
    for name, (flops, nbytes, ops) in table.items():
        if mixed and name in MIXED_HBM_KERNELS:
            continue
        ms = m["profile"].get(name, -1.0)
        if mixed and name == "nload_density" and ms and ms > 0:
            ipeak = ISSUE_PER_CLK_SM * N_SM * sm_max * 1e6 / 1e12
            ach = DF_INSTR_PER_NODE[m["dim"]] * nodes / (ms * 1e-3) / 1e12
            roof[name] = {"bound": "alu", "achieved": ach, "peak": ipeak, "unit": "Tinst/s",
                          "frac": ach / ipeak, "traffic": DF_TRAFFIC_PER_NODE[m["dim"]] * nodes,
                          "launch_ms": ms, "arithmetic": "double-float on the FP32 pipes",
                          "peak_source": ("instruction issue: 152 SMs x 4 schedulers x 32 lanes "
                                          "x sm_max_mhz (derived from unit counts and clock)")}
            continue
        if ms and ms > 0:
            ach = flops * nodes / (ms * 1e-3) / 1e12
            # (the DRAM figures were captured on the walk kernels)
            tpn = None if node_run and name in NODE_KERNELS[m["dim"]] else \
                TRAFFIC_PER_NODE.get((m["dim"], name))
            ops_ach = ops * nodes / (ms * 1e-3) / 1e12
            roof[name] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "traffic": tpn * nodes if tpn else None,
                          "peak_nominal": nominal, "frac_nominal": ach / nominal,
                          "launch_ms": ms,
                          "hbm_gbs_algorithmic": nbytes * nodes / (ms * 1e-3) / 1e9,
                          "fp64_inst": {"per_node": ops, "achieved": ops_ach, "peak": ops_peak,
                                        "unit": "T FP64 instructions/s",
                                        "frac": ops_ach / ops_peak}}
    dom = DOMINANT[m["dim"]]
    if dom not in roof:  # FP32 V-cycles (mixed modes): the FP64 nonlinear pass dominates
        dom = "nload_density"
    main = dict(roof.get(dom, {}))
    main["kernel"] = dom
    if fp64_peak:
        main.setdefault("peak_source", "of measured: FP64 multiply-add probe of this run "
                        f"(fmg_eig_probe_fma, best of {fp64_peak['launches']} launches, "
                        f"{fp64_peak['tflops']:.4f} TFLOP/s); peak_nominal = 152 SMs x 2 FP64 "
                        "FMA lanes/clk x sm_max_mhz")
    else:
        main.setdefault("peak_source", "FP64 (the kernel is FP64-ALU bound): 152 SMs x 2 FP64 "
                        "FMA lanes/clk x sm_max_mhz, nominal 1.26 TFLOP/s (no probe run)")
    return main, {k: v for k, v in roof.items() if k != dom}


def fma_probe(fp64: bool = True, shapes=(2, 4, 8), reps: int = 3) -> dict:
    """Best multiply-add rate of the library's probe over a few launch shapes (TFLOP/s)."""
    from paper_1502_04657_gb300 import fmg

    iters = 16384 if fp64 else 262144
    best, rows = 0.0, []
    for cps in shapes:
        for _ in range(reps):
            ms, fl = fmg.probe_fma(fp64, cps, iters)
            tf = fl / (ms * 1e-3) / 1e12
            rows.append({"ctas_per_sm": cps, "ms": ms, "tflops": tf})
            best = max(best, tf)
    return {"tflops": best, "launches": len(rows), "iters": iters, "rows": rows,
            "precision": "fp64" if fp64 else "fp32"}


def probe_arm(args):
    """--probe-fp64: the FP64 (and FP32) multiply-add rate, with the SM clock sampled while the
    probe runs (about 2 s of launches), reported as measured, per sampled clock and scaled to
    the maximum clock (time x median SM MHz)."""
    import torch

    torch.cuda.set_device(rank_info()[2])
    fma_probe(True, (4,), 1)  # warm-up
    clk_s = Clocks(rank_info()[2])
    clk_s.start()
    time.sleep(0.25)
    t_end = time.perf_counter() + 2.0
    runs = []
    while time.perf_counter() < t_end:
        runs.append(fma_probe(True, (2, 4, 8), 1))
    fp32 = fma_probe(False, (2, 4, 8), 2)
    clk = clk_s.stop()
    best = max(r["tflops"] for r in runs)
    mhz, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    out = {"probe": "fmg_eig_probe_fma", "fp64_tflops_best": best,
           "fp64_tflops_median": statistics.median(x["tflops"] for r in runs for x in r["rows"]),
           "fp64_launches": sum(r["launches"] for r in runs),
           "fp64_rows_last": runs[-1]["rows"], "fp32_tflops_best": fp32["tflops"],
           "fp32_rows": fp32["rows"], "clocks": clk,
           "fp64_nominal_tflops_at_sm_max": FP64_FLOP_PER_CLK_SM * N_SM * (mx or 2070) * 1e6 / 1e12}
    if mhz and mx:
        out["fp64_tflops_scaled_to_sm_max"] = best * mx / mhz
    print(json.dumps(out), flush=True)


def ours_arm(args):
    import torch

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "config4":
        return batch_arm(args, world, local, dist)
    if args.workload == "config5":
        return serve_arm(args, world, local, dist)
    if args.workload == "paper-examples":
        return paper_examples_arm(args, world, local, dist)
    m = measure(args.workload, args.steps, args.warmup, world, local, dist, levels=args.levels,
                autotune=not args.no_autotune)
    main, other = roofline(m, m["clocks"])
    step_ms = m["step_ms"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64+bf16" if m["mixed"] == "bf16" else "f64+f32") if m["mixed"] else "f64",
        "data": "synthetic",
        "config": {"workload": m["desc"], "dofs": m["dofs"], "parallelism": "replicas",
                   "l2": "per-step working set > 2 GB >> 129 MB L2; no flush"},
        "mdof_per_s": m["value"] * m["dofs"] / 1e6,
        # one finest-level V-cycle (event-timed inside the solve graph): finest dofs / its time
        "mdof_per_s_per_vcycle": (m["dofs"] / (m["profile"]["vcycle"] * 1e-3) / 1e6
                                  if m["profile"].get("vcycle", -1) > 0 else None),
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "lambda": m["lambda"], "lambda_e2e": m["lambda_e2e"],
        "clocks": m["clocks"], "e2e": m["e2e"], "gpu_launches": args.steps * m["kernels"],
        "kernels_per_step": m["kernels"], "roofline": main, "roofline_other": other,
        "kernel_ms_finest": m["profile"],
        "small_solve_iters_per_level": m.get("scf_iters"),
        "identity_defect": m.get("identity_defect"),
    }
    extras = args.workload == "config2" and not args.no_extras
    if extras:
        for key, wl, flags in (("mixed_fp32", "config2-mixed", 0),
                               ("mixed_fp32_rhs32", "config2-mixed", 2),
                               ("mixed_bf16_storage", "config2-bf16", 0)):
            mx = measure(wl, max(3, args.steps // 2), 3, world, local, dist,
                         with_e2e=False, clocks=False, flags=flags)
            _, mroof = roofline(mx, m["clocks"])
            line[key] = {"value": mx["value"], "unit": "solves/s", "ms_per_step": mx["ms_per_step"],
                         "lambda": mx["lambda"],
                         "dlambda_rel_vs_fp64": abs(mx["lambda"] - m["lambda"]) / m["lambda"],
                         "roofline_v_cycle": {k: v for k, v in mroof.items() if k.endswith("32")},
                         "kernel_ms_finest": mx["profile"]}
    if not args.no_extras and m["dim"] in (2, 3):
        # the FP64 roofline against this run's own multiply-add probe
        probe = fma_probe(True)
        main, other = roofline(m, m["clocks"], probe)
        line["roofline"], line["roofline_other"] = main, other
        line["fp64_probe"] = {"tflops": probe["tflops"], "launches": probe["launches"],
                              "rows": probe["rows"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np

        config = WORKLOADS[args.workload][0]
        levels = ORACLE_SAMPLE[config][0]
        fd, u_path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        r = run_oracle(config, levels, 1, u_path=u_path)
        u_or = np.load(u_path)
        os.unlink(u_path)
        allc = run_oracle_all_cores(config, levels)
        full = dofs_of(problem_kwargs(config))
        scale = full / r["dofs"]
        t = r["times"][0]
        line["cpu_baseline"] = {
            "value": 1.0 / (allc["per_sample_s"] * scale), "unit": "solves/s",
            "cores": allc["procs"], "kind": "oracle",
            "sample": (f"{allc['procs']} single-threaded oracle solves of the same discretisation "
                       f"truncated to {levels} levels ({r['dofs']} dofs), one per host core at "
                       f"once, took {allc['wall_s']:.1f} s of wall time; solves/s of the sample "
                       f"scaled x{scale:.1f} to {full} dofs by the method's linear work "
                       f"(Theorem 3.3)"),
            "nproc": os.cpu_count(),
            "bitwise_equal_across_cores": allc["digests"] == [r["digest"]],
            "single_core": {
                "value": 1.0 / (t * scale), "cores": 1,
                "sample": (f"one oracle solve of the same {r['dofs']} dofs took {t:.1f} s on 1 "
                           f"host core, scaled x{scale:.1f}")},
            "lambda_sample": r["lam"],
        }
        if config in ("config2", "config3") and not args.no_extras:
            acc = accuracy_vs_oracle(r["lam"], u_or, levels, read_golden_3d()) \
                if config == "config2" else None
            if acc:
                line["accuracy_vs_oracle"] = acc
                for key, _, _ in ACCURACY_MODES:
                    row = acc[key][f"config2_{levels}levels"]
                    tgt = line if key == "fp64" else line.get(key)
                    if tgt is not None:
                        tgt["dlambda_rel_vs_oracle"] = row["dlambda_rel"]
                        tgt["du_rel_vs_oracle"] = row["du_rel_l2"]
                        tgt["vs_oracle_at"] = (f"config 2 truncated to {levels} levels "
                                               f"({r['dofs']} dofs), the oracle's own size")
    if extras:
        b = measure_batch(5, 3, world, local, dist)
        line["config4_batch"] = {
            "workload": WORKLOADS["config4"][2], "steps": 5, "warmup": 3,
            "value": b["value"], "unit": "solves/s", "ms_per_step": b["ms_per_step"],
            "sequential_fp64": b["sequential_fp64"],
            "speedup_vs_sequential_fp64": b["value"] / world / b["sequential_fp64"]["value"],
            "max_dlambda_rel_vs_sequential_fp64": b["max_dlambda_rel_vs_sequential_fp64"],
            "all_converged": b["all_converged"], "e2e": b["e2e"], "clocks": b["clocks"],
            "kernels_per_step": b["kernels"]}
        sv = measure_serve(2000, args.serve_batch, args.serve_inflight, args.serve_window,
                           world, local, dist)
        line["config5_serve"] = {
            "workload": "the config-5 stream's first 2,000 requests (200/s offered, 70% 2D / "
                        "30% 3D), FP32 V-cycles in FP64 defect correction",
            "value": sv["value"], "unit": "solves/s", "makespan_s": sv["st"]["makespan_s"],
            **serve_summary(sv), "clocks": sv["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_arm(args, world, local, dist):
    rank = rank_info()[0]
    m = measure_batch(args.steps, args.warmup, world, local, dist)
    main, other = roofline(m, m["clocks"])
    step_ms = m["step_ms"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["config4"][2], "instances": m["nb"], "dofs": m["dofs"],
                   "levels_histogram": m["levels_histogram"], "parallelism": "replicas",
                   "tiles": m["tiles"],
                   "l2": "per-step working set > 10 GB >> 129 MB L2; no flush"},
        "mdof_per_s": m["value"] / m["nb"] * m["dofs"] / 1e6,
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "sequential_fp64": m["sequential_fp64"],
        "speedup_vs_sequential_fp64": m["value"] / world / m["sequential_fp64"]["value"],
        "max_dlambda_rel_vs_sequential_fp64": m["max_dlambda_rel_vs_sequential_fp64"],
        "all_converged": m["all_converged"], "handle_create_s": m["create_s"],
        "clocks": m["clocks"], "e2e": m["e2e"], "gpu_launches": args.steps * m["kernels"],
        "kernels_per_step": m["kernels"], "roofline": main, "roofline_other": other,
        "kernel_ms_finest": m["profile"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


BATCH_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import fmg_oracle as O
from workloads import batch_instances
kws = batch_instances(256)[:{count}]
t = time.perf_counter()
dofs = 0
for kw in kws:
    kw = dict(kw, levels=min(kw["levels"], {cap}))
    p = O.Problem(**kw)
    O.fmg_solve(p)
    dofs += (p.cells(p.levels) - 1) ** 2
print(json.dumps({{"time": time.perf_counter() - t, "dofs": dofs}}))
"""


def batch_cpu_baseline(count: int = 8, cap: int = 6) -> dict:
    """The oracle on the first instances of the batch (levels capped), scaled by dofs."""
    from workloads import batch_instances as bi

    env = {**os.environ, "OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    code = BATCH_ORACLE_SNIPPET.format(root=ROOT, count=count, cap=cap)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    full = sum(((kw["coarse_cells"] << (kw["levels"] - 1)) - 1) ** 2 for kw in bi(256))
    per_dof = r["time"] / r["dofs"]
    return {"value": 256 / (per_dof * full), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle solves of the first {count} batch instances with levels capped at "
                       f"{cap} ({r['dofs']} dofs, {r['time']:.1f} s on 1 host core), scaled by "
                       f"total dofs to the 256-instance batch ({full} dofs)")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="config2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--levels", type=int, default=None,
                    help="truncate a single-solve workload's level count (small profiling cases)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default 32x8 tiles (a fixed launch sequence for ncu captures)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-batch", type=int, default=32)
    ap.add_argument("--serve-inflight", type=int, default=6)
    ap.add_argument("--serve-window", type=float, default=0.002)
    ap.add_argument("--probe-fp64", action="store_true",
                    help="measure the FP64 / FP32 multiply-add rate with clocks and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.probe_fp64:
        probe_arm(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
