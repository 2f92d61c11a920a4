#!/usr/bin/env python3
"""Benchmark of the full multigrid GP ground-state solver (one JSON line on rank 0).

Workload (N = 1): the 16.8M-dof 2D configuration - unit square, P1 mesh with (1,1)
diagonals, coarsest h = 1/8 refined 9 times to h = 1/4096 (16,769,025 interior dofs),
W = x^2 + y^2, zeta = 10, 2 V-cycles of 2 + 2 damped Jacobi (omega = 2/3) per level, one
correction per level, FP64 throughout.  A step is one complete solve (Algorithm 3.2,
including the per-solve operator setup and the upload of the problem parameters); inputs are
resident and the per-solve working set (~2.3 GB) is far larger than the 129 MB L2, so no
flush is needed between steps.

--impl ours (default): the CUDA library.  value = solves/s over the timed steps (CUDA events
on the launch stream), max over ranks; e2e = the same metric through fmg_eig_solve with a
pinned host output buffer (parameter upload and the D2H copy of lambda and u inside).
--impl reference: the FP64 CPU oracle on this host's cores (rank 0 only), each step a
bounded sample of the workload (h = 1/256), scaled to the full size by the method's linear
work (Theorem 3.3).
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

from workloads import seeded_problem_2d  # noqa: E402

METRIC = "GP ground-state solves/s and fine-grid MDOF/s at |Δλ|≤1e-8; p50/p99 latency"
CONFIG = "config2"
WORKLOAD = ("2D unit square, P1 right-triangle mesh, coarsest h=1/8 refined to h=1/4096 "
            "(10 levels, 16,769,025 dofs), W=x^2+y^2, zeta=10, m=2 V-cycles, p=1, 2+2 damped "
            "Jacobi omega=2/3, FP64 plain per-instance solve")
FP64_FLOP_PER_CLK_SM = 4      # 2 DFMA per clock per SM (1.25 TFLOP/s nominal at 2070 MHz)
N_SM = 152
# Algorithmic FP64 flops per finest-level launch unit ("Kernels"):
#   Jacobi sweep: 7-point L x (7 mul + 6 add) + residual (1) + scale (1) + update (1) = 16 per node
#   moments: per fine triangle 6 quadrature points x 68 flops = 408 (2 triangles per node)
FLOPS_PER_UNIT = {"jacobi": 16.0, "moments": 816.0, "residual": 14.0, "rhs": 66.0}
BYTES_PER_UNIT = {"jacobi": 24.0 + 40.0, "moments": 8.0, "residual": 24.0 + 40.0, "rhs": 16.0}
DOMINANT = "moments"


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class Clocks:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] != "[N/A]")}


def problem_kwargs(levels=None):
    kw = seeded_problem_2d(CONFIG)
    if levels is not None:
        kw["levels"] = levels
    return kw


ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import fmg_oracle as O
from workloads import seeded_problem_2d
kw = seeded_problem_2d({cfg!r}, levels={levels})
times = []
for _ in range({reps}):
    t = time.perf_counter()
    prob = O.Problem(**kw)
    r = O.fmg_solve(prob)
    times.append(time.perf_counter() - t)
print(json.dumps({{"times": times, "lam": r.lam, "dofs": (prob.cells(prob.levels) - 1) ** 2}}))
"""


def run_oracle(levels: int, reps: int) -> dict:
    """The oracle in a fresh single-threaded interpreter (exec'd, never forked from CUDA)."""
    env = {**os.environ, "OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=CONFIG, levels=levels, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def full_dofs() -> int:
    kw = problem_kwargs()
    return ((kw["coarse_cells"] << (kw["levels"] - 1)) - 1) ** kw["dim"]


def reference_arm(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    sample_levels = 6
    steps = []
    for i in range(args.warmup + args.steps):
        r = run_oracle(sample_levels, 1)
        if i >= args.warmup:
            steps.append(r["times"][0])
    scale = full_dofs() / r["dofs"]
    per_solve = statistics.mean(steps) * scale
    value = 1.0 / per_solve
    sample = (f"oracle solve of the same discretisation truncated to 6 levels (h=1/256, {r['dofs']} dofs) "
              f"per step, scaled x{scale:.1f} to 16,769,025 dofs by the method's linear work (Theorem 3.3)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ours_arm(args):
    import numpy as np
    import torch

    from paper_1502_04657_gb300 import fmg

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kw = problem_kwargs()
    gp = fmg.Problem(**{k: v for k, v in kw.items() if k in fmg.Problem.__dataclass_fields__})
    n = gp.size(gp.levels)
    solver = fmg.Solver(gp)
    stream = torch.cuda.Stream()
    lam_d = torch.empty(1, dtype=torch.float64, device="cuda")
    u_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            solver.solve_dev(lam_d, u_d, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        time.sleep(0.25)
        evs[0].record(stream)
        for i in range(args.steps):
            solver.solve_dev(lam_d, u_d, stream=stream.cuda_stream)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if dist:
            dist.barrier()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)
    prof = solver.profile()  # finest-level launches of the last timed solve
    lam = float(lam_d.item())

    # end to end: public host-buffer call, parameter upload + D2H of lambda and u inside
    u_host = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(3, min(args.steps, 10))
    solver.solve(u_host)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lam_e2e, _, _ = solver.solve(u_host)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 112,
           "d2h_bytes_per_step": 8 + 8 * n + 4 * 16}

    kernels_per_solve = solver.kernel_count()
    gpu_launches = args.steps * (kernels_per_solve)
    sm_max = clk.get("sm_max_mhz") or 2070
    peak_tflops = FP64_FLOP_PER_CLK_SM * N_SM * sm_max * 1e6 / 1e12
    roof = {}
    for name in ("moments", "jacobi"):
        ms = prof.get(name, -1.0)
        if ms and ms > 0:
            units = n
            ach = FLOPS_PER_UNIT[name] * units / (ms * 1e-3) / 1e12
            roof[name] = {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                          "frac": ach / peak_tflops, "traffic": None, "launch_ms": ms,
                          "hbm_gbs": BYTES_PER_UNIT[name] * units / (ms * 1e-3) / 1e9}
    roofline = dict(roof.get(DOMINANT, {}))
    roofline["kernel"] = DOMINANT
    roofline["peak_source"] = "FP64: 152 SMs x 2 DFMA/clk x sm_max_mhz (nominal 1.25 TFLOP/s)"

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dofs": n, "parallelism": "replicas",
                   "l2": "per-step working set ~2.3 GB >> 129 MB L2; no flush"},
        "mdof_per_s": value * n / 1e6,
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "lambda": lam, "lambda_e2e": lam_e2e,
        "clocks": clk, "e2e": e2e, "gpu_launches": gpu_launches,
        "kernels_per_step": kernels_per_solve, "roofline": roofline,
        "kernel_ms_finest": prof, "roofline_other": {k: v for k, v in roof.items() if k != DOMINANT},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle(7, 1)
        scale = full_dofs() / r["dofs"]
        t = r["times"][0]
        line["cpu_baseline"] = {
            "value": 1.0 / (t * scale), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"one oracle solve of the same discretisation truncated to 7 levels (h=1/512, "
                       f"{r['dofs']} dofs) took {t:.1f} s on 1 host core; scaled x{scale:.1f} to "
                       f"16,769,025 dofs by the method's linear work (Theorem 3.3)"),
            "lambda_sample": r["lam"],
        }
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
