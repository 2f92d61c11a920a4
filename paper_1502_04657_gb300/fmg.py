"""ctypes binding of libfmg_eig (include/fmg_eig.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels.  Importing this module never
falls back to anything else: if the shared library is missing the first call raises."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmg_eig.so")

FMG_OK, FMG_EINVAL, FMG_ENOMEM, FMG_ENOCONV, FMG_ECUDA, FMG_ETIMEOUT, FMG_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
FMG_FP64, FMG_MIXED_FP32, FMG_MIXED_BF16 = 0, 1, 2
FMG_W_LEFT, FMG_PAPER_LITERAL = 0, 1
FMG_SMOOTH_JACOBI, FMG_SMOOTH_CHEBYSHEV, FMG_SMOOTH_CG = 0, 1, 2
FMG_FLAG_NO_AUTOTUNE = 1
FMG_FLAG_FP32_RHS = 2
FMG_FLAG_NO_TMA = 4
FMG_FLAG_STAR_WALKS = 8
FMG_FLAG_SEPARATE_VCYCLE = 16
FMG_FLAG_EXPIRE_WAITS = 32
FMG_MAX_LEVELS = 16


class fmg_eig_problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("coarse_cells", C.c_int32), ("levels", C.c_int32),
        ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("vcycles", C.c_int32),
        ("corrections", C.c_int32), ("smoother", C.c_int32), ("precision", C.c_int32),
        ("operator_form", C.c_int32), ("scf_max_iter", C.c_int32), ("flags", C.c_int32),
        ("box_len", C.c_double), ("w_const", C.c_double), ("w_quad", C.c_double * 3),
        ("zeta", C.c_double), ("omega", C.c_double), ("scf_tol", C.c_double),
    ]


class fmg_eig_stats(C.Structure):
    _fields_ = [
        ("lambda_", C.c_double), ("solve_ms", C.c_double), ("norm_defect", C.c_double),
        ("identity_defect", C.c_double), ("lambda_levels", C.c_double * FMG_MAX_LEVELS),
        ("scf_iters", C.c_int32 * FMG_MAX_LEVELS), ("levels", C.c_int32), ("status", C.c_int32),
    ]


class fmg_eig_serve_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("batch_window_s", C.c_double),
                ("max_batch", C.c_int32), ("max_inflight", C.c_int32)]


class fmg_eig_request(C.Structure):
    _fields_ = [("problem", fmg_eig_problem), ("arrival_s", C.c_double),
                ("u", C.c_void_p), ("u_len", C.c_size_t)]


class fmg_eig_result(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("latency_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double), ("status", C.c_int32), ("cohort", C.c_int32)]


class fmg_eig_serve_stats(C.Structure):
    _fields_ = [("p50_s", C.c_double), ("p99_s", C.c_double), ("mean_s", C.c_double),
                ("max_s", C.c_double), ("solves_per_s", C.c_double), ("makespan_s", C.c_double),
                ("peak_bytes", C.c_double), ("budget_bytes", C.c_double), ("cohorts", C.c_int32),
                ("max_cohort", C.c_int32), ("max_inflight_seen", C.c_int32),
                ("completed", C.c_int32), ("reused", C.c_int32), ("evicted", C.c_int32)]


class FmgError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.c_int32

_SIGS = {
    "fmg_eig_create": (C.c_int, [C.POINTER(fmg_eig_problem), C.POINTER(_P)]),
    "fmg_eig_level_size": (C.c_size_t, [_P, _I32]),
    "fmg_eig_solve": (C.c_int, [_P, _D, _P, C.c_size_t, C.POINTER(fmg_eig_stats)]),
    "fmg_eig_solve_dev": (C.c_int, [_P, _P, _P, C.c_size_t, _P]),
    "fmg_eig_destroy": (None, [_P]),
    "fmg_eig_strerror": (C.c_char_p, [C.c_int]),
    "fmg_eig_set_params": (C.c_int, [_P, C.POINTER(fmg_eig_problem)]),
    "fmg_eig_kernel_count": (C.c_int, [_P]),
    "fmg_eig_profile": (C.c_int, [_P, _D, _I32]),
    "fmg_eig_apply_operator": (C.c_int, [_P, _I32, _P, _P, _P]),
    "fmg_eig_apply_mass": (C.c_int, [_P, _I32, _P, _P, _P]),
    "fmg_eig_jacobi": (C.c_int, [_P, _I32, _P, _P, _P, _P]),
    "fmg_eig_residual_restrict": (C.c_int, [_P, _I32, _P, _P, _P, _P]),
    "fmg_eig_prolong_add": (C.c_int, [_P, _I32, _P, _P, _P]),
    "fmg_eig_nonlinear_load": (C.c_int, [_P, _I32, _P, _P, _P]),
    "fmg_eig_aux_rhs": (C.c_int, [_P, _I32, C.c_double, _P, _P, _P]),
    "fmg_eig_multigrid": (C.c_int, [_P, _I32, _P, _P, _P]),
    "fmg_eig_correction": (C.c_int, [_P, _I32, C.c_double, _P, _D, _P, _P, C.POINTER(_I32)]),
    "fmg_eig_coarse_solve": (C.c_int, [_P, _D, _P, C.POINTER(_I32)]),
    "fmg_eig_augmented_system": (C.c_int, [_P, _I32, _P, _P, _I32, _P, _P, _P]),
    "fmg_eig_inject_alloc_failure": (C.c_int, [C.c_int64]),
    "fmg_eig_probe_fma": (C.c_int, [_I32, _I32, _I32, _P, _D, _D]),
    "fmg_eig_coarse_solve_noalloc": (C.c_int, [C.POINTER(fmg_eig_problem), _D, _P, C.POINTER(_I32), _P]),
    "fmg_eig_batch_create": (C.c_int, [C.POINTER(fmg_eig_problem), _I32, C.POINTER(_P)]),
    "fmg_eig_batch_count": (_I32, [_P]),
    "fmg_eig_batch_solve": (C.c_int, [_P, _D, C.POINTER(_P), C.POINTER(C.c_size_t),
                                      C.POINTER(fmg_eig_stats), C.POINTER(_I32)]),
    "fmg_eig_solve_batch": (C.c_int, [C.POINTER(fmg_eig_problem), _I32, _D, C.POINTER(_P),
                                      C.POINTER(C.c_size_t), C.POINTER(fmg_eig_stats),
                                      C.POINTER(_I32)]),
    "fmg_eig_level_tile": (C.c_int, [_P, _I32, C.POINTER(_I32), C.POINTER(_I32)]),
    "fmg_eig_batch_solve_dev": (C.c_int, [_P, _P, _P]),
    "fmg_eig_estimate_bytes": (C.c_size_t, [C.POINTER(fmg_eig_problem), _I32]),
    "fmg_eig_serve": (C.c_int, [C.POINTER(fmg_eig_serve_config), C.POINTER(fmg_eig_request), _I32,
                                C.POINTER(fmg_eig_result), C.POINTER(fmg_eig_serve_stats)]),
}


def inject_alloc_failure(after: int) -> None:
    """fmg_eig_inject_alloc_failure: the device allocation after `after` more successful ones
    fails once (test hook; negative cancels)."""
    load_library().fmg_eig_inject_alloc_failure(int(after))


def probe_fma(fp64: bool = True, ctas_per_sm: int = 4, iters: int = 4096, stream=None):
    """fmg_eig_probe_fma: (ms, flops) of one timed launch of the multiply-add probe."""
    ms, fl = C.c_double(), C.c_double()
    rc = load_library().fmg_eig_probe_fma(1 if fp64 else 0, ctas_per_sm, iters, stream,
                                          C.byref(ms), C.byref(fl))
    if rc != FMG_OK:
        raise FmgError(rc, "fmg_eig_probe_fma")
    return ms.value, fl.value


def coarse_solve_noalloc(problem: "Problem", u_dev, stream=None):
    """fmg_eig_coarse_solve_noalloc: the coarsest-level solve without a handle and without any
    device allocation (for callers that may not allocate).  u_dev receives u_{h_1}."""
    lib = load_library()
    cp = problem.to_c()
    lo = C.c_double()
    it = C.c_int32()
    rc = lib.fmg_eig_coarse_solve_noalloc(C.byref(cp), C.byref(lo), _ptr(u_dev), C.byref(it), stream)
    if rc not in (FMG_OK, FMG_ENOCONV):
        raise FmgError(rc, "fmg_eig_coarse_solve_noalloc")
    return lo.value, it.value, rc


def load_library(path: str = LIB_PATH):
    """Load libfmg_eig.so and declare every exported entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FmgError(FMG_ECUDA, f"libfmg_eig.so not built at {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load_library().fmg_eig_strerror(code).decode()
    except Exception:  # library missing: still give a readable message
        return str(code)


def exported_symbols() -> list[str]:
    return list(_SIGS)


@dataclass
class Problem:
    """Mirror of fmg_eig_problem with the defaults of the 2D benchmark configurations."""

    dim: int = 2
    coarse_cells: int = 8
    levels: int = 6
    nu_pre: int = 2
    nu_post: int = 2
    vcycles: int = 2
    corrections: int = 1
    precision: int = FMG_FP64
    operator_form: int = FMG_W_LEFT
    smoother: int = FMG_SMOOTH_JACOBI
    scf_max_iter: int = 100
    box_len: float = 1.0
    w_const: float = 0.0
    w_quad: tuple = (1.0, 1.0, 1.0)
    zeta: float = 1.0
    omega: float = 2.0 / 3.0
    scf_tol: float = 1e-13
    flags: int = 0

    def to_c(self) -> fmg_eig_problem:
        p = fmg_eig_problem()
        for f in ("dim", "coarse_cells", "levels", "nu_pre", "nu_post", "vcycles", "corrections",
                  "precision", "operator_form", "scf_max_iter", "box_len", "w_const", "zeta",
                  "omega", "scf_tol", "flags", "smoother"):
            setattr(p, f, getattr(self, f))
        p.w_quad[:] = [float(x) for x in self.w_quad]
        return p

    def cells(self, k: int) -> int:
        return self.coarse_cells << (k - 1)

    def size(self, k: int) -> int:
        return (self.cells(k) - 1) ** self.dim


def _ptr(t) -> int | None:
    """Device or host address of a torch tensor / numpy array (None passes NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


class Solver:
    """One handle of libfmg_eig; methods map 1:1 to the C entry points."""

    def __init__(self, problem: Problem):
        self.lib = load_library()
        self.problem = problem
        self._cp = problem.to_c()
        h = _P()
        rc = self.lib.fmg_eig_create(C.byref(self._cp), C.byref(h))
        if rc != FMG_OK:
            raise FmgError(rc, "fmg_eig_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmg_eig_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def level_size(self, k: int) -> int:
        return self.lib.fmg_eig_level_size(self.h, k)

    def level_tile(self, k: int) -> tuple:
        bx, by = _I32(), _I32()
        self._check(self.lib.fmg_eig_level_tile(self.h, k, C.byref(bx), C.byref(by)), "level_tile")
        return bx.value, by.value

    PROFILE_KEYS = ("jacobi", "residual", "restrict", "prolong", "rhs", "nload_density", "dense",
                    "vcycle", "t3", "coef")

    def set_params(self, problem: Problem):
        cp = problem.to_c()
        self._check(self.lib.fmg_eig_set_params(self.h, C.byref(cp)), "set_params")
        self.problem, self._cp = problem, cp

    def kernel_count(self) -> int:
        return self.lib.fmg_eig_kernel_count(self.h)

    def profile(self) -> dict:
        buf = (C.c_double * 10)()
        n = self.lib.fmg_eig_profile(self.h, buf, 10)
        if n < 0:
            raise FmgError(n, "profile")
        return {k: buf[i] for i, k in enumerate(self.PROFILE_KEYS[:n])}

    def _check(self, rc, what, allow=()):
        if rc != FMG_OK and rc not in allow:
            raise FmgError(rc, what)
        return rc

    # -- whole solve ---------------------------------------------------------------------
    def solve(self, u_host=None, stats: bool = False):
        lam = C.c_double()
        st = fmg_eig_stats() if stats else None
        n = 0 if u_host is None else int(u_host.size if hasattr(u_host, "size") and not callable(u_host.size) else u_host.numel())
        rc = self.lib.fmg_eig_solve(self.h, C.byref(lam), _ptr(u_host), n,
                                    C.byref(st) if st is not None else None)
        self._check(rc, "fmg_eig_solve", allow=(FMG_ENOCONV,))
        return lam.value, st, rc

    def solve_dev(self, lam_dev, u_dev=None, stream=None):
        n = 0 if u_dev is None else u_dev.numel()
        rc = self.lib.fmg_eig_solve_dev(self.h, _ptr(lam_dev), _ptr(u_dev), n, stream)
        return self._check(rc, "fmg_eig_solve_dev")

    # -- components ----------------------------------------------------------------------
    def apply_operator(self, k, x, y, stream=None):
        return self._check(self.lib.fmg_eig_apply_operator(self.h, k, _ptr(x), _ptr(y), stream), "apply_operator")

    def apply_mass(self, k, x, y, stream=None):
        return self._check(self.lib.fmg_eig_apply_mass(self.h, k, _ptr(x), _ptr(y), stream), "apply_mass")

    def jacobi(self, k, f, x_in, x_out, stream=None):
        return self._check(self.lib.fmg_eig_jacobi(self.h, k, _ptr(f), _ptr(x_in), _ptr(x_out), stream), "jacobi")

    def residual_restrict(self, k, f, x, rc, stream=None):
        return self._check(self.lib.fmg_eig_residual_restrict(self.h, k, _ptr(f), _ptr(x), _ptr(rc), stream), "residual_restrict")

    def prolong_add(self, k, ec, x, stream=None):
        return self._check(self.lib.fmg_eig_prolong_add(self.h, k, _ptr(ec), _ptr(x), stream), "prolong_add")

    def nonlinear_load(self, k, u, out, stream=None):
        return self._check(self.lib.fmg_eig_nonlinear_load(self.h, k, _ptr(u), _ptr(out), stream), "nonlinear_load")

    def aux_rhs(self, k, lam, u, f, stream=None):
        return self._check(self.lib.fmg_eig_aux_rhs(self.h, k, float(lam), _ptr(u), _ptr(f), stream), "aux_rhs")

    def multigrid(self, k, f, x, stream=None):
        return self._check(self.lib.fmg_eig_multigrid(self.h, k, _ptr(f), _ptr(x), stream), "multigrid")

    def correction(self, k, lam, u_in, u_out, u_tilde=None):
        lo = C.c_double()
        it = C.c_int32()
        rc = self.lib.fmg_eig_correction(self.h, k, float(lam), _ptr(u_in), C.byref(lo), _ptr(u_out),
                                         _ptr(u_tilde), C.byref(it))
        self._check(rc, "correction", allow=(FMG_ENOCONV,))
        return lo.value, it.value, rc

    def augmented_system(self, k, u_tilde, c):
        """(K, M, G(c)) of the augmented space V_H + span{u~} on level k, as numpy arrays."""
        import numpy as np
        c = np.ascontiguousarray(c, dtype=np.float64)
        n = c.size
        K, M, G = (np.empty((n, n)) for _ in range(3))
        rc = self.lib.fmg_eig_augmented_system(self.h, k, _ptr(u_tilde), _ptr(c), n, _ptr(K), _ptr(M), _ptr(G))
        self._check(rc, "augmented_system")
        return K, M, G

    def coarse_solve(self, u_out):
        lo = C.c_double()
        it = C.c_int32()
        rc = self.lib.fmg_eig_coarse_solve(self.h, C.byref(lo), _ptr(u_out), C.byref(it))
        self._check(rc, "coarse_solve", allow=(FMG_ENOCONV,))
        return lo.value, it.value, rc


def _batch_outputs(problems, with_u, stats):
    import numpy as np
    n = len(problems)
    lams = (C.c_double * n)()
    us = [np.empty(p.size(p.levels)) for p in problems] if with_u else None
    ptrs = (_P * n)(*[u.ctypes.data for u in us]) if with_u else None
    lens = (C.c_size_t * n)(*[u.size for u in us]) if with_u else None
    st = (fmg_eig_stats * n)() if stats else None
    codes = (_I32 * n)()
    return lams, us, ptrs, lens, st, codes


class BatchSolver(Solver):
    """A batch handle (fmg_eig_batch_create): instances that may differ in level count, W and
    zeta, solved by one CUDA graph with one launch per step and level for all of them."""

    def __init__(self, problems: list):
        self.lib = load_library()
        self.problems = list(problems)
        self.problem = self.problems[0]
        arr = (fmg_eig_problem * len(self.problems))(*[p.to_c() for p in self.problems])
        h = _P()
        rc = self.lib.fmg_eig_batch_create(arr, len(self.problems), C.byref(h))
        if rc != FMG_OK:
            raise FmgError(rc, "fmg_eig_batch_create")
        self.h = h

    def count(self) -> int:
        return self.lib.fmg_eig_batch_count(self.h)

    def solve_dev_all(self, lams_dev, stream=None):
        """fmg_eig_batch_solve_dev: lambdas into a device tensor, no host synchronisation."""
        return self._check(self.lib.fmg_eig_batch_solve_dev(self.h, _ptr(lams_dev), stream),
                           "fmg_eig_batch_solve_dev")

    def solve_all(self, with_u: bool = True, stats: bool = False, allow=()):
        """lambdas (list), u per instance (numpy, or None), stats records (or None), codes.
        Return codes in `allow` (besides FMG_ENOCONV) are reported in codes, not raised."""
        lams, us, ptrs, lens, st, codes = _batch_outputs(self.problems, with_u, stats)
        rc = self.lib.fmg_eig_batch_solve(self.h, lams, ptrs, lens, st, codes)
        self._check(rc, "fmg_eig_batch_solve", allow=(FMG_ENOCONV, *allow))
        return list(lams), us, (list(st) if stats else None), list(codes)


def solve_batch(problems: list, with_u: bool = True, stats: bool = False, allow=()):
    """fmg_eig_solve_batch: one-shot batch over problems of any mix of settings.  Return codes
    in `allow` (besides FMG_ENOCONV) are reported per instance in codes, not raised."""
    lib = load_library()
    arr = (fmg_eig_problem * len(problems))(*[p.to_c() for p in problems])
    lams, us, ptrs, lens, st, codes = _batch_outputs(problems, with_u, stats)
    rc = lib.fmg_eig_solve_batch(arr, len(problems), lams, ptrs, lens, st, codes)
    if rc not in (FMG_OK, FMG_ENOCONV, *allow):
        raise FmgError(rc, "fmg_eig_solve_batch")
    return list(lams), us, (list(st) if stats else None), list(codes)


def estimate_bytes(problems: list) -> int:
    """fmg_eig_estimate_bytes: device bytes of a batch handle for these problems."""
    arr = (fmg_eig_problem * len(problems))(*[p.to_c() for p in problems])
    return load_library().fmg_eig_estimate_bytes(arr, len(problems))


def serve(problems: list, arrivals: list, *, budget_bytes: float = 0.0, max_batch: int = 32,
          max_inflight: int = 4, batch_window_s: float = 0.0, with_u: bool = False, allow=()):
    """fmg_eig_serve over requests (problem, arrival time in s): per-request results as dicts
    (lambda, latency_s, admit_s, done_s, status, cohort, u) and the serve statistics.  Return
    codes in `allow` (besides FMG_ENOCONV) are left to the per-request statuses."""
    import numpy as np
    lib = load_library()
    n = len(problems)
    reqs = (fmg_eig_request * n)()
    us = []
    for i, (p, t) in enumerate(zip(problems, arrivals)):
        reqs[i].problem = p.to_c()
        reqs[i].arrival_s = float(t)
        if with_u:
            u = np.empty(p.size(p.levels))
            us.append(u)
            reqs[i].u = u.ctypes.data
            reqs[i].u_len = u.size
    cfg = fmg_eig_serve_config(float(budget_bytes), float(batch_window_s), int(max_batch),
                               int(max_inflight))
    res = (fmg_eig_result * n)()
    st = fmg_eig_serve_stats()
    rc = lib.fmg_eig_serve(C.byref(cfg), reqs, n, res, C.byref(st))
    if rc not in (FMG_OK, FMG_ENOCONV, *allow):
        raise FmgError(rc, "fmg_eig_serve")
    out = [{"lambda": r.lambda_, "latency_s": r.latency_s, "admit_s": r.admit_s,
            "done_s": r.done_s, "status": r.status, "cohort": r.cohort,
            "u": us[i] if with_u else None} for i, r in enumerate(res)]
    stats = {k: getattr(st, k) for k, _ in fmg_eig_serve_stats._fields_}
    return out, stats
