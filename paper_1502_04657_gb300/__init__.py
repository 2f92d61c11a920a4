"""GB300-native full multigrid solver for the Gross-Pitaevskii ground state.

The compute path is the C-ABI library ``libfmg_eig.so`` (hand-written sm_103a CUDA kernels);
``paper_1502_04657_gb300.fmg`` is its thin ctypes binding."""
from .fmg import FmgError, Problem, Solver, load_library  # noqa: F401
