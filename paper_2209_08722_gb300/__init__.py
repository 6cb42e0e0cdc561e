"""GB300-native sketched inexact interior-point LP solver (arXiv 2209.08722).

The solver is a CUDA library (``_lib/liblpsketch.so``, C ABI in
``include/lp_sketch_ipm.h``) built for sm_103a; this package is its thin
Python front-end.  Importing ``LPSolver`` loads the library and raises
ImportError if it has not been built -- there is no CPU fallback.
"""

from .build_native import build, lib_path  # noqa: F401


def __getattr__(name):
    if name in ("LPSolver", "LPError", "from_planted", "phase1_start", "solve_batch", "Mlp", "csr_to_csc",
                "release_cached_memory"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
