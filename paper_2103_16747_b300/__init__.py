"""B300-native quasi-static tet-FEM indentation solver (hot path of the
fingertip FEM of arXiv 2103.16747, Sec. III-A), behind the C ABI in
include/fem.h. ``_lib`` is the ctypes binding; ``solver`` adds a small
convenience layer that only marshals workload objects into C-ABI calls."""
from . import _lib  # noqa: F401  (raises ImportError if the CUDA library is missing)
from ._lib import *  # noqa: F401,F403
from .solver import IndentationSolver, solve_indentation  # noqa: F401
