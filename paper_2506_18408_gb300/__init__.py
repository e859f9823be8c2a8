"""GB300-native sketched FGMRES: FGMRES wrapped around sketched-GMRES cycles, in hand-written sm_103a CUDA.

The compute path is the C-ABI library ``_lib/libsfgmres.so`` (declared in ``include/sfgmres.h``); this package is
its Python binding.  Build the library with ``paper_2506_18408_gb300.build.build()``.
"""
from .sfgmres import (  # noqa: F401
    BREAKDOWN, NOT_CONVERGED, OK, SFGMRESError, Solver, Stats, load, sfgmres_create, sfgmres_destroy,
    sfgmres_get_option, sfgmres_inner_cycle, sfgmres_set_option, sfgmres_sketch_apply, sfgmres_sketch_apply_noalloc, sfgmres_sketch_pattern,
    sfgmres_solve, sfgmres_solve_transpose, sfgmres_update_values, sfgmres_pattern_outer, sfgmres_spmv,
    sfgmres_version,
)
from .autograd import SFGMRESSolve, sfgmres_solve_autograd  # noqa: F401
