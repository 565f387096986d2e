"""GB300-native H^2-ULV dense solver (Ma & Yokota, arXiv 2502.02395).

The computation lives in the C-ABI library ``libh2ulv.so`` (CUDA for sm_103a,
see ``include/h2ulv.h``); ``binding`` is a thin ctypes layer over it.
"""
from .binding import (H2Error, H2Solver, h2_build, h2_destroy, h2_export, h2_factor, h2_import,  # noqa: F401
                      h2_last_error, h2_matvec, h2_matvec_arith, h2_matvec_noalloc, h2_set_memory_limit, h2_set_option,
                      h2_wait_selftest, h2_plan, h2_set_refinement, h2_set_stream, h2_solve, h2_stats, h2_ulv_apply, lib,
                      make_params, H2Batch, h2_build_forest, h2_tree_depth)
