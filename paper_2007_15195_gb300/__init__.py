"""GB300-native Vecchia approximation to high-dimensional Gaussian CDFs.

Hot path of Nascimento & Shaby (arXiv 2007.15195) as hand-written CUDA for
sm_103a behind the C ABI in include/vecchia.h; this package is its Python
binding (``binding``), seeded workload generators (``inputs``), the
continuous-batching request loop (``serve``) and the tile autotuner
(``autotune``).  Importing the package does not load the library; the first
call does, and fails if it has not been built.
"""
from .binding import (COND_NEAREST, COND_RANDOM, COV_ANISO_EXP, COV_EXPONENTIAL, COV_MATERN, FP64, MIXED,
                      ORDER_IDENTITY, ORDER_MAXMIN, ORDER_XY, Context, Plan, VecchiaError, make_cov,
                      vecchia_censored_log_cdf, vecchia_create, vecchia_destroy, vecchia_apply_order, vecchia_full_genz,
                      vecchia_genz_time_ms,
                      vecchia_group_conditioning, vecchia_grouped_log_cdf, vecchia_last_error_site,
                      vecchia_lattice, vecchia_log_cdf, vecchia_log_cdf_batch, vecchia_log_cdf_terms,
                      vecchia_log_cdf_unordered,
                      vecchia_mixture_log_cdf, vecchia_neighbors, vecchia_order, vecchia_plan_create,
                      vecchia_reset_tiles, vecchia_set_tile, vecchia_set_timing, vecchia_shifts)

__all__ = [
    "COND_NEAREST", "COND_RANDOM", "COV_ANISO_EXP", "COV_EXPONENTIAL", "COV_MATERN", "FP64", "MIXED",
    "ORDER_IDENTITY", "ORDER_MAXMIN", "ORDER_XY", "Context", "Plan", "VecchiaError", "vecchia_plan_create",
    "make_cov", "vecchia_censored_log_cdf", "vecchia_create", "vecchia_destroy", "vecchia_apply_order", "vecchia_full_genz",
    "vecchia_genz_time_ms",
    "vecchia_group_conditioning", "vecchia_grouped_log_cdf", "vecchia_last_error_site", "vecchia_lattice",
    "vecchia_log_cdf", "vecchia_log_cdf_batch", "vecchia_log_cdf_terms", "vecchia_log_cdf_unordered", "vecchia_mixture_log_cdf",
    "vecchia_neighbors", "vecchia_order", "vecchia_reset_tiles", "vecchia_set_tile", "vecchia_set_timing",
    "vecchia_shifts",
]
