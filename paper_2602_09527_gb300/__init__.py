"""GB300-native (sm_103a) variance-reduced ProxSkip for tomography (arXiv 2602.09527).

The compute path is the CUDA library ``_lib/libvrps.so`` (C ABI in ``include/vrps.h``);
this package is its thin ctypes binding.  Entry points keep the C names without the
``vrps_`` prefix: ``proj_fwd``, ``proj_adj``, ``prox_tv``, ``solve``, ``power_iteration``,
``objective``, ``philox_schedule``, the ``Geometry`` handle and the ``Batch`` of jobs
(``vrps_batch_*``).
"""
from ._binding import (ALGOS, ESTIMATORS, Batch, autotune, check_error, Geometry, Report, SolveOpts, VrpsError, job_footprint,
                       kernel_launches, lib, objective, pdhg, philox_schedule, power_iteration, profile_enable,
                       profile_read, prox_tv, prox_tv2d_noalloc, proj_adj, proj_fwd, set_launch_shape, launch_shape,
                       launch_shape_full, selftest_bounded_wait, solve)

__all__ = ["ALGOS", "ESTIMATORS", "Batch", "autotune", "check_error", "Geometry", "job_footprint", "Report", "SolveOpts", "VrpsError", "kernel_launches", "lib",
           "objective", "pdhg", "philox_schedule", "power_iteration", "profile_enable", "profile_read", "prox_tv",
           "prox_tv2d_noalloc", "proj_adj", "proj_fwd", "set_launch_shape", "launch_shape", "launch_shape_full",
           "selftest_bounded_wait", "solve"]
