"""GB300 (sm_103a) implicit immersed-boundary multigrid.

The compute path is ``libibmg.so`` (hand-written CUDA behind the C ABI of
``include/ib.h``); this package is its ctypes binding.  Build it with
``__graft_entry__.build()`` or ``python -m paper_1311_5614_gb300.build``.
"""
from .capi import (KERNEL_CLASSES, UNet, ib_unet_num_params, IBBatch, IBError, IBSolver, ib_setup_batch, ib_solve_step_batch, ib_apply, ib_launch_count, ib_profile,
                   ib_profile_read, ib_default_params, ib_destroy, ib_last_error,
                   ib_level_size, ib_num_levels, ib_num_struct_boxes, ib_rhs, ib_setup,
                   ib_solve_step, ib_update_points, ib_vcycle, ib_version, lib, make_params)

__all__ = ["UNet", "ib_unet_num_params", "IBBatch", "ib_setup_batch", "ib_solve_step_batch", "KERNEL_CLASSES", "ib_launch_count", "ib_profile", "ib_profile_read", "IBError", "IBSolver", "ib_apply", "ib_default_params", "ib_destroy", "ib_last_error",
           "ib_level_size", "ib_num_levels", "ib_num_struct_boxes", "ib_rhs", "ib_setup",
           "ib_solve_step", "ib_update_points", "ib_vcycle", "ib_version", "lib", "make_params"]
