"""GB300 (sm_103a) hybrid demagnetization-field library.

The compute path is ``libdemag.so`` (CUDA kernels behind the C ABI of
``include/demag.h``); this package holds its build script, its ctypes binding
(``_lib``) and the seeded input generators (``inputs``).
"""
from ._lib import (DemagError, Plan, PREC_FP32, PREC_FP64, PREC_SPLIT_BF16, PREC_SPLIT_TF32, demag_apply, demag_apply_adjoint,
                   demag_apply_dthickness, demag_apply_host, demag_apply_host_async, demag_apply_host_wait,
                   demag_apply_static, demag_apply_timed,
                   demag_destroy, demag_last_error, demag_layer_mean, demag_mlp_adam,
                   demag_mlp_backward, demag_mlp_forward, demag_mlp_mse, demag_mlp_param_count, demag_plan_create, demag_plan_create_equidistant, demag_plan_info,
                   demag_relax_layer,
                   demag_plan_compress, demag_plan_keep_slab, demag_plan_set_path, demag_rows_forward,
                   demag_columns_slab, demag_rows_inverse, demag_plan_tensor, demag_status_string,
                   demag_tensor_points,
                   demag_tensor_points_dt, demag_thickness_grad, demag_wait_timeouts,
                   demag_selftest_bounded_wait, demag_debug_fail_alloc, lib, library_path)

__all__ = ["DemagError", "Plan", "PREC_FP32", "PREC_FP64", "PREC_SPLIT_BF16", "PREC_SPLIT_TF32", "demag_apply", "demag_apply_adjoint",
           "demag_apply_dthickness", "demag_plan_compress", "demag_plan_keep_slab", "demag_rows_forward",
           "demag_columns_slab", "demag_rows_inverse", "demag_plan_set_path", "demag_tensor_points_dt",
           "demag_thickness_grad", "demag_apply_host", "demag_apply_host_async", "demag_apply_host_wait",
           "demag_apply_static", "demag_apply_timed", "demag_destroy", "demag_layer_mean",
           "demag_mlp_adam", "demag_mlp_backward", "demag_mlp_forward", "demag_mlp_mse",
           "demag_mlp_param_count", "demag_last_error",
           "demag_plan_create", "demag_plan_create_equidistant", "demag_plan_info", "demag_relax_layer", "demag_plan_tensor", "demag_status_string",
           "demag_tensor_points", "demag_wait_timeouts", "demag_selftest_bounded_wait",
           "demag_debug_fail_alloc", "lib", "library_path"]
