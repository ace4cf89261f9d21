"""GB300-native fast directional Burton-Miller BEM (Cao, Wen, Xiao).

The compute path is the CUDA library libfdabem.so (C ABI in
include/fda_bem.h); this package is its Python binding.  `FDAProblem` is a
convenience wrapper that takes torch CUDA tensors for vectors.
"""
from ._lib import (FDA_OK, FDA_ERR_ARG, FDA_ERR_STATE, FDA_ERR_CUDA, FDA_ERR_OOM, FDA_ERR_NOT_CONVERGED,
                   FDA_ERR_TIMEOUT, FDA_ERR_NUMERIC, FDA_PLAIN_FP64, FDA_CHOSEN_FP32, FDA_MODE_FDA, FDA_MODE_DENSE,
                   FDAError, fda_config, fda_info, fda_stats, load, fda_default_config, fda_create, fda_build_tree,
                   fda_precompute_translations, fda_apply, fda_apply_host, fda_rhs_plane_wave,
                   fda_rhs_plane_wave_noalloc, fda_rhs_neumann, fda_rhs_point_source, fda_far_field, fda_far_field_fast, fda_scattered_field, fda_scattered_field_fast,
                   fda_solve,
                   fda_get_stats, fda_set_precision, fda_set_precond, fda_set_tensor_cores, fda_set_tc_tiles, fda_get_tree,
                   fda_set_timing, fda_get_pass_times, fda_cone_symmetry_table, fda_launch_count,
                   fda_sai_config, fda_sai_report, fda_sai_num_params, fda_sai_default_config,
                   fda_sai_init_weights, fda_sai_train, fda_sai_set, fda_sai_loss_grad,
                   fda_sai_set_pattern, fda_sai_loss_grad_near, fda_last_error, fda_destroy,
                   fda_batch_stats, fda_create_batch, fda_build_batch, fda_precompute_batch, fda_apply_batch,
                   fda_batch_mesh, fda_get_batch_stats, fda_batch_last_error, fda_destroy_batch)
from .problem import FDAProblem, FDABatch

__all__ = ["FDA_OK", "FDA_ERR_ARG", "FDA_ERR_STATE", "FDA_ERR_CUDA", "FDA_ERR_OOM", "FDA_ERR_NOT_CONVERGED",
           "FDA_ERR_TIMEOUT", "FDA_ERR_NUMERIC", "FDA_PLAIN_FP64", "FDA_CHOSEN_FP32", "FDA_MODE_FDA",
           "FDA_MODE_DENSE", "FDAError", "fda_config", "fda_info", "fda_stats", "load", "fda_default_config",
           "fda_create", "fda_build_tree", "fda_precompute_translations", "fda_apply", "fda_apply_host",
           "fda_rhs_plane_wave", "fda_rhs_plane_wave_noalloc", "fda_rhs_neumann", "fda_rhs_point_source", "fda_far_field", "fda_far_field_fast",
           "fda_scattered_field", "fda_scattered_field_fast", "fda_solve", "fda_get_stats", "fda_set_precision", "fda_set_precond", "fda_set_tensor_cores", "fda_set_tc_tiles", "fda_get_tree", "fda_set_timing", "fda_get_pass_times",
           "fda_cone_symmetry_table", "fda_launch_count", "fda_sai_config", "fda_sai_report", "fda_sai_num_params",
           "fda_sai_default_config", "fda_sai_init_weights", "fda_sai_train", "fda_sai_set", "fda_sai_loss_grad", "fda_sai_set_pattern", "fda_sai_loss_grad_near",
           "fda_last_error", "fda_destroy", "fda_batch_stats", "fda_create_batch", "fda_build_batch",
           "fda_precompute_batch", "fda_apply_batch", "fda_batch_mesh", "fda_get_batch_stats", "fda_batch_last_error",
           "fda_destroy_batch", "FDAProblem", "FDABatch"]
