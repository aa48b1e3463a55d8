"""GB300 (sm_103a) LoRADS hot path: C-ABI CUDA library + thin Python binding.

The compute path is ``liblorads.so`` (built by ``builder.py`` from ``csrc/``);
``_native`` only marshals arguments.  Importing this package does not load the
library; the first call does, and fails loudly when it is missing.
"""
from . import _native
from ._native import (  # noqa: F401
    LoradsError, default_params, lorads_create, lorads_destroy, lorads_spmm, lorads_constraint_eval,
    lorads_linesearch_coeffs, lorads_solve, lorads_get_solution, lorads_problem_info, padded_ld,
    lorads_kernel_times, lorads_dual_min_eig, lorads_admm_operator, lorads_admm_cg, lorads_admm_stage,
    lorads_batch_create, lorads_batch_solve, lorads_batch_tune, lorads_batch_set_shape,
    lorads_batch_get_solution, lorads_batch_destroy, lorads_batch_phase_times,
    lorads_gnn_param_count, lorads_gnn_create, lorads_gnn_get_params, lorads_gnn_set_params, lorads_gnn_predict,
    lorads_gnn_edge_targets, lorads_gnn_train_step, lorads_gnn_destroy,
    LORADS_FP64, LORADS_FP32, LORADS_BF16, LORADS_MIXED, LORADS_DF64, LORADS_MIXED_BF16, load, SIGNATURES,
)

__all__ = [
    "LoradsError", "default_params", "lorads_create", "lorads_destroy", "lorads_spmm",
    "lorads_constraint_eval", "lorads_linesearch_coeffs", "lorads_solve", "lorads_get_solution",
    "lorads_problem_info", "padded_ld", "load", "build", "lorads_kernel_times", "lorads_dual_min_eig",
    "lorads_batch_create", "lorads_batch_solve", "lorads_batch_tune", "lorads_batch_set_shape",
    "lorads_batch_get_solution", "lorads_batch_destroy", "lorads_admm_operator", "lorads_admm_cg",
    "lorads_admm_stage",
]


def build(verbose: bool = False):
    from .builder import build as _b
    return _b(verbose=verbose)
