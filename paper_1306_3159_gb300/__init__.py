"""GB300-native solver for the minimally-resolved reactive-blob model.

Python binding of ``libibrd`` (C ABI in ``include/ibrd.h``). The functions
below marshal arguments only: every arithmetic step runs in the library's CUDA
kernels. Fields and blob arrays are CUDA ``torch`` tensors (FP64, contiguous);
their device pointers and the current torch stream are passed to the library.
Importing this package does not need a GPU; calling into it does, and a
missing or unloadable library raises ``ImportError``/``RuntimeError``: there is
no CPU fallback.

Single solves: ``Grid`` (or ``ibrd_solve_reaction`` / ``ibrd_solve_saddle``);
many independent solves on their own handles and streams:
``ibrd_solve_reaction_batch``, ``ibrd_solve_saddle_batch``, ``ibrd_solve_many``;
launch-shape tuning: ``ibrd_autotune``; the learned multiplier predictor:
``GNN``.
"""
from ._abi import (
    EXPORTED, GNN, IBRD_FP64, IBRD_GUESS_GIVEN, IBRD_GUESS_NONE, IBRD_GUESS_PENALTY, IBRD_GUESS_UNIFORM,
    IBRD_MIXED_FP32, IBRD_MIXED_REFINE, IBRD_PESKIN3, IBRD_PESKIN4, IBRD_PRECOND_AUTO, IBRD_PRECOND_BLOCK, IBRD_PRECOND_DIAG,
    IBRD_PRECOND_SCHUR,
    Grid, IbrdError, SolveOpts, ibrd_apply_L, ibrd_autotune, ibrd_default_opts, ibrd_gnn_num_params,
    ibrd_grid_create, ibrd_grid_destroy, ibrd_interp, ibrd_last_error, ibrd_profile_enable, ibrd_profile_read,
    ibrd_periodic_constant, ibrd_residual, ibrd_set_blobs, ibrd_solve_many, ibrd_solve_reaction, ibrd_solve_reaction_batch, ibrd_solve_saddle,
    ibrd_solve_saddle_batch, ibrd_spread, ibrd_set_wait_limit, ibrd_tune_clear, ibrd_tune_set, ibrd_vcycle,
    ibrd_vcycle_f32, ibrd_vcycle_f32_sweeps,
    load_library)

__all__ = [
    "EXPORTED", "GNN", "IBRD_FP64", "IBRD_GUESS_GIVEN", "IBRD_GUESS_NONE", "IBRD_GUESS_PENALTY",
    "IBRD_GUESS_UNIFORM", "IBRD_MIXED_FP32", "IBRD_MIXED_REFINE", "IBRD_PESKIN3", "IBRD_PESKIN4",
    "IBRD_PRECOND_AUTO", "IBRD_PRECOND_BLOCK", "IBRD_PRECOND_DIAG", "IBRD_PRECOND_SCHUR", "Grid", "IbrdError", "SolveOpts", "ibrd_apply_L",
    "ibrd_autotune", "ibrd_default_opts", "ibrd_gnn_num_params", "ibrd_grid_create", "ibrd_grid_destroy",
    "ibrd_interp", "ibrd_last_error", "ibrd_profile_enable", "ibrd_profile_read", "ibrd_periodic_constant", "ibrd_residual", "ibrd_set_blobs",
    "ibrd_solve_many", "ibrd_solve_reaction", "ibrd_solve_reaction_batch", "ibrd_solve_saddle",
    "ibrd_solve_saddle_batch", "ibrd_spread", "ibrd_set_wait_limit", "ibrd_tune_clear", "ibrd_tune_set", "ibrd_vcycle",
    "ibrd_vcycle_f32", "ibrd_vcycle_f32_sweeps", "load_library",
]
