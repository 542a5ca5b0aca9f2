"""GB300-native feasible-triplet sweep for lower bounds on the Chvatal-Sankoff
constants (Heineman et al., arXiv 2407.10925).

The product is the CUDA library built from ``csrc/`` behind the C ABI in
``include/lcs_bound.h``; ``binding`` is its thin ctypes binding.
"""
from .binding import (  # noqa: F401
    LcsBatch,
    LcsBound,
    LcsError,
    LcsMlp,
    lcs_bound_batch_create,
    lcs_bound_batch_export_fx,
    lcs_bound_batch_info,
    lcs_bound_batch_read,
    lcs_bound_batch_report,
    lcs_bound_batch_set_mode,
    lcs_bound_batch_set_spin_budget,
    lcs_bound_check_vector,
    lcs_bound_create,
    lcs_bound_default_opts,
    lcs_bound_destroy,
    lcs_bound_errstr,
    lcs_bound_export,
    lcs_bound_export_fx,
    lcs_bound_iterate,
    lcs_bound_last_error,
    lcs_bound_read,
    lcs_bound_read_report,
    lcs_bound_set_start,
    lcs_bound_set_start_fx,
    lcs_bound_size,
    lcs_bound_stats,
    lcs_bound_synchronize,
    lcs_fp32_experiment,
    lcs_lift_prefix,
    lcs_sweep_fx,
    lcs_sweep_incr_fx_noalloc,
    lib,
)
