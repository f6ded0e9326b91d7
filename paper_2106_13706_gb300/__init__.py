"""GB300-native exact ddKS distance (arXiv 2106.13706).

The statistic, the permutation test, the analytic significance, batched and
served distances, and the vdKS / rdKS approximations all run in the CUDA
kernels of libddks.so (C ABI in
include/ddks.h); this package is the thin Python binding over it.
"""
from .binding import (  # noqa: F401
    Context, DdksError, DDKS_F32, DDKS_F64, DDKS_OK, DDKS_PENDING, MAX_D, PATH_AUTO, PATH_DOMINANCE, PATH_LANE,
    PATH_REGISTER, PATH_SORT, PATH_WARP, PATH_BYTE, ddks_autotune, ddks_batch_distance, ddks_ctx_create, ddks_ctx_destroy,
    ddks_ctx_stats, ddks_distance, ddks_distance_noalloc, ddks_distance_range, ddks_permutation_test, ddks_poll,
    ddks_rdks, ddks_rescale, ddks_significance, ddks_strerror, ddks_submit, ddks_vdks, ddks_version,
    declared_symbols, load,
    RDKS_MAX_D, VDKS_MAX_D,
)
