"""GB300-native Householder-aligned permutation test (Ehara, ACL 2026).

The compute path is libhbperm.so (hand-written sm_103a CUDA behind the C ABI
in include/hbperm.h); this package is its thin Python binding plus the seeded
synthetic-cloud generator used by the benchmark.
"""
from .hbperm import (  # noqa: F401
    HB_ALT_GREATER, HB_ALT_LESS, HB_ALT_TWO_SIDED, HB_BF16, HB_ERR_CUDA, HB_ERR_DEGENERATE, HB_ERR_INVALID_ARG,
    HB_ERR_OOM, HB_ERR_TIMEOUT, HB_ERR_UNSUPPORTED, HB_F32, HB_OK, HB_PATH_FP32_PLAIN, HB_PATH_MIXED,
    HB_STAT_LOGVOL_VMF, HB_STAT_MEAN_COSDIST, HB_STAT_ONE_MINUS_R2, Context, HbError, hb_align, hb_perm_labels,
    hb_perm_test, hb_perm_test_batched, make_opts,
)
