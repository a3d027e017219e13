"""GB300-native Fast Cauchy Transform ℓ1 regression (FastCauchyRegression, Figure 2).

The compute path is libl1fct.so (CUDA for sm_103a, built in-tree by
`paper_1207_4684_gb300.build`); `paper_1207_4684_gb300.l1fct` is its ctypes
binding.  PyTorch provides device memory and streams only.
"""
from .l1fct import (  # noqa: F401
    BF16,
    EXPORTS,
    F32,
    L1SError,
    Params,
    Problem,
    Schedule,
    batched_workspace,
    fct_embed,
    flag,
    l1_coreset,
    l1_coreset_host,
    l1_condition,
    l1_lambda,
    l1_lambda_noalloc,
    l1_objective,
    l1_regress,
    l1_regress_batched,
    l1_sample,
    l1_sample_from_p,
    l1_solve,
    l1s_debug_pi2,
    l1s_autotune,
    l1s_batched_workspace_size,
    l1s_debug_variates,
    l1s_kernel_launches,
    l1s_schedule_get,
    l1s_schedule_set,
    l1s_status_read,
    l1s_status_reset,
    l1s_workspace_size,
    load,
    make_params,
    make_problem,
    version,
    workspace,
)
