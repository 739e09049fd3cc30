"""GB300-native (sm_103a) sparse MTTKRP along every mode of a small N-mode
COO tensor, and CP-ALS on top of it.

The computation lives in hand-written CUDA kernels behind the C ABI of
``include/spmttkrp.h`` (library ``_lib/libspmttkrp.so``); :mod:`.binding` is
a thin ctypes layer over it that takes PyTorch CUDA tensors and streams.
"""
from .binding import (SPM_FACTOR_BF16, SPM_FACTOR_FP32, SPM_KAPPA,  # noqa: F401
                      SPM_POLICY_ADAPTIVE, SPM_POLICY_BALANCED,
                      SPM_PLAN_FIBRE, SPM_PLAN_LEAN, SPM_POLICY_SCHEME1, SPM_POLICY_SCHEME2, SPM_ROW_COST,
                      SPM_UNITS_PER_PARTITION, Batch, Plan, Server, SpmError, cpd_als_reset,
                      cpd_als_step,
                      load, spm_batch_autotune, spm_batch_create, spm_batch_destroy, spm_batch_status,
                      spm_batch_sweep,
                      spm_device_sm_count, spm_selftest_tc_rowpass, spm_status_string, spmttkrp_plan,
                      spmttkrp_plan_bytes, spmttkrp_plan_bytes_estimate,
                      spmttkrp_plan_destroy, spmttkrp_plan_fibre_count,
                      spmttkrp_plan_partition, spmttkrp_plan_permutation,
                      spmttkrp_plan_autotune, spmttkrp_plan_repartition,
                      spmttkrp_plan_scheme,
                      spmttkrp_plan_status,
                      spmttkrp_plan_work_units, spmttkrp_run, spmttkrp_run_all_host,
                      spmttkrp_run_noalloc)
