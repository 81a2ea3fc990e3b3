"""libgpa: forward passes and Accum-based reverse-mode gradients of pointful
array programs (Gaussian mixture with a Wishart prior; camera reprojection) on
NVIDIA B300 (sm_103a), with a C ABI (include/gpa.h) and this thin binding.

The CUDA library is loaded on first use; there is no CPU fallback.
"""
from . import _lib, data_parallel
from ._lib import (GpaError, PREC_BF16_TC, PREC_FP32, accum_scatter_add, gmm_jvp, gmm_objective, gmm_vjp,
                   gmm_vjp_finalize, gmm_vjp_host, gmm_vjp_partial, gpa_gmm_vjp_host_workspace_bytes, gpa_gmm_exchange_len, gpa_gmm_workspace_bytes, gpa_index_plan_build, gpa_obs_plan_build, gpa_plan_bytes,
                   gpa_plan_workspace_bytes, gpa_reproj_workspace_bytes, reproj_jvp, reproj_normal_eqs, reproj_residual,
                   reproj_residual_vjp, reproj_vjp, status_string, version)

__all__ = [
    "GpaError", "PREC_FP32", "PREC_BF16_TC", "accum_scatter_add", "data_parallel", "gmm_jvp", "gmm_objective", "gmm_vjp",
    "gmm_vjp_finalize", "gmm_vjp_host", "gmm_vjp_partial", "gpa_gmm_vjp_host_workspace_bytes", "gpa_gmm_exchange_len", "gpa_gmm_workspace_bytes", "gpa_index_plan_build", "gpa_obs_plan_build", "gpa_plan_bytes",
    "gpa_plan_workspace_bytes", "gpa_reproj_workspace_bytes", "reproj_jvp", "reproj_normal_eqs", "reproj_residual", "reproj_residual_vjp",
    "reproj_vjp", "status_string", "version",
]
