"""GB300-native batched shared-LHS tridiagonal/pentadiagonal solver
(arXiv:1909.04539).  The compute path is the CUDA library ``libbsolve.so``
behind the C ABI in ``include/bsolve.h``; this package only marshals torch
tensors into it."""
from .api import (ADIHalfStepFn, Factor, SolveFn, adi_halfstep, band_grad, cn_steps, solve, solve_adjoint, solve_bf16, solve_refine,  # noqa: F401
                  set_option, lhs_bytes, measure_fp64_rate, device_status,
                  OPT_INFLIGHT_BYTES, OPT_BLOCKS_PER_SM, OPT_SWEEP_KERNEL, OPT_TMA_AHEAD, OPT_PARTITION, OPT_UNIFORM, OPT_TWISTED,
                  OPT_CTA_THREADS, OPT_F64_PAIRS, OPT_WINDOW,
                  REFINE_FACTOR, REFINE_SYSTEM, REFINE_AUTO)
from ._lib import BsolveError  # noqa: F401
