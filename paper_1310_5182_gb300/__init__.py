"""GB300 (sm_103a) library for local approximate Gaussian process regression
with greedy ALC local designs (Gramacy, Niemi & Weiss, arXiv:1310.5182).

The compute path is liblagp.so (hand-written CUDA kernels behind the C ABI of
include/lagp.h); this package is its thin Python binding.  Importing the
binding requires the built library: there is no CPU fallback.
"""
from .lagp import (  # noqa: F401
    LagpError,
    context,
    get_tuning,
    lagp_agp,
    lagp_alc_select,
    lagp_knn,
    lagp_mle_step,
    lagp_predict,
    lagp_predict_grad,
    launch_count,
    library,
    set_tuning,
)
