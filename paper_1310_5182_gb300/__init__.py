"""GB300 (sm_103a) library for local approximate Gaussian process regression
with greedy ALC local designs (Gramacy, Niemi & Weiss, arXiv:1310.5182).

The compute path is liblagp.so (hand-written CUDA kernels behind the C ABI of
include/lagp.h); the binding in .lagp marshals arguments to it.  The binding
is loaded on first use of any of its names, and raises ImportError if the
library has not been built: there is no CPU fallback.  The build module
(paper_1310_5182_gb300.build) imports without the library.
"""
_BINDING = ("LagpError", "context", "get_tuning", "lagp_agp", "lagp_alc_predict", "lagp_alc_select",
            "lagp_knn", "lagp_autotune", "lagp_alc_eval", "lagp_scale_inputs",
            "lagp_mle_step", "lagp_predict", "lagp_predict_grad", "lagp_predict_noalloc",
            "launch_count", "library", "alc_work", "mle_work", "exp64_check", "df_check", "lagp_knn_tc_dist", "knn_stats", "knn_tc_stall",
            "set_tuning")

__all__ = list(_BINDING)


def __getattr__(name):
    if name in _BINDING:
        from . import lagp
        return getattr(lagp, name)
    if name in ("local_gp", "local_loglik", "LocalGP", "LocalLogLik"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
