"""GB300-native ripALM minimum-enclosing-ball hot path (arxiv 2605.31425).

``solve``, ``eval_alm`` and ``feas_check`` call the C ABI of libmeb
(include/meb.h), whose kernels are hand-written CUDA for sm_103a.
``workloads`` holds the seeded input generators (importing it does not load
the CUDA library).
"""
_API = ("MEB_PTR_DEVICE", "Context", "MebError", "MebInfo", "MebParams", "default_context",
        "eval_alm", "feas_check", "feas_check_noalloc", "load", "params_default", "solve", "stats", "reset_stats",
        "solve_batch", "tune_batch", "MEB_ETIMEOUT", "MEB_ENOTCONV", "MEB_EINVAL", "Server",
        "footprint")


def __getattr__(name):
    if name in _API:
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
