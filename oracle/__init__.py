"""CPU FP64 oracle for the ripALM minimum-enclosing-ball method (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    OracleParams,
    build,
    eval_alm,
    feas_check,
    kkt,
    params_default,
    set_threads,
    soc_dist,
    soc_jacobian,
    soc_project,
    solve,
)
