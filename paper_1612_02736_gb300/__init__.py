"""GB300 (sm_103a) implementation of the hierarchical direct solver for variable-coefficient
2D elliptic problems with body loads (Babb, Gillman, Hao, Martinsson, arXiv 1612.02736).

The native library ``libhps_gb300.so`` (C ABI: include/hps.h) does all the work; this
package only marshals arguments.  Build it with ``python -m paper_1612_02736_gb300.build``.
"""
from ._native import HPSError, load  # noqa: F401


def __getattr__(name):
    # torch-dependent wrappers are imported lazily
    if name in ("Tree", "Solver", "HPSFunction"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
