"""GB300-native sketched flexible LSQR / LSMR (sFLSQR, sFLSMR).

The solvers of "Randomized Flexible LSQR and LSMR with applications to inverse
problems" (Algorithms 1 and 2) as hand-written sm_103a CUDA behind a C ABI
(include/sfl.h, libsfl.so), with this thin Python binding.  There is no CPU
path: every call needs the CUDA library and a GPU.
"""
from .builder import build  # noqa: F401

__all__ = ["build", "Plan", "sflsqr", "sflsmr", "sketch_export", "sketch_apply", "SolveInfo"]


def __getattr__(name):
    if name in ("Plan", "sflsqr", "sflsmr", "sketch_export", "sketch_apply", "SolveInfo"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
