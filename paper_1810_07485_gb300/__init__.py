"""GB300 (sm_103a) continuous-time loop-cluster QMC update of the
antiferromagnetic Heisenberg chain (Todo, Matsuo, Shitara, arXiv:1810.07485).

The compute path is liblcqmc.so (CUDA kernels behind the C ABI of
include/lcqmc.h); lcqmc.py is a thin ctypes binding of it.
"""
from .build import build as build_library  # noqa: F401


def __getattr__(name):
    if name in ("Chain", "Batch", "Server", "lib", "LcqmcError", "u128", "RECORD_DTYPE", "PHASES"):
        from . import lcqmc
        return getattr(lcqmc, name)
    raise AttributeError(name)
