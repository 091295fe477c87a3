"""GB300-native differentiable evolution of superconducting circuits.

The compute path is libsupergpu.so (CUDA for sm_103a, C ABI in include/sg.h);
this package is its thin Python binding.  Importing the package does not load
the library; the first call does, and raises if it has not been built.
"""


def __getattr__(name):
    if name in ("Context", "System", "evolve_opts", "workload_fidelity"):
        from . import api
        return getattr(api, name)
    if name == "FidelityFn":
        from .autograd import FidelityFn
        return FidelityFn
    raise AttributeError(name)
