"""GB300-native differentiable evolution of superconducting circuits.

The compute path is libsupergpu.so (CUDA for sm_103a, C ABI in include/sg.h);
this package is its thin Python binding.  Importing the package does not load
the library; the first call does, and raises if it has not been built.
"""
import os as _os

# Concurrent solves run on one stream each (the server's slots).  With the CUDA
# default of 8 hardware work queues, two streams share a queue and a kernel waiting
# on its own stream holds back the other stream's launches; 32 queues give every
# slot its own.  Takes effect only if set before the process creates its CUDA
# context, so import this package before initialising CUDA; a value already set is
# kept.
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")


def __getattr__(name):
    if name in ("Context", "System", "evolve_opts", "workload_fidelity"):
        from . import api
        return getattr(api, name)
    if name == "FidelityFn":
        from .autograd import FidelityFn
        return FidelityFn
    raise AttributeError(name)
