"""GB300 (sm_103a) hot path of the ROM-accelerated minimum-compliance SIMP method
(Yano, Huang and Zahr, arXiv 2004.05756): libtopo.so (C ABI, include/topo.h) and its thin
Python binding.

Submodules are imported lazily so that the seeded input generators (workloads) can be used
without loading the CUDA library.
"""
import importlib

__all__ = ["workloads", "native", "build", "serving", "profcase"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
