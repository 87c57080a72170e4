"""GB300 (sm_103a) implementation of the FastTuckerPlus stochastic epoch
(arXiv 2404.10087).

Submodules:
  ft      ctypes binding of the C ABI in include/ft.h (the CUDA library)
  synth   seeded synthetic workloads (draws only, no method arithmetic)
  _build  nvcc build of the in-tree library
"""
__all__ = ["ft", "synth"]


def __getattr__(name):
    if name in ("ft", "synth", "_build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
