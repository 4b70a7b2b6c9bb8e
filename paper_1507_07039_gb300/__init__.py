"""PANDA message passing on one GB300: C-ABI CUDA library plus a thin binding.

``panda`` (the ctypes binding over ``libpanda_gb300.so``) is imported on
demand so that ``synth`` stays usable without the CUDA library.
"""
__all__ = ["synth", "panda"]
