"""GB300-native SSPRK2-SE / SSPRK3-SE multirate split-explicit time stepping.

The compute path lives in ``libsse.so`` (CUDA, sm_103a) behind the C ABI
declared in ``include/sse.h``; ``binding`` is its thin ctypes binding.
``mesh`` and ``inputs`` generate seeded synthetic meshes and states.
Submodules are imported on demand so that the input generators can be used
without loading the CUDA library.
"""
__all__ = ["mesh", "inputs", "binding"]
