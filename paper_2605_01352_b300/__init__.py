"""Co-scheduled simulate-then-render for batched embodied-AI environments on B300.

The compute path lives in the CUDA library ``libvuda.so`` (C-ABI in
``include/vuda.h``); ``paper_2605_01352_b300.vuda`` is its thin ctypes
binding and ``paper_2605_01352_b300.scene`` builds seeded inputs.  Importing
the package itself loads nothing, so the input generator can be used on a
machine without the library.
"""
__all__ = ["scene", "vuda"]
