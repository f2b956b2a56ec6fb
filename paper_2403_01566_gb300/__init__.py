"""GB300-native adaptive H^2-matrix multiplication with block-relative error control.

The compute path lives in the CUDA library under ``csrc/`` (C ABI declared in
``include/h2.h``); ``paper_2403_01566_gb300.h2`` is the thin ctypes binding.
This ``__init__`` deliberately imports nothing so that the seeded input
generators in ``paper_2403_01566_gb300.inputs`` can be used without loading
the CUDA library.
"""
