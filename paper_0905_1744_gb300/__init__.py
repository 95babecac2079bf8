"""GB300-native k-mer rank and regular-sampling partitioner (Sample-Align-D, Sec. 3.1).

The compute path is the CUDA library ``libsad.so`` (built from ``csrc/`` for
sm_103a) behind the C-ABI declared in ``include/sad.h``; ``sad`` is the thin
Python binding. Importing this package does not load the library; the first
call into ``sad`` does, and raises if the library is missing.
"""
__all__ = ["sad", "datagen"]
