"""GB300-native data-parallel core of Sample-Align-D (k-mer-rank partitioning
and per-bucket all-pairs affine-gap alignment scores).

The compute path is the C-ABI library ``libsad.so`` (CUDA for sm_103a) under
``csrc/``; ``paper_0901_2742_gb300.sad`` is its thin ctypes binding. Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["sad", "synth"]
