"""B300-native multi-order retarded-time imaging operator A / A^T.

The compute path lives in the C-ABI library ``librtt.so`` (hand-written CUDA
for sm_103a, sources in ``csrc/``, declarations in ``include/rtt.h``).
``paper_2609_05528_b300.rtt`` is the thin ctypes binding with the same entry
point names; ``paper_2609_05528_b300.inputs`` holds the seeded synthetic
workloads.  Importing the package does not load the CUDA library.
"""
__all__ = ["inputs", "rtt"]
