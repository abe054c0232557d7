"""GB300-native PGD-TO optimizer step (arXiv 2511.13905).

The compute path is the C-ABI library ``libpgdto.so`` built from ``csrc/`` (hand-written
sm_103a CUDA); ``binding`` wraps it with ctypes.  ``inputs`` draws the seeded synthetic
workloads.  Nothing in this package falls back to CPU arithmetic: if the library is
missing, ``binding.load()`` raises.
"""

__all__ = ["binding", "inputs"]
