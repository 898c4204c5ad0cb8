"""GB300-native LB-IB-MLS adhesion solver (arXiv:1808.01448 hot path).

The compute path is the CUDA library ``_build/liblbib.so`` (sm_103a) behind the
C ABI declared in ``include/lbib.h``; ``lbib`` is its ctypes binding.
"""
