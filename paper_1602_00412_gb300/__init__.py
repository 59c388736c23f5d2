"""GB300 Sparse Frequent Directions (Ghashami, Liberty, Phillips).

The compute path lives in libsfd.so (CUDA for sm_103a, C ABI in
include/sfd.h); ``paper_1602_00412_gb300.sfd`` is its thin ctypes binding.
``paper_1602_00412_gb300.synth`` makes seeded synthetic inputs.
"""
