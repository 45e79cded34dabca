"""GB300-native many-variable VMC hot path (mVMC, arXiv:1711.11418).

The compute path lives in ``libvmc.so`` (CUDA, sm_103a) behind the C ABI of
``include/vmc.h``; ``paper_1711_11418_gb300.vmc`` is its thin ctypes binding.
Importing this package does not load the library.
"""
