"""DG-HGKS per-stage residual on one NVIDIA B300 (sm_103a).

The compute path is the CUDA library ``libdghgks.so`` (C ABI, declared in
``include/dghgks.h``); ``api`` is its thin Python binding.
"""
