"""GB300 (sm_103a) blockwise 2-D DCT approximations of arXiv 2207.11638.

The compute path is the CUDA library ``libcdct.so`` (C ABI in
``include/cdct.h``); ``binding`` is its thin ctypes wrapper and ``synth`` the
seeded synthetic inputs.  Importing ``binding`` fails if the library has not
been built (``python -m paper_2207_11638_gb300.build``).
"""
__all__ = ["binding", "synth", "build"]
