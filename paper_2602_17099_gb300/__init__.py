"""GB300 (sm_103a) implementation of the RNSM merge path and the MOS planner.

The compute lives in ``librnsm.so`` (hand-written CUDA kernels behind the C
ABI of ``include/rnsm.h``); :mod:`paper_2602_17099_gb300.rnsm` is its Python
binding.  Build the library with :func:`paper_2602_17099_gb300.build.build`.
"""
__all__ = ["rnsm", "build"]
