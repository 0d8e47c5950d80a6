"""GB300-native hot path of the mass-conserving mixed-stress Stokes method (arXiv 2207.08481).

The computation lives in the C-ABI library ``libmcs.so`` (CUDA, sm_103a); ``mcs`` is its
ctypes binding.  Build it with ``paper_2207_08481_gb300.build.build()``.
"""
