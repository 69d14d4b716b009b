"""GB300-native multigrid for multi-patch isogeometric Poisson problems.

Submodules:
  mgiga      -- ctypes binding of the C-ABI library libmgiga.so (import it
                explicitly: it loads the CUDA library)
  workloads  -- seeded synthetic problems (inputs only)
  build      -- compiles libmgiga.so for sm_103a
"""
