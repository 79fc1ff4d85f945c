"""GB300-native encrypted DLRM inference (HE-LRM hot path).

Submodules (nothing is imported eagerly, so ``synthetic`` can be used without
loading the CUDA library):
  helrm      -- ctypes binding of the C-ABI library libhelrm.so (csrc/).
  build      -- compiles csrc/ for sm_103a.
  synthetic  -- seeded synthetic workloads shaped like the paper's datasets.
"""
