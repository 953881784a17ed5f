"""GB300-native ADER-DG predictor/corrector (Dumbser et al. 2018).

Submodules:
  aderdg  -- ctypes binding of the C-ABI library (libaderdg.so), same names
             as include/aderdg.h; the only compute path (CUDA, sm_103a)
  build   -- compiles the CUDA library in-tree with nvcc
  inputs  -- seeded synthetic initial conditions / exact solutions
"""
