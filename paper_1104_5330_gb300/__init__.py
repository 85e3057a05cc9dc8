"""GB300 library for one time step of the 6-D spectral transport method
(Bonazzola, Vasset & Peres 2011) behind the C ABI of include/ts.h.

Submodules:
  ts        -- ctypes binding of libts.so (same names as the C ABI) and a Grid handle
  autograd  -- torch.autograd.Function over ts_step / ts_adjoint_step with
               sqrt(N) step checkpointing
  inputs    -- seeded synthetic inputs (no arithmetic of the method)
  build     -- nvcc build of libts.so for sm_103a

Importing the package loads nothing; ``paper_1104_5330_gb300.ts`` loads the
library and raises if it is missing.
"""
