"""GB300-native Newton-FGMRES for MAC Navier-Stokes on voxel images with pore-level multiscale
preconditioners (gPLMM, aPLMM_NS, aPLMM_S).  The compute path is the C-ABI library libpns
(hand-written sm_103a CUDA); `pns` is its Python binding and `inputs` makes seeded workloads."""
