"""GB300 (sm_103a) chemical-potential multiphase lattice Boltzmann method
(Wen, Zhao, Qiu, Ye and Shan, arXiv:1906.09530).

The compute path is the CUDA library libcplbm.so (C ABI in include/cplbm.h);
this package is its ctypes binding plus the seeded synthetic workloads.
"""
from ._binding import (LBM_PREC_FP64, LBM_PREC_MIXED, LBM_PREC_MIXED_DF,  # noqa: F401
                       Batch, LbmError, Mlp, Simulation, cs_eos, lbm_cfd, lbm_cfd_df,
                       lbm_critical, lbm_maxwell, lbm_strerror, lbm_workspace_bytes, lib,
                       make_eos)
