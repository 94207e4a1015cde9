"""FP64 CPU oracle of the chemical-potential multiphase LBM (arXiv:1906.09530).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the CUDA library never does, and the two
share no code.  `sim` wraps the plain C restatement of one time step
(cplbm_oracle.c); `thermo` holds the Carnahan-Starling thermodynamics and
`eos` the other equations of state of Sec. 3.2 (VDW, RK, RKS, PR, and CS again
by a generic route).
"""
from . import eos, thermo  # noqa: F401
from .sim import OracleSim, cfd_alpha, cfd_line, cs_mu0, cs_p0, forcing_terms  # noqa: F401
