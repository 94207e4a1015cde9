"""GB300 (sm_103a) chemical-potential multiphase lattice Boltzmann method
(Wen, Zhao, Qiu, Ye and Shan, arXiv:1906.09530)."""
