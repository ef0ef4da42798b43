"""GB300-native homogenized lattice Boltzmann (HLBM) time step for fully
resolved particulate flow (arXiv:2312.14172), behind the C-ABI of
include/hlbm.h.  ``hlbm`` is the Python binding; ``workloads`` draws the
seeded synthetic inputs; ``build`` compiles libhlbm.so for sm_103a."""
