"""GB300-native two-component pseudopotential (Shan-Chen) D2Q9 lattice
Boltzmann method with the improvements of arXiv:2111.08666: modified explicit
forcing with a system relaxation time, improved virtual solid density wetting,
boundary-column force mirroring and the Set-3 inlet/outlet pressure
boundaries.

The compute path is the CUDA library ``libmclbm.so`` behind the C ABI in
``include/mclbm.h``; ``paper_2111_08666_gb300.mclbm`` is its ctypes binding.
Importing the package does not load the library.
"""
