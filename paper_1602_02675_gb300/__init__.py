"""GB300 tau = 1 semi-discrete lattice Boltzmann solver.

The compute path is the CUDA library ``liblbm.so`` (C ABI in
``include/lbm.h``); ``paper_1602_02675_gb300.lbm`` is its Python binding.
Importing this package does not load the library; importing ``.lbm`` does,
and fails loudly when it has not been built.
"""
