"""GB300 (sm_103a) implementation of the RD3Q81 lattice Boltzmann step (arXiv 2409.05114).

The compute path is liblbm_rd3q81.so (hand-written CUDA behind a C ABI, include/lbm.h);
``binding`` is its ctypes binding, ``workloads`` builds seeded initial fields.
"""
