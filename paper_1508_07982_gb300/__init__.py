"""GB300-native refined-grid D3Q19 lattice Boltzmann (Schornbaum & Ruede, arXiv:1508.07982).

The compute path is the C-ABI library built from ``csrc/`` (see ``include/lbm_gb300.h``);
``lbm`` is its thin ctypes binding and ``inputs`` holds the seeded synthetic workloads.
Importing the package itself loads nothing.
"""
