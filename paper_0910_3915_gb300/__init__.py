"""GB300-native two-component Shan-Chen D3Q19 lattice Boltzmann library.

The compute path is the C-ABI shared library built from ``csrc/`` (CUDA for
sm_103a); ``lbsc`` is its thin ctypes binding. Importing this package loads
nothing; ``paper_0910_3915_gb300.lbsc`` loads the library and raises if it is
missing.
"""
