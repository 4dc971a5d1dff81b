"""GB300-native monolithic n-field coupled solver (BGS(AMG), SIMPLE(AMG),
AMG(BGS) preconditioned GMRES).  The solver lives in the C-ABI library
``libmfs.so`` built from ``csrc/``; ``mfs`` is its thin ctypes binding and
``inputs`` the seeded synthetic block-system generators."""
