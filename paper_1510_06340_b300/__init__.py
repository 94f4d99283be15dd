"""MUSTA-FORCE relativistic hydrodynamics on B300 (sm_103a).

The solver itself is the C-ABI library ``libhydro.so`` built from ``csrc/``;
``hydro`` is its thin ctypes binding and ``inputs`` the seeded workload
generators.  Importing the package loads nothing.
"""
