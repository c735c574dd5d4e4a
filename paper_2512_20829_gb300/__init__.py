"""GB300 (sm_103a) library for the fully Lagrangian approach (FLA) advance and the
kernel-regression / PSI-CELL source-term deposits of Stafford & Rybdylova,
"Interphase coupling for gas-droplet flows using the fully Lagrangian approach".

``fla`` is the Python binding of the C-ABI library ``libfla.so`` (built by
``build.build()``); ``inputs`` describes the seeded synthetic workloads.
Importing the package loads nothing; the binding loads the library on first use.
"""
__all__ = ["fla", "inputs", "build"]
