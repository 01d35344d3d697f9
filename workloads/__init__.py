"""Seeded synthetic workloads: initial fields, unit-test inputs and continuum references.

Shared by the tests, the benchmark and the oracle.  Holds none of the MSC-LBM
arithmetic (no equilibrium, sweep, transform or solve of the method): only
initial macroscopic fields, random inputs for unit tests, the Taylor-Green
closed form, an independent pseudo-spectral Navier-Stokes reference for the
random-phase fields, and error metrics.
"""
