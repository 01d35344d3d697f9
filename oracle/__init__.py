"""Plain, slow FP64 CPU oracle of periodic MSC-LBM (test infrastructure).

This package is the independent reference that the CUDA library is checked
against.  It is test infrastructure only: the tests, the smoke entry point and
the CPU-baseline leg of the benchmark may call it; the product path never does.
It shares no code with the CUDA library.  Everything is numpy in float64,
written to be checked against the paper by eye:

* ``lattice``   D2Q9 / D3Q19 velocity sets (Appendix A, Eqs. d2q9 / d3q19).
* ``kinetics``  moments, He-Luo equilibrium, BDF coefficients, half-source
                reconstruction, source distribution, TRT collision
                (Section 2.2, Eqs. moments .. collision-operating).
* ``sweep``     push streaming, the full sweep T and the raw residual
                (Eqs. sweep, residual).
* ``shadow``    DFT convention, wavenumbers, mask, Schur solve of the shadow
                system and the equilibrium lift (Section 3.2, Eqs. schur ..
                shadow-update), with the DFT as a naive separable sum.
* ``march``     Algorithm 1 (MSC and plain Picard dual-time stepping), the
                explicit LBM, population/moment histories (Section 3.1).
* ``linear``    the linearised Fourier symbol of one sweep and of one corrected
                iteration (Eqs. local-linear-response, symbol).
* ``fullsymbol``  the full-symbol reference operator of off-design runs
                (Eq. full-symbol) and the TRT rate / ghost-survival relations
                (Eqs. trt, eta).
* ``adjoint``   the discrete adjoint of the converged march (implicit
                differentiation of every accepted fixed point; exact sparse
                solves, complex-step collision Jacobians) and the body force.

Parity status per function is stated in each module header; every function
here is pinned by at least one ``-m "not gpu"`` test except where a header says
"parity unpinned".
"""
