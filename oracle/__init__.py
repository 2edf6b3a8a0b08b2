"""CPU oracle for the spectral finite-element Magnus-Lanczos TDKS step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the test suite, the smoke check and the benchmark's CPU-baseline leg may.
It shares no code with the CUDA library (no tables, helpers or kernels).

Plain, slow, double-precision (complex128) numpy implementation of what
Kanungo & Gavini (arXiv 1810.13130) define:

* basis.py        GLL nodes/weights (spectral elements, Sec. VI.A) and Gauss rule
* mesh.py         tensor-product hexahedral mesh, nodal map, GLL-lumped (diagonal) M
* hamiltonian.py  discrete Hamiltonian Eq. 15 by Gauss quadrature, Loewdin transform
                  Eq. 21, density Eq. 2, Poisson load vector Eq. 19, dipole (Sec. V)
* xc.py           adiabatic LDA (Ceperley-Alder data, Perdew-Zunger fit), Sec. II
* poisson.py      Hartree potential from K phi = 4 pi c (Eq. 19) by Jacobi PCG
* lanczos.py      Krylov approximation of exp(-i tau Hbar) psi, Eqs. 36-38
* propagate.py    second-order Magnus step with midpoint rule (Eqs. 25-26) and the
                  predictor-corrector of Sec. VI.B
* ground_state.py self-consistent ground state used as the initial state (Sec. VII)

Parity pins for every module live in tests/test_oracle_*.py.  Parity status:
all functions are pinned (closed forms, textbook special cases, library routines
or invariants); the predictor-corrector is pinned only through the Dt^2 rate,
the harmonic-potential theorem and conservation laws.
"""
