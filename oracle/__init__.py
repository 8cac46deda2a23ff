"""Plain FP64 CPU oracle for the generalized Stokes solve (TEST INFRASTRUCTURE).

This package is the independent checker of the CUDA path.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it; the product path (the C ABI library and its
Python binding) never does and shares no code with it.

It follows the paper's definitions with assembled sparse matrices, standard
Gauss quadrature and textbook Krylov / multigrid steps, without blocking,
fusion or reordering:

* ``mesh``   structured Q2-Q1 numbering, Dirichlet and obstacle constraints
             (Sec. 3.2, Eq. "spaces"; nested meshes of Sec. 4).
* ``fem``    reference element, cell matrices by 3-point Gauss quadrature,
             assembly of A, B and the pressure masses (Eqs. "form_a_j",
             "form_b", "stokes-discrete-block").
* ``mg``     level hierarchy, Q2 prolongation, Lanczos eigenvalue estimate,
             Chebyshev smoother, velocity V-cycle, Schur mass approximation
             (Sec. 4, the Cheb(A, diag A, k_A) smoother).
* ``krylov`` right-preconditioned FGMRES with classical Gram-Schmidt applied
             twice and Givens rotations (Sec. 5, "Linear solver settings").

Parity status of each function is stated in its module header.
"""
