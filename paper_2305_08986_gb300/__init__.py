"""GB300-native matrix-free solver for the generalized Stokes problem.

alpha u - div(2 eta eps(u)) + grad p = f,  div u = 0, Q2-Q1 Taylor-Hood on structured
quad/hex meshes with per-cell viscosity (Wichrowski, Krzyzanowski, Heltai, Stupkiewicz,
"Exploiting high-contrast Stokes preconditioners to efficiently solve incompressible
fluid-structure interaction problems", Sec. 4 and 5).

The compute path is the C-ABI library ``libgs.so`` built from ``csrc/`` (hand-written
sm_103a CUDA); ``gs`` is its thin Python binding.  Importing this package does not load
the library; ``paper_2305_08986_gb300.gs`` does, and fails loudly when it is missing.
"""
__all__ = ["inputs"]
