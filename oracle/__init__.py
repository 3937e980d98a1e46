"""Plain FP64 CPU oracle of the CTD (convolution tensor decomposition) Allen-Cahn step.

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA path; it is not part of
the product.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code, constants or
helpers with ``paper_2410_15519_gb300`` and never imports it.

Modules
-------
actd      Adaptive CTD (Section 3.3, "Adaptivity"): the full-grid C-FEM step by fast
          diagonalisation when a step needs more than M_c modes.
cfem      1D C-FEM shape functions (App. B radial basis interpolation, App. C), the 1D
          stiffness matrix (Eq. KxxMxx), the nodal and Gauss quadrature rules.
ctd       The stabilized semi-implicit step (Eq. AC-discrete-semi-stable-K) solved in
          separated form by greedy enrichment + alternating fixed point (Section 3.3,
          Eq. ux, Eq. KxQx, Eq. KyQy, App. D), the discrete energy, reconstruction.
fullgrid  Brute-force full-grid solve of the same stabilized step (Eq.
          AC-discrete-semi-stable-K with Kronecker-assembled operators), used only to pin
          ``ctd``.
splitmix  SplitMix64, the counter-based generator used to initialise new modes.

Every function is written in FP64 with library primitives (matmul, banded Cholesky,
dense solve) as single steps and no blocking, fusion or reordering beyond the paper's
definitions.  Readings of places where the paper is silent are listed in each docstring.
"""
