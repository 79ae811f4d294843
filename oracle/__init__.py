"""Naive FP64 CPU oracle for the matrix-free DG compressible Navier--Stokes operator.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  It shares no
code with the CUDA path (``paper_1806_03095_gb300``); the only module both
sides use is the seeded input generator ``paper_1806_03095_gb300.inputs``,
which holds none of the method's arithmetic.

Every integral is a plain Gauss sum with full interpolation matrices
(``(k+1)^3 x n_q^3`` values and gradients per cell, ``(k+1)^3 x n_q^2`` per face):
no sum factorization, no even-odd decomposition, no fusion.  Plain PyTorch CPU
float64 ops; cells are processed in chunks only to bound memory.

Modules
-------
basis        1D Gauss--Legendre rule, LGL nodes, Lagrange basis (Sec. 2.2.1, 2.2.3)
mesh         structured hexahedral box meshes, isoparametric degree-k mappings
physics      fluxes F_c, F_v, pressure, speed of sound (Sec. 2.1)
operator     weak form (Eq. WeakFormulationConservedVariables), mass matrix, L(U)
rk           low-storage RK(5,4) in 2N form (Carpenter & Kennedy 1994)
diagnostics  kinetic energy, dissipation, conservation totals (Sec. 4.2.3)
mms          manufactured-solution sources by automatic differentiation

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` except the channel wall boundary state, whose
imposition the paper omits (parity unpinned beyond conservation of mass
through the wall and free-stream checks; see the wall reading in ``physics``).
"""
