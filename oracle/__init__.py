"""FP64 CPU oracle for the SIP-DG Stokes solver of Charrier, May & Schnepp
(arXiv 1607.03777).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code, table or helper with the CUDA library; the two meet only
through seeded inputs drawn by ``paper_1607_03777_gb300.synth``.

Design: every operator is *assembled explicitly* from the paper's bilinear
forms (Sec. 4, eqs. stiffness_form / divergence_form / rhs_f) by
Gauss-Legendre quadrature at physical points, with basis functions
evaluated through ``numpy.polynomial.legendre``.  Solvers are written from
Sec. 5-6 (Algorithm 1, the Chebyshev / block-Jacobi smoother, the
Q^2_1 coarse space with its continuous bilinear h-hierarchy, PCG and
right-preconditioned FGMRES with the upper block-triangular preconditioner).

Modules
  basis      orthonormal Legendre basis, quadrature, dof numbering
  sip        A, B, f, S*, block-Jacobi blocks, per-element rows
  materials  element-wise max-viscosity / min-density rasterisation (Sec. 7.3)
  rng        SplitMix64 counter-based generator (published definition)
  multigrid  Chebyshev, eigen estimate, p-transfer, P_cd, h-hierarchy, V-cycle
  krylov     PCG, FGMRES with the block preconditioner, sparse-direct solve
  exact      manufactured solutions used by the convergence-rate pins

Parity status of each function is stated in its docstring; every function
is pinned by a ``-m "not gpu"`` test against something other than itself
(closed forms, invariants, brute force) unless it says "parity unpinned".
"""
