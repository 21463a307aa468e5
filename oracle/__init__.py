"""Plain, slow, FP64 CPU oracle of one semi-implicit CH / AC / NS step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package;
the product path (the CUDA library and its Python binding) never does.  The
oracle shares no code with the CUDA path: it builds its own mesh, its own
quadrature (collapsed Gauss-Legendre rules from numpy), its own assembly
(dense element matrices scattered with scipy.sparse), and its own solvers,
each written out from the paper's equations in the paper's order.

Modules
  mesh        structured triangulation, P1 / P2 node numbering (Sec. 3)
  quadrature  collapsed Gauss rules on the reference triangle and tetrahedron
  fem         element integrals and global assembly (Sec. 3, Sec. 4)
  model       potential, right-hand sides and the linear systems (Sec. 2-4)
  mg          geometric multigrid used as the inner solves of Sec. 4
  krylov      FGMRES / PCG / Chebyshev iteration (Sec. 5 solver setup)
  step        one semi-implicit step (Sec. 3 time scheme, Sec. 4 systems)
  adjoint     the discrete adjoint of the step and trajectory gradients
  three_d     the step on Kuhn tetrahedral meshes of a box (Sec. 5's 3D runs)
  adjoint_three_d  the discrete adjoint of the 3D step
"""
