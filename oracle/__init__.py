"""Plain FP64 CPU oracle for the SIPG hp-multigrid smoothing path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
Python binding) may import this package; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

Every routine here is written for a reader checking it against the paper
(Baccas, Belozerov, Mueller, Weinzierl, "Implementation techniques for multigrid
solvers for high-order Discontinuous Galerkin methods", arXiv 2510.00998):
numpy / scipy library primitives (tensordot, sparse products, dense solves) are
used as steps, with no blocking, fusion or reordering beyond what the paper's
definitions and algorithms state.

Modules
  refelem   1D reference element: GLL nodes, Lagrange basis, exact M and K (Sec. 2.2)
  sipg      SIPG bilinear form (Eq. weak_form_IP extended with kappa), assembled by
            quadrature (Sec. 2.3.2), the matrix-free facet route (Alg. 2, Eq.
            weak_form_IP_facet_spaces), the block diagonal (Schur complement
            block, Sec. 4.1), block-Jacobi in Alg. 2 and Alg. 4 order, load
            vector and L2 error
  hpmg      p-transfer (Eq. prolongation), Q1 CG levels (Sec. 2.4, 5.2), point
            Jacobi, h-transfer, V-cycle (Alg. 6/7 shape), PCG and MGMult
  traffic   the memory-access model of Sec. 4.1 (Table 1)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``, ``hpmg.mgmult`` included (its iterates against the
dense cycle matrix, its exit rules against the norms of those iterates). Its
cycle counts against Tables 3-5 are a comparison under a reading, not a pin: the
paper does not state omega, nu or the penalty it used there.
"""
