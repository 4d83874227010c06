"""Plain, slow FP64 CPU oracle of the HHG / HyTeG P1 multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library (``paper_1805_10167_gb300``): the two meet
only through the seeded inputs of ``paper_1805_10167_gb300.inputs`` and through
vectors in the canonical DoF order.

Paper: Kohl, Thoennes, Drzisga, Bartuschat, Ruede, "A Scalable and Modular
Software Architecture for Finite Elements on Hierarchical Hybrid Grids" (2018).

Modules
  mesh       macro-primitive graph (Sec. 2.1), structured refinement (Sec. 3.1),
             canonical numbering of the unknowns with unique ownership (Sec. 2.2)
  fem        P1 element stiffness / mass, brute-force CSR assembly, element-loop
             apply (Sec. 4.2), quadrature-based L2 error
  multigrid  colour-ordered Gauss-Seidel, damped Jacobi, prolongation and
             restriction, coarse CG, V-cycle and the V-cycle solver (Sec. 4.3)
  krylov     flexible GMRES (Saad 1993) and preconditioned / flexible conjugate
             gradients, each taking the operator and preconditioner as callables
  learned    the learned smoother's network (convolutions, forward, hand-derived
             backward passes, BF16 rounding, Adam step, face images and crops)

Iterative refinement has no oracle function of its own: its FP64 outer loop is
checked against the tolerance and against the oracle's V-cycle solve.  Single
rows of the operator at sizes the oracle cannot assemble are built in
``tests/fullsize_rows.py`` from this package's element matrices.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, invariants or brute force; the multigrid cycle as a whole is an
iteration with no closed form and is pinned by invariants only (convergence
factor level independence, two-grid agreement, Galerkin identity).
"""
