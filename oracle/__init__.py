"""Plain FP64 CPU oracle for the matrix-free spectral-element Burgers operator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything
under ``oracle/``.  The product path (``paper_1806_01422_gb300``) never imports
it and shares no code with it.

Contents (each function cites the passage of Marin, Constantinescu & Smith,
"A scalable matrix-free spectral element approach for unsteady PDE constrained
optimization using PETSc/TAO", arXiv:1806.01422, that it follows):

* ``gll``        -- Gauss-Lobatto-Legendre nodes, weights, derivative matrix (Sec. 3.2).
* ``sem``        -- the semi-discrete operator F(u), its tangent J(u)w and the
                    transpose J(u)^T v (Sec. 3.2-3.3, eqs. rhsvec/jacvec/jactransvec),
                    the global mass and the misfit objective (eq. ourcost).
* ``rk``         -- explicit Runge-Kutta forward sweep and its discrete adjoint
                    (Sec. 4.1, eqs. adjointloop/initadj/gradient, eq. adjtime).
* ``checkpoint`` -- binomial (revolve-optimal) checkpoint schedule by brute-force
                    dynamic programming, and a checkpointed adjoint (Sec. 5.3).

Everything is numpy float64.  Library primitives (tensordot, add.at) serve as
steps; there is no blocking, fusion or reordering beyond the formulas.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
the mathematics (exact quadrature, exact polynomial derivatives, spectral
convergence to closed forms, exact central differences of a quadratic map,
transposes of assembled Jacobians, Taylor polynomials of exp(dt A), brute-force
schedules).  No function is "parity unpinned".
"""
