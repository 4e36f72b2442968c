"""Plain FP64 CPU oracle for the Ohta--Kawasaki Newton linear solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check of the package entry file and the CPU-baseline
leg of the benchmark may call it.  It shares no code with the CUDA library;
both sides take their inputs from ``ok_inputs``.

Contents (each function cites the passage of Farrell & Pearson,
"A preconditioner for the Ohta--Kawasaki equation", that it follows):

``fem``      uniform P1 simplex meshes, assembled CSR matrices M, K, M_E,
             the nonlinear term N(u), the residual F and the Jacobian J
             (Sec. 2, eqns oka/okb and newton).
``solvers``  Jacobi--Chebyshev semi-iteration, geometric multigrid V-cycles,
             the block lower-triangular preconditioner with the matching
             Schur approximation (eqns prec, outer_approx, schurinv), FGMRES,
             Newton and the theta-method timestep.

Everything is float64, assembled from element integrals with the exact
simplex monomial rule, and written for a reader to check against the paper
by eye rather than for speed.  Pinned by tests/test_oracle_*.py; the one
function without an independent pin is listed there as "parity unpinned".
"""
