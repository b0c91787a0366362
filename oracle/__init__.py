"""FP64 CPU oracle for variance-reduced ProxSkip tomography (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow, obviously-correct statement of what the CUDA library
computes.  It exists so that the GPU path can be checked against something written
independently from the paper.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path (the C-ABI library and its Python
binding) never does, and the two share no code.  All floating point is float64.

Passages followed (arXiv 2602.09527):
  * problem:        Eq. (tomography_problem), Section 2.1 -- 1/2||Ax-b||^2 + alpha TV(x) + I_{x>=0}
  * subsets:        Section 1.2 (finite-sum split) and Fig. 1 caption (staggered angle subsets)
  * estimators:     Section 1.2, Eq. (saga_estimator) and the SVRG / L-SVRG paragraph,
                    and the estimator table of Algorithm 1
  * ProxSkip:       Algorithm 1 (parameters gamma, p, N; x_hat, Bernoulli(p) coin, prox with
                    scale gamma/p, control-variate update of h)
  * prox:           Eq. (proximal_definition); FGP with warm-started, fixed inner iterations
                    (Section 2.1, Beck & Teboulle 2009)
  * step sizes:     Section 3 (ISTA 1.99/L, FISTA 1/L, SAGA 1/(3L), SVRG/L-SVRG 1/L)

Parity status: every function here is pinned by a test in ``tests/test_oracle_*.py``
against closed forms, brute force or invariants (see the module docstrings); none is
"parity unpinned" except the long-run reference value F* used to define a relative
objective gap at large sizes, which is not computed here.
"""
