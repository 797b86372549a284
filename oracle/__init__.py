"""FP64 CPU oracle for the multiple-domain Galerkin BEM of arXiv 1910.01011.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, independently
written reference that the CUDA library is checked against.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may
import it; the library never does, and the two share no code (only the
seeded input generators of the separate `synth` package).

Modules: quadrature (rules), galerkin (C element-pair integrals, P1 mass and
stiffness), pmchwt (block system, right-hand side, dense solve), mie
(analytic sphere), osrc (preconditioner), rayleigh (transducer field),
gmres (restarted GMRES).

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, identities or brute force; see each test's docstring.
"""
