"""CPU oracle for the xTC grid build (test infrastructure only).

Plain, slow FP64 numpy restatements of the paper (arXiv 2304.07006), written
from its equations and sharing nothing with the CUDA library:

* ``jastrow``     -- the Jastrow factor u(r1, r2), its gradient with respect
                     to the first electron (the nabla_1 u in the three-body L)
                     and its Laplacian (in the two-body integrals K).
* ``direct``      -- Route 2: the restricted closed-shell working equations of
                     Appendix B (Delta U, Delta h, <Phi0|L|Phi0>), with the
                     intermediate vector field V of the "Decomposition of two-body
                     correction" section.
* ``spin``        -- Route 2 for two spin densities: the restricted open-shell
                     working equations of Appendix A (Delta U^{aa}, ^{ab}, ^{bb},
                     Delta h^a, Delta h^b, <Psi0|L|Psi0>).
* ``frozen_core`` -- xTC-FC: the standard closed-shell frozen-core folding of
                     Delta U and Delta h over a core orbital set (Results section,
                     "Frozen core approximation").
* ``two_body_k``  -- the two-body integrals K of the Theory section on the grid
                     (the double grid sum of the operator 1/2 P12 [lap_1 u +
                     (grad_1 u)^2 + 2 grad_1 u . grad_1] between orbital products).
* ``bruteforce``  -- Route 1: the six-index L from eq. (Ldecomp) or from the
                     literal triple quadrature of its definition, normal-ordered
                     explicitly in spin orbitals with eqs. (dU), (Delta h with the
                     two-body density), (zero-body) and (1Ddens), for one density
                     or for separate alpha and beta densities.

Only the tests, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may import this package; the library never does.

Parity status: every function here is pinned by CPU tests
(``tests/test_oracle_*.py``) against finite differences, the literal triple
quadrature, the paper's own identities between its two routes, symmetry and
homogeneity invariants, a closed form for a separable Jastrow factor, for
the frozen-core folding Fock-space matrix elements of the second-quantised
operator with the core filled, and for K the similarity transformation
e^{-u} lap (e^{u} f) - lap f evaluated by differences.
"""
