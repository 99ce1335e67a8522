"""Two-body transcorrelated integrals K on the grid (oracle, FP64).

Theory section, the non-hermitian two-body integrals that the similarity transformation adds
beside V (and that U = V - K combines, Generalized normal ordering section):

    K_PR^QS = 1/2 <PR| P12 [ nabla_1^2 u(1,2) + (nabla_1 u(1,2))^2 + 2 nabla_1 u(1,2) . nabla_1 ] |QS>,
    P12 f(1,2) = f(1,2) + f(2,1).

For real spatial orbitals the spin deltas factor out, and on the quadrature grid the matrix
element of an operator O(1,2) is

    <PR| O |QS> = sum_{i,j} w_i w_j phi_P(r_i) phi_R(r_j) [ O phi_Q(1) phi_S(2) ](r_i, r_j),

where the nabla_1 of the derivative term acts on phi_Q (taken from the orbital gradients, an
input).  f(2,1) is the same operator with the electrons' roles exchanged: the Laplacian, the
square and the gradient of u with respect to its first slot evaluated with electron 2 there,
and the derivative acting on phi_S.

Output: K[p, q, r, s] = K_pr^qs (electron 1: p -> q, electron 2: r -> s), the index order of
Delta U in this package.

Readings where the paper is silent: the coincident pair of grid points (j = i) stays in the double
sum, with the readings of ``jastrow.grad1`` and ``jastrow.lap1`` (unit vectors and the 2 a'/r terms
of the Laplacian are 0 below 1e-14 bohr; the rest is evaluated as written), the same reading as
for the gradient in V.  ``coincident=False`` drops the pair instead (for comparisons that cannot
evaluate it, such as differences).

Test infrastructure only: only the tests, the smoke entry point and the CPU baseline may import it.
"""
from __future__ import annotations

import numpy as np

from . import jastrow


def _pair_fields(first, second, jas):
    """(nabla_1 u, nabla_1^2 u + |nabla_1 u|^2) with u's first slot at ``first`` and its second at
    ``second``, both broadcast (n, n, 3) views of the grid."""
    g = jastrow.grad1(first, second, *jas)
    f = jastrow.lap1(first, second, *jas) + np.sum(g * g, axis=-1)
    return g, f


def k_integrals(grid, weights, phi, dphi, nuc_xyz, nuc_set, terms, coef, coincident=True):
    """K[p, q, r, s] for the orbitals ``phi`` (n_grid, N) with gradients ``dphi`` (n_grid, N, 3);
    ``coincident=False`` leaves out the pairs j = i."""
    X = np.asarray(grid, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    dphi = np.asarray(dphi, dtype=np.float64)
    jas = (nuc_xyz, nuc_set, terms, coef)
    n, N = phi.shape
    ri = np.broadcast_to(X[:, None, :], (n, n, 3))  # electron 1 at grid point i
    rj = np.broadcast_to(X[None, :, :], (n, n, 3))  # electron 2 at grid point j
    # f(1,2): u's first slot holds electron 1;  f(2,1): it holds electron 2
    g12, f12 = _pair_fields(ri, rj, jas)
    g21, f21 = _pair_fields(rj, ri, jas)
    if not coincident:
        off = 1.0 - np.eye(n)
        g12, g21 = g12 * off[..., None], g21 * off[..., None]
        f12, f21 = f12 * off, f21 * off

    wphi = w[:, None] * phi                                   # w_i phi_P(i)
    pair = (wphi[:, :, None] * phi[:, None, :]).reshape(n, N * N)  # w_i phi_P(i) phi_Q(i), (P, Q)

    # f(1,2): the multiplicative part, then the derivative acting on phi_Q(1)
    A = pair.T @ (f12 @ pair)
    for x in range(3):
        bra_der = (wphi[:, :, None] * dphi[:, None, :, x]).reshape(n, N * N)  # w phi_P d_x phi_Q
        A = A + 2.0 * bra_der.T @ (g12[:, :, x] @ pair)
    # f(2,1): the multiplicative part, then the derivative acting on phi_S(2)
    B = pair.T @ (f21 @ pair)
    for x in range(3):
        ket_der = (wphi[:, :, None] * dphi[:, None, :, x]).reshape(n, N * N)  # w phi_R d_x phi_S at j
        B = B + 2.0 * pair.T @ (g21[:, :, x] @ ket_der)
    return 0.5 * (A + B).reshape(N, N, N, N)
