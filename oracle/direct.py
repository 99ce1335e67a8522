"""Route 2: the restricted closed-shell xTC working equations (oracle, FP64).

Written from Appendix B ("Restricted closed-shell working equations") with the
intermediate V of the "Decomposition of two-body correction" section:

    V_rs(i)  = sum_j w_j phi_r(j) nabla_1 u(r_i, r_j) phi_s(j)          (intermediate V)
    rho_pq(i) = w_i phi_p(i) phi_q(i)
    W(i)     = 2 V_tu(i) gamma_tu
    Vt_rs(i) = W(i) . V_rs(i)
    X_us(i)  = V_ts(i) gamma_tu
    Zt_rs(i) = V_ru(i) . X_us(i)
    A_rs(i)  = Vt_rs(i) - Zt_rs(i)
    Wt(i)    = 2 rho_tu(i) gamma_tu
    Y_rt(i)  = V_ru(i) gamma_tu
    Z_rs(i)  = rho_ru(i) X_us(i) + Y_rt(i) rho_ts(i)
    B_rs(i)  = 1/2 Wt(i) V_rs(i) - Z_rs(i)
    dU[p,q,r,s] = Delta U_pr^qs = -P^(pq)_(rs) sum_i (rho_pq A_rs + V_pq . B_rs)
    dh[p,q]  = -1/2 (2 Delta U_pr^qs gamma_rs - Delta U_pr^sq gamma_rs)
    e0       = <Phi0|L|Phi0> = -2/3 dh_pq gamma_pq

The pair symmetriser P^(pq)_(rs) f = f(pq, rs) + f(rs, pq) (reading of the
undefined operator; it follows from eq. (Ldecomp) inserted in eq. (dU)).
Repeated indices are summed (the paper's Einstein convention, grid index i
included).  gamma is the per-spin density; the spin factor 2 is explicit.

Every sum is evaluated as written; the sum over inner grid points j is
accumulated over pieces of the grid and the sum over outer points i over
pieces of the requested outer set, which bounds memory and changes only the
order of additions.  ``outer`` restricts the i-sum to a subset of grid
points (the result is linear in that sum), which is how large workloads are
checked on sampled outer points.
"""
from __future__ import annotations

import numpy as np

from . import jastrow


def vfield(grid, weights, phi, jas, outer_idx, j_block=2048):
    """V[i, x, r, s] for the outer points ``outer_idx`` (full inner j-sum)."""
    nuc_xyz, nuc_set, terms, coef = jas
    ri = grid[outer_idx]
    n_orb = phi.shape[1]
    V = np.zeros((len(outer_idx), 3, n_orb, n_orb))
    for j0 in range(0, grid.shape[0], j_block):
        j1 = min(j0 + j_block, grid.shape[0])
        G = jastrow.grad1(ri[:, None, :], grid[None, j0:j1, :], nuc_xyz, nuc_set, terms, coef)
        rho_j = np.einsum("j,jr,js->jrs", weights[j0:j1], phi[j0:j1], phi[j0:j1])
        V += np.einsum("ijx,jrs->ixrs", G, rho_j, optimize=True)
    return V


def intermediates(V, weights_i, phi_i, gamma):
    """The Appendix B intermediates for a batch of outer points.

    V: (ni, 3, N, N); weights_i: (ni,); phi_i: (ni, N).  Returns rho, A, B."""
    g = gamma
    rho = np.einsum("i,ip,iq->ipq", weights_i, phi_i, phi_i)
    W = 2.0 * np.einsum("ixtu,tu->ix", V, g)
    Vt = np.einsum("ix,ixrs->irs", W, V)
    X = np.einsum("ixts,tu->ixus", V, g)
    Zt = np.einsum("ixru,ixus->irs", V, X)
    A = Vt - Zt
    Wt = 2.0 * np.einsum("itu,tu->i", rho, g)
    Y = np.einsum("ixru,tu->ixrt", V, g)
    Z = np.einsum("iru,ixus->ixrs", rho, X) + np.einsum("ixrt,its->ixrs", Y, rho)
    B = 0.5 * Wt[:, None, None, None] * V - Z
    return rho, A, B


def assemble_dU(rho, A, V, B):
    """dU[p,q,r,s] = -sum_i (rho_pq A_rs + V_pq.B_rs + rho_rs A_pq + V_rs.B_pq)."""
    ni, n = rho.shape[0], rho.shape[1]
    f = rho.reshape(ni, n * n).T @ A.reshape(ni, n * n)
    f += V.transpose(1, 0, 2, 3).reshape(3 * ni, n * n).T @ B.transpose(1, 0, 2, 3).reshape(3 * ni, n * n)
    return -(f + f.T).reshape(n, n, n, n)


def onebody(dU, gamma):
    """Delta h_pq = -1/2 (2 Delta U_pr^qs gamma_rs - Delta U_pr^sq gamma_rs) (App. B)."""
    return -0.5 * (2.0 * np.einsum("pqrs,rs->pq", dU, gamma) - np.einsum("psrq,rs->pq", dU, gamma))


def constant(dh, gamma):
    """<Phi0|L|Phi0> = -2/3 Delta h_pq gamma_pq (App. B)."""
    return -2.0 / 3.0 * float(np.einsum("pq,pq->", dh, gamma))


def build(problem, gamma=None, outer=None, i_block=64, j_block=2048):
    """Delta U (N^4, dU[p,q,r,s] = (pq|rs)-ordered), Delta h (N x N) and the
    constant for ``problem`` (a synth.Problem).  ``outer``: optional index array
    of outer grid points; default all points."""
    p = problem
    g = p.gamma if gamma is None else np.asarray(gamma, dtype=np.float64)
    jas = (p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    idx = np.arange(p.n_grid) if outer is None else np.asarray(outer)
    n = p.n_orb
    dU = np.zeros((n, n, n, n))
    for b0 in range(0, len(idx), i_block):
        sel = idx[b0:b0 + i_block]
        V = vfield(p.grid, p.weights, p.phi, jas, sel, j_block)
        rho, A, B = intermediates(V, p.weights[sel], p.phi[sel], g)
        dU += assemble_dU(rho, A, V, B)
    dh = onebody(dU, g)
    return {"dU": dU, "dh": dh, "e0": constant(dh, g)}
