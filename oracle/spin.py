"""Route 2 for two spin densities: the restricted open-shell xTC working equations (oracle, FP64).

Test infrastructure only (see the package docstring).  Written from Appendix A ("Restricted
open-shell working equations"): both spins share the real spatial orbitals and the Jastrow
factor, so rho, V and everything built from them alone are spin-free; only the per-spin densities
gamma^a and gamma^b carry spin.  With g = gamma^a + gamma^b, and t, s in {a, b}:

    W(i)        = V_tu(i) g_tu                      Wt(i)      = rho_tu(i) g_tu
    Vt_rs(i)    = W(i) . V_rs(i)
    X^t_us(i)   = V_ks(i) gamma^t_ku                Zt^t_rs(i) = V_ru(i) . X^t_us(i)
    Y^t_rk(i)   = V_ru(i) gamma^t_ku                Z^t_rs(i)  = rho_ru(i) X^t_us(i) + Y^t_rk(i) rho_ks(i)
    A^t_rs(i)   = Vt_rs(i) - Zt^t_rs(i)             B^t_rs(i)  = 1/2 Wt(i) V_rs(i) - Z^t_rs(i)

    dU^{st}[p,q,r,s] = [Delta U_pr^qs]^{st}
                     = -sum_i (rho_pq A^t_rs + V_pq . B^t_rs + rho_rs A^s_pq + V_rs . B^s_pq)
    dh^s[p,q]   = -1/2 (sum_t [Delta U_pr^qs]^{st} gamma^t_rs - [Delta U_pr^sq]^{ss} gamma^s_rs)
    e0          = <Psi0|L|Psi0> = -1/3 sum_s dh^s_pq gamma^s_pq

Electron 1 (pair pq) has spin s, electron 2 (pair rs) spin t.  The symmetriser P^(pq s)_(rs t) is
read as identity + the exchange of (pq, s) with (rs, t), as for the closed-shell P^(pq)_(rs)
(it follows from eq. Ldecomp inserted in eq. dU, where the exchange terms of electron 2 carry
electron 2's spin density and those of electron 1 electron 1's).  dU^{ba}[p,q,r,s] =
dU^{ab}[r,s,p,q], so only the aa, ab and bb blocks are returned.  With gamma^a = gamma^b = gamma
every block equals the closed-shell Delta U of Appendix B, dh^a = dh^b its Delta h, and e0 its
constant.
"""
from __future__ import annotations

import numpy as np

from . import direct


def intermediates(V, weights_i, phi_i, gamma_a, gamma_b):
    """rho and, per spin t, (A^t, B^t) for a batch of outer points (Appendix A).

    V: (ni, 3, N, N); weights_i: (ni,); phi_i: (ni, N).  Returns rho, {"a": (A, B), "b": (A, B)}."""
    rho = np.einsum("i,ip,iq->ipq", weights_i, phi_i, phi_i)
    g = gamma_a + gamma_b
    W = np.einsum("ixtu,tu->ix", V, g)
    Vt = np.einsum("ix,ixrs->irs", W, V)
    Wt = np.einsum("itu,tu->i", rho, g)
    out = {}
    for spin, gt in (("a", gamma_a), ("b", gamma_b)):
        X = np.einsum("ixks,ku->ixus", V, gt)
        Zt = np.einsum("ixru,ixus->irs", V, X)
        Y = np.einsum("ixru,ku->ixrk", V, gt)
        Z = np.einsum("iru,ixus->ixrs", rho, X) + np.einsum("ixrk,iks->ixrs", Y, rho)
        out[spin] = (Vt - Zt, 0.5 * Wt[:, None, None, None] * V - Z)
    return rho, out


def _f(rho, V, A, B):
    """f[pq, rs] = sum_i (rho_pq A_rs + V_pq . B_rs), flattened pair indices."""
    ni, n = rho.shape[0], rho.shape[1]
    f = rho.reshape(ni, n * n).T @ A.reshape(ni, n * n)
    f += V.transpose(1, 0, 2, 3).reshape(3 * ni, n * n).T @ B.transpose(1, 0, 2, 3).reshape(3 * ni, n * n)
    return f


def onebody(dU_aa, dU_ab, dU_bb, gamma_a, gamma_b):
    """dh^a and dh^b of Appendix A from the three Delta U blocks."""
    dh_a = -0.5 * (np.einsum("pqrs,rs->pq", dU_aa, gamma_a) + np.einsum("pqrs,rs->pq", dU_ab, gamma_b)
                   - np.einsum("psrq,rs->pq", dU_aa, gamma_a))
    # dU^{ba}[p,q,r,s] = dU^{ab}[r,s,p,q]
    dh_b = -0.5 * (np.einsum("rspq,rs->pq", dU_ab, gamma_a) + np.einsum("pqrs,rs->pq", dU_bb, gamma_b)
                   - np.einsum("psrq,rs->pq", dU_bb, gamma_b))
    return dh_a, dh_b


def constant(dh_a, dh_b, gamma_a, gamma_b):
    """<Psi0|L|Psi0> = -1/3 sum_s dh^s_pq gamma^s_pq (Appendix A)."""
    return -1.0 / 3.0 * float(np.einsum("pq,pq->", dh_a, gamma_a) + np.einsum("pq,pq->", dh_b, gamma_b))


def build(problem, gamma_a, gamma_b, outer=None, i_block=64, j_block=2048):
    """Delta U^{aa}, Delta U^{ab}, Delta U^{bb} (each dU[p,q,r,s] = [Delta U_pr^qs]^{st}),
    Delta h^a, Delta h^b and the constant for ``problem`` and the two spin densities."""
    p = problem
    ga = np.asarray(gamma_a, dtype=np.float64)
    gb = np.asarray(gamma_b, dtype=np.float64)
    jas = (p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    idx = np.arange(p.n_grid) if outer is None else np.asarray(outer)
    n = p.n_orb
    fa = np.zeros((n * n, n * n))
    fb = np.zeros((n * n, n * n))
    for b0 in range(0, len(idx), i_block):
        sel = idx[b0:b0 + i_block]
        V = direct.vfield(p.grid, p.weights, p.phi, jas, sel, j_block)
        rho, AB = intermediates(V, p.weights[sel], p.phi[sel], ga, gb)
        fa += _f(rho, V, *AB["a"])
        fb += _f(rho, V, *AB["b"])
    shape = (n, n, n, n)
    dU_aa = -(fa + fa.T).reshape(shape)
    dU_ab = -(fb + fa.T).reshape(shape)      # electron 2 (rs) beta: f^b[pq, rs] + f^a[rs, pq]
    dU_bb = -(fb + fb.T).reshape(shape)
    dh_a, dh_b = onebody(dU_aa, dU_ab, dU_bb, ga, gb)
    return {"dU_aa": dU_aa, "dU_ab": dU_ab, "dU_bb": dU_bb, "dh_a": dh_a, "dh_b": dh_b,
            "e0": constant(dh_a, dh_b, ga, gb)}
