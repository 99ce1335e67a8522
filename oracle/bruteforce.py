"""Route 1: explicit six-index L and explicit normal ordering (oracle, FP64).

For tiny inputs only.  Spatial L_prt^qsu is built either from eq. (Ldecomp),

    L_prt^qsu = sum_i w_i [ phi_p phi_q(i) V_rs(i).V_tu(i)
                          + phi_r phi_s(i) V_pq(i).V_tu(i)
                          + phi_t phi_u(i) V_pq(i).V_rs(i) ],

(the three placements of the centre electron that the symmetric permutation
operator P^1_{2,3} of the L definition produces), or from the literal triple
quadrature of the definition L_PRT^QSU = <PRT| P^1_{2,3}(nabla_1 u_12 .
nabla_1 u_13) |QSU> over grid points (i, j, k) for electrons (1, 2, 3).

Spin orbitals P = (p, sigma) carry spin-independent real orbitals and a
spin-independent Jastrow factor, so L_PRT^QSU = L_prt^qsu d(sP,sQ) d(sR,sS)
d(sT,sU), and the per-spin closed-shell density gives gamma_PQ =
gamma_pq d(sP,sQ).  Normal ordering then follows the Theory section as written:

    Delta U_PR^QS = -(L_PRT^QSU - L_PRT^QUS - L_PRT^USQ) gamma_TU               eq. (dU)
    Delta h_P^Q   = (L_PRT^QSU - L_PRT^SQU - L_PRT^USQ)
                    (gamma_RS gamma_TU - gamma_RU gamma_TS - 1/2 gamma^RT_SU)   (general Delta h)
    Delta h_P^Q   = -1/2 (Delta U_PR^QS - Delta U_PR^SQ) gamma_RS               eq. (tcmf:1el)
    <L>           = -1/6 L_PRT^QSU gamma^PRT_QSU                               (zero-body)
    <L>           = -1/3 Delta h_P^Q gamma_PQ                                  eq. (tcmf:0el)

with the determinant densities gamma^RT_SU and gamma^PRT_QSU the antisymmetrised
products of eq. (1Ddens).  Array layouts: L[p,r,t,q,s,u] = L_prt^qsu and
dU_so[P,R,Q,S] = Delta U_PR^QS.
"""
from __future__ import annotations

import numpy as np

from . import direct, jastrow


def L_ldecomp(problem, i_block=128):
    """Spatial L[p,r,t,q,s,u] from eq. (Ldecomp)."""
    p = problem
    n = p.n_orb
    jas = (p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    t1 = np.zeros((n * n, n ** 4))
    for b0 in range(0, p.n_grid, i_block):
        sel = np.arange(b0, min(b0 + i_block, p.n_grid))
        V = direct.vfield(p.grid, p.weights, p.phi, jas, sel)
        rho = np.einsum("i,ip,iq->ipq", p.weights[sel], p.phi[sel], p.phi[sel]).reshape(len(sel), n * n)
        vv = np.einsum("ixrs,ixtu->irstu", V, V).reshape(len(sel), n ** 4)
        t1 += rho.T @ vv
    t1 = t1.reshape(n, n, n, n, n, n)           # t1[p,q,r,s,t,u] = sum_i rho_pq V_rs.V_tu
    lpq = t1 + t1.transpose(2, 3, 0, 1, 4, 5) + t1.transpose(4, 5, 2, 3, 0, 1)
    return np.einsum("pqrstu->prtqsu", lpq)


def L_triple(problem):
    """Spatial L[p,r,t,q,s,u] by the literal triple grid sum (micro inputs)."""
    p = problem
    G = jastrow.grad1(p.grid[:, None, :], p.grid[None, :, :], p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    # f(1,2,3) + f(2,1,3) + f(3,2,1) with f(1,2,3) = nabla_1 u(1,2) . nabla_1 u(1,3),
    # electron 1 at point i, electron 2 at j, electron 3 at k.
    F = (np.einsum("ijx,ikx->ijk", G, G)
         + np.einsum("jix,jkx->ijk", G, G)
         + np.einsum("kjx,kix->ijk", G, G))
    d = np.einsum("i,ip,iq->ipq", p.weights, p.phi, p.phi)
    return np.einsum("ijk,ipq,jrs,ktu->prtqsu", F, d, d, d, optimize=True)


def spin_orbital(L, gamma, gamma_b=None):
    """Spin-orbital L_so[P,R,T,Q,S,U] and gamma_so; P = p + N * sigma.  gamma is the alpha
    density and gamma_b the beta one (default: the same, the closed-shell case)."""
    n = gamma.shape[0]
    gb = gamma if gamma_b is None else np.asarray(gamma_b, dtype=np.float64)
    idx = np.arange(2 * n) % n
    spin = np.arange(2 * n) // n
    D = (spin[:, None] == spin[None, :]).astype(np.float64)
    Lso = L[np.ix_(idx, idx, idx, idx, idx, idx)]
    Lso = Lso * D[:, None, None, :, None, None] * D[None, :, None, None, :, None] * D[None, None, :, None, None, :]
    gso = np.zeros((2 * n, 2 * n))
    gso[:n, :n] = gamma
    gso[n:, n:] = gb
    return Lso, gso


def normal_order(Lso, gso):
    """Delta U, Delta h (both forms) and <L> (both forms) in spin orbitals."""
    g = gso
    dU = -(np.einsum("prtqsu,tu->prqs", Lso, g)
           - np.einsum("prtqus,tu->prqs", Lso, g)
           - np.einsum("prtusq,tu->prqs", Lso, g))
    g2 = np.einsum("rs,tu->rtsu", g, g) - np.einsum("ru,ts->rtsu", g, g)      # gamma^RT_SU, eq. (1Ddens)
    K = np.einsum("rs,tu->rstu", g, g) - np.einsum("ru,ts->rstu", g, g) - 0.5 * g2.transpose(0, 2, 1, 3)
    dh_general = (np.einsum("prtqsu,rstu->pq", Lso, K)
                  - np.einsum("prtsqu,rstu->pq", Lso, K)
                  - np.einsum("prtusq,rstu->pq", Lso, K))
    dh_from_dU = -0.5 * (np.einsum("prqs,rs->pq", dU, g) - np.einsum("prsq,rs->pq", dU, g))
    # gamma^PRT_QSU = det [[g_PQ, g_PS, g_PU], [g_RQ, g_RS, g_RU], [g_TQ, g_TS, g_TU]]
    terms = [(+1, "pq,rs,tu"), (-1, "pq,ru,ts"), (-1, "ps,rq,tu"),
             (+1, "ps,ru,tq"), (+1, "pu,rq,ts"), (-1, "pu,rs,tq")]
    e_det = 0.0
    for sgn, spec in terms:
        e_det += sgn * float(np.einsum("prtqsu," + spec + "->", Lso, g, g, g, optimize=True))
    e_rdm = -e_det / 6.0
    e_from_dh = -float(np.einsum("pq,pq->", dh_from_dU, g)) / 3.0
    return {"dU": dU, "dh_general": dh_general, "dh_from_dU": dh_from_dU,
            "e_rdm": e_rdm, "e_from_dh": e_from_dh}


def closed_shell_blocks(res, n):
    """Spatial closed-shell views: dU[p,q,r,s] = Delta U_pr^qs (alpha alpha block),
    the alpha-beta block, Delta h^alpha and the total constant."""
    a = np.arange(n)
    b = a + n
    dU = res["dU"]
    dU_aa = dU[np.ix_(a, a, a, a)].transpose(0, 2, 1, 3)      # [P,R,Q,S] -> [p,q,r,s]
    dU_ab = dU[np.ix_(a, b, a, b)].transpose(0, 2, 1, 3)
    return {"dU": dU_aa, "dU_ab": dU_ab,
            "dh": res["dh_from_dU"][np.ix_(a, a)], "dh_general": res["dh_general"][np.ix_(a, a)],
            "dh_beta": res["dh_from_dU"][np.ix_(b, b)],
            "e0": res["e_from_dh"], "e0_rdm": res["e_rdm"]}


def spin_blocks(res, n):
    """Spatial views of the spin blocks: dU_st[p,q,r,s] = Delta U_pr^qs with p, q of spin s and
    r, s of spin t (s, t in {a, b}), Delta h^a and Delta h^b in both forms, and the constant in
    both forms."""
    a = np.arange(n)
    b = a + n
    dU = res["dU"]
    blk = lambda s1, s2: dU[np.ix_(s1, s2, s1, s2)].transpose(0, 2, 1, 3)    # [P,R,Q,S] -> [p,q,r,s]
    return {"dU_aa": blk(a, a), "dU_ab": blk(a, b), "dU_ba": blk(b, a), "dU_bb": blk(b, b),
            "dh_a": res["dh_from_dU"][np.ix_(a, a)], "dh_b": res["dh_from_dU"][np.ix_(b, b)],
            "dh_general_a": res["dh_general"][np.ix_(a, a)], "dh_general_b": res["dh_general"][np.ix_(b, b)],
            "dh_ab": res["dh_from_dU"][np.ix_(a, b)],
            "e0": res["e_from_dh"], "e0_rdm": res["e_rdm"]}


def build_spin(problem, gamma_a, gamma_b, L=None):
    """Route 1 with two spin densities: the spin blocks of the normal-ordered L."""
    if L is None:
        L = L_ldecomp(problem)
    Lso, gso = spin_orbital(L, np.asarray(gamma_a, dtype=np.float64), gamma_b)
    return spin_blocks(normal_order(Lso, gso), problem.n_orb)


def build(problem, gamma=None, L=None):
    """Route 1 end to end: spatial closed-shell blocks of the normal-ordered L."""
    g = problem.gamma if gamma is None else np.asarray(gamma, dtype=np.float64)
    if L is None:
        L = L_ldecomp(problem)
    Lso, gso = spin_orbital(L, g)
    return closed_shell_blocks(normal_order(Lso, gso), problem.n_orb)
