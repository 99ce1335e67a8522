"""Jastrow factor of the build and its first-electron gradient (oracle, FP64).

The factor is a sum over nuclei I (nucleus I uses the coefficients of its
centre set) and terms t = (m, n, o):

    u(r1, r2) = sum_I sum_t c[set(I), t] (a1^m a2^n + a1^n a2^m) b^o,
    a_k = |r_k - R_I| / (1 + |r_k - R_I|),   b = r12 / (1 + r12).

The three-body integral L of the paper is built from nabla_1 u(r1, r2), the
gradient with respect to the first argument (Theory, definition of L; the
intermediate V of the "Decomposition of two-body correction" section uses the
same gradient with the outer grid point in the first slot).  By the chain rule

    nabla_1 u = sum_I sum_t c [ (m a1^(m-1) a2^n + n a1^(n-1) a2^m) b^o ] a'(r1I) (r1 - R_I)/r1I
              + sum_I sum_t c [ (a1^m a2^n + a1^n a2^m) o b^(o-1) ] b'(r12) (r1 - r2)/r12,

with a'(r) = b'(r) = 1/(1 + r)^2.  Readings where the paper is silent: the unit
vector (r1 - R_I)/r1I is taken as 0 when r1I < 1e-14 bohr, and the electron-
electron unit vector (r1 - r2)/r12 as 0 when r12 < 1e-14 bohr (this covers the
diagonal j = i of the grid sums); the electron-nucleus part is kept there.
"""
from __future__ import annotations

import numpy as np

EPS = 1e-14


def _pow(a, k):
    return np.ones_like(a) if k == 0 else a ** k


def _dpow(a, k):
    """d/da a^k."""
    return np.zeros_like(a) if k == 0 else k * _pow(a, k - 1)


def _ddpow(a, k):
    """d^2/da^2 a^k."""
    return np.zeros_like(a) if k < 2 else k * (k - 1) * _pow(a, k - 2)


def u_value(r1, r2, nuc_xyz, nuc_set, terms, coef):
    """u(r1, r2) for broadcastable (..., 3) arrays."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    r12 = np.linalg.norm(r1 - r2, axis=-1)
    b = r12 / (1.0 + r12)
    u = np.zeros(np.broadcast_shapes(r1.shape[:-1], r2.shape[:-1]))
    for I, R in enumerate(np.asarray(nuc_xyz, dtype=np.float64)):
        d1 = np.linalg.norm(r1 - R, axis=-1)
        d2 = np.linalg.norm(r2 - R, axis=-1)
        a1 = d1 / (1.0 + d1)
        a2 = d2 / (1.0 + d2)
        for t, (m, n, o) in enumerate(terms):
            c = coef[nuc_set[I], t]
            u = u + c * (_pow(a1, m) * _pow(a2, n) + _pow(a1, n) * _pow(a2, m)) * _pow(b, o)
    return u


def grad1(r1, r2, nuc_xyz, nuc_set, terms, coef):
    """nabla_1 u(r1, r2), shape broadcast(r1, r2)[:-1] + (3,)."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    d12 = r1 - r2
    r12 = np.linalg.norm(d12, axis=-1)
    b = r12 / (1.0 + r12)
    bp = 1.0 / (1.0 + r12) ** 2
    safe12 = np.where(r12 < EPS, 1.0, r12)
    e12 = np.where((r12 < EPS)[..., None], 0.0, d12 / safe12[..., None])
    shape = np.broadcast_shapes(r1.shape[:-1], r2.shape[:-1])
    g = np.zeros(shape + (3,))
    for I, R in enumerate(np.asarray(nuc_xyz, dtype=np.float64)):
        v1 = r1 - R
        d1 = np.linalg.norm(v1, axis=-1)
        d2 = np.linalg.norm(r2 - R, axis=-1)
        a1 = d1 / (1.0 + d1)
        a2 = d2 / (1.0 + d2)
        ap1 = 1.0 / (1.0 + d1) ** 2
        safe1 = np.where(d1 < EPS, 1.0, d1)
        e1 = np.where((d1 < EPS)[..., None], 0.0, v1 / safe1[..., None])
        for t, (m, n, o) in enumerate(terms):
            c = coef[nuc_set[I], t]
            # derivative through a1 (electron-nucleus distance of electron 1)
            da = c * (_dpow(a1, m) * _pow(a2, n) + _dpow(a1, n) * _pow(a2, m)) * _pow(b, o)
            # derivative through b (electron-electron distance)
            db = c * (_pow(a1, m) * _pow(a2, n) + _pow(a1, n) * _pow(a2, m)) * _dpow(b, o)
            g = g + (da * ap1)[..., None] * e1 + (db * bp)[..., None] * e12
    return g


def lap1(r1, r2, nuc_xyz, nuc_set, terms, coef):
    """nabla_1^2 u(r1, r2), the Laplacian with respect to the first argument (the two-body
    integrals K of the Theory section hold it beside (nabla_1 u)^2).

    Each term is P(a1) Q(b) with P = c (a1^m a2^n + a1^n a2^m) and Q = b^o, so
        nabla_1^2 (P Q) = Q nabla^2 P + P nabla^2 Q + 2 nabla P . nabla Q,
    and for a function f(a(r)) of one distance r = |r1 - X| (a = r / (1 + r))
        nabla^2 f = f_aa a'^2 + f_a (a'' + 2 a' / r),   a' = (1 + r)^-2,  a'' = -2 (1 + r)^-3,
        nabla P . nabla Q = P_a a'(r1I) Q_b a'(r12) e1I . e12 (unit vectors).
    Readings as for grad1: a unit vector and the 2 a'/r term are taken as 0 when their distance
    is below 1e-14 bohr."""
    r1 = np.asarray(r1, dtype=np.float64)
    r2 = np.asarray(r2, dtype=np.float64)
    d12 = r1 - r2
    r12 = np.linalg.norm(d12, axis=-1)
    small12 = r12 < EPS
    safe12 = np.where(small12, 1.0, r12)
    inv12 = np.where(small12, 0.0, 1.0 / safe12)
    e12 = d12 * inv12[..., None]
    b = r12 / (1.0 + r12)
    bp = 1.0 / (1.0 + r12) ** 2
    bpp = -2.0 / (1.0 + r12) ** 3
    shape = np.broadcast_shapes(r1.shape[:-1], r2.shape[:-1])
    lap = np.zeros(shape)
    for I, R in enumerate(np.asarray(nuc_xyz, dtype=np.float64)):
        v1 = r1 - R
        d1 = np.linalg.norm(v1, axis=-1)
        small1 = d1 < EPS
        inv1 = np.where(small1, 0.0, 1.0 / np.where(small1, 1.0, d1))
        e1 = v1 * inv1[..., None]
        d2 = np.linalg.norm(r2 - R, axis=-1)
        a1 = d1 / (1.0 + d1)
        a2 = d2 / (1.0 + d2)
        ap = 1.0 / (1.0 + d1) ** 2
        app = -2.0 / (1.0 + d1) ** 3
        cos = np.sum(e1 * e12, axis=-1)
        for t, (m, n, o) in enumerate(terms):
            c = coef[nuc_set[I], t]
            P = c * (_pow(a1, m) * _pow(a2, n) + _pow(a1, n) * _pow(a2, m))
            Pa = c * (_dpow(a1, m) * _pow(a2, n) + _dpow(a1, n) * _pow(a2, m))
            Paa = c * (_ddpow(a1, m) * _pow(a2, n) + _ddpow(a1, n) * _pow(a2, m))
            Q, Qb, Qbb = _pow(b, o), _dpow(b, o), _ddpow(b, o)
            lapP = Paa * ap ** 2 + Pa * (app + 2.0 * ap * inv1)
            lapQ = Qbb * bp ** 2 + Qb * (bpp + 2.0 * bp * inv12)
            lap = lap + Q * lapP + P * lapQ + 2.0 * (Pa * ap) * (Qb * bp) * cos
    return lap
