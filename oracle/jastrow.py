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
