"""Frozen-core folding of the xTC corrections, xTC-FC (oracle, FP64).

Results section, "Frozen core approximation": in xTC-FC the xTC corrections to the integrals are
evaluated first for the whole orbital space, and the core orbitals are frozen afterwards with the
standard frozen-core equations.  For a set C of doubly occupied core orbitals (spin-restricted)
and an operator  sum_pq h_pq E_pq + 1/2 sum_pqrs U(pq|rs) e_pqrs  (chemist order, U with the 8-fold
symmetry of real orbitals, as Delta U of Appendix B has), freezing C leaves

    E_core      = sum_c 2 h_cc + sum_{c,d} [2 U(cc|dd) - U(cd|dc)]
    h^FC_pq     = h_pq + sum_c [2 U(pq|cc) - U(pc|cq)]            (p, q not in C)
    U^FC(pq|rs) = U(pq|rs)                                        (p, q, r, s not in C).

The folding is linear in (h, U), so the xTC parts (h = Delta h, U = Delta U) fold on their own;
a caller adds the folding of its own h and V - K.  With C = the occupied orbitals of the density
gamma = sum_{c in C} |c><c| these equations and Appendix B's Delta h give h^FC = -Delta h and
E_core = 0 for the xTC parts (tested).

Test infrastructure only: only the tests, the smoke entry point and the CPU baseline may import it.
"""
from __future__ import annotations

import numpy as np


def fold(dU, dh, core):
    """(dh_fc [n_act, n_act], e_core, active indices) for core index list ``core``."""
    dU = np.asarray(dU, dtype=np.float64)
    dh = np.asarray(dh, dtype=np.float64)
    n = dh.shape[0]
    core = np.asarray(sorted(set(int(c) for c in core)), dtype=np.int64)
    act = np.array([p for p in range(n) if p not in set(core.tolist())], dtype=np.int64)
    e_core = 0.0
    for c in core:
        e_core += 2.0 * dh[c, c]
        for d in core:
            e_core += 2.0 * dU[c, c, d, d] - dU[c, d, d, c]
    h = dh.copy()
    for c in core:
        h += 2.0 * dU[:, :, c, c] - dU[:, c, c, :]
    return h[np.ix_(act, act)], float(e_core), act
