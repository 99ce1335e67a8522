"""Pins of the frozen-core folding oracle (xTC-FC, Results section "Frozen core approximation").

The folded one- and two-body parts and the core energy are compared with matrix elements of the
second-quantised operator  sum h_pq E_pq + 1/2 sum U(pq|rs) e_pqrs  evaluated determinant by
determinant in a small Fock space: with the core spin orbitals filled, <C|H|C> is the core energy,
<C; p up|H|C; q up> adds the folded one-body part and <C; p up, r down|H|C; q up, s down> adds the
two-body part.  Nothing of the folding formula enters that evaluation."""
import numpy as np
import pytest

import synth
from oracle import direct, frozen_core


def _sym8(a):
    perms = ["pqrs", "qprs", "pqsr", "qpsr", "rspq", "srpq", "rsqp", "srqp"]
    return sum(np.einsum("pqrs->" + p, a) for p in perms) / 8.0


def _random_operator(n, seed, hermitian=True):
    """Random (U, h): 8-fold symmetric U and symmetric h, or (hermitian=False) U with only the
    pair symmetry U(pq|rs) = U(rs|pq) and a non-symmetric h, as a transcorrelated V - K has."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((n, n))
    a = rng.standard_normal((n, n, n, n))
    if hermitian:
        return _sym8(a), 0.5 * (h + h.T)
    return 0.5 * (a + a.transpose(2, 3, 0, 1)), h


# ---------------------------------------------------------------- Fock space, one determinant at a time

def _apply(op, orb, det):
    """a+_orb (op = +1) or a_orb (op = -1) on a determinant given as an occupation bit mask;
    returns (sign, new mask) or None.  Spin orbitals are ordered by bit index."""
    occ = (det >> orb) & 1
    if (op > 0 and occ) or (op < 0 and not occ):
        return None
    sign = -1.0 if bin(det & ((1 << orb) - 1)).count("1") % 2 else 1.0
    return sign, det ^ (1 << orb)


def _string(ops, det):
    """Applies a right-to-left operator string [(op, orb), ...] (rightmost acts first)."""
    sign = 1.0
    for op, orb in reversed(ops):
        r = _apply(op, orb, det)
        if r is None:
            return None
        s, det = r
        sign *= s
    return sign, det


def _h_on(h, U, det):
    """H |det> as {mask: amplitude}, spin orbital of (p, spin) = 2 p + spin."""
    n = h.shape[0]
    out = {}

    def add(res, c):
        if res is not None and c != 0.0:
            out[res[1]] = out.get(res[1], 0.0) + c * res[0]

    for p in range(n):
        for q in range(n):
            for s in (0, 1):
                add(_string([(1, 2 * p + s), (-1, 2 * q + s)], det), h[p, q])
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for t in range(n):
                    c = 0.5 * U[p, q, r, t]
                    if c == 0.0:
                        continue
                    for s1 in (0, 1):
                        for s2 in (0, 1):
                            # e_pqrs = sum a+_p s1 a+_r s2 a_s s2 a_q s1
                            add(_string([(1, 2 * p + s1), (1, 2 * r + s2), (-1, 2 * t + s2), (-1, 2 * q + s1)], det), c)
    return out


def _core_mask(core):
    m = 0
    for c in core:
        m |= 3 << (2 * c)
    return m


def _state(ops, core):
    """(sign, mask) of the operator string ``ops`` applied to the filled core."""
    return _string(ops, _core_mask(core))


def _matrix_element(h, U, core, bra_ops, ket_ops):
    sb, mb = _state(bra_ops, core)
    sk, mk = _state(ket_ops, core)
    return sb * sk * _h_on(h, U, mk).get(mb, 0.0)


@pytest.mark.parametrize("n,core,seed,hermitian", [(4, [1], 3, True), (5, [0, 3], 4, True), (4, [], 5, True),
                                                  (4, [2], 6, False), (5, [1, 4], 7, False)])
def test_fold_matches_fock_space_matrix_elements(n, core, seed, hermitian):
    U, h = _random_operator(n, seed, hermitian)
    h_fc, e_core, act = frozen_core.fold(U, h, core)
    assert abs(_matrix_element(h, U, core, [], []) - e_core) < 1e-12 * (1 + abs(e_core))
    up = lambda p: (1, 2 * p)
    dn = lambda p: (1, 2 * p + 1)
    for a, p in enumerate(act):
        for b, q in enumerate(act):
            got = _matrix_element(h, U, core, [up(p)], [up(q)])
            want = h_fc[a, b] + (e_core if p == q else 0.0)
            assert abs(got - want) < 1e-12 * (1 + abs(want)), (p, q)
    # two-body part: a+_{p up} a+_{r down} |C> against a+_{q up} a+_{s down} |C>
    for a, p in enumerate(act):
        for b, q in enumerate(act):
            for c, r in enumerate(act):
                for d, s in enumerate(act):
                    got = _matrix_element(h, U, core, [up(p), dn(r)], [up(q), dn(s)])
                    want = U[p, q, r, s] + h_fc[a, b] * (r == s) + h_fc[c, d] * (p == q)
                    want += e_core * (p == q) * (r == s)
                    assert abs(got - want) < 1e-12 * (1 + abs(want)), (p, q, r, s)


def test_fock_space_pin_catches_planted_mistakes():
    """Plausible slips in the folding (exchange sign, Coulomb factor, one-body factor of the core
    energy, Coulomb and exchange indices swapped) each break agreement with the Fock space."""
    n, core = 4, [0, 2]
    U, h = _random_operator(n, 11)
    act = [1, 3]
    e_true = _matrix_element(h, U, core, [], [])
    want = np.array([[_matrix_element(h, U, core, [(1, 2 * p)], [(1, 2 * q)]) - (e_true if p == q else 0.0)
                      for q in act] for p in act])

    def variant(kind):
        hh = h.copy()
        e = 0.0
        for x in core:
            e += (1.0 if kind == "half_h" else 2.0) * h[x, x]
            for y in core:
                e += 2.0 * U[x, x, y, y] - U[x, y, y, x]
            if kind == "exchange_sign":
                hh += 2.0 * U[:, :, x, x] + U[:, x, x, :]
            elif kind == "coulomb_factor":
                hh += U[:, :, x, x] - U[:, x, x, :]
            elif kind == "swapped":
                hh += 2.0 * U[:, x, x, :] - U[:, :, x, x]
            else:
                hh += 2.0 * U[:, :, x, x] - U[:, x, x, :]
        return hh[np.ix_(act, act)], e

    h_ok, e_ok = variant("none")
    assert np.abs(h_ok - want).max() < 1e-12 and abs(e_ok - e_true) < 1e-12
    for kind in ("exchange_sign", "coulomb_factor", "swapped"):
        hb, _ = variant(kind)
        assert np.abs(hb - want).max() > 1e-3, kind
    _, eb = variant("half_h")
    assert abs(eb - e_true) > 1e-3


@pytest.fixture(scope="module")
def xtc_small():
    p = synth.make_small(n_orb=5, n_rad=5, n_theta=3, n_phi=4, n_atoms=2, seed=8, n_occ=2)
    g = np.diag([1.0, 1.0, 0.0, 0.0, 0.0])
    return p, g, direct.build(p, g)


def test_freezing_the_occupied_orbitals_negates_delta_h(xtc_small):
    """With the core equal to the occupied orbitals of gamma, Appendix B's Delta h is -1/2 of the
    core fold of Delta U, so the folded one-body part is -Delta h and the core energy vanishes."""
    _, _, r = xtc_small
    h_fc, e_core, act = frozen_core.fold(r["dU"], r["dh"], [0, 1])
    s = np.abs(r["dh"]).max()
    assert np.abs(h_fc + r["dh"][np.ix_(act, act)]).max() < 1e-13 * s
    assert abs(e_core) < 1e-13 * s


def test_empty_core_and_linearity(xtc_small):
    _, _, r = xtc_small
    h0, e0, act = frozen_core.fold(r["dU"], r["dh"], [])
    assert e0 == 0.0 and list(act) == list(range(5)) and np.array_equal(h0, r["dh"])
    U2, h2 = _random_operator(5, 21)
    a = frozen_core.fold(r["dU"], r["dh"], [1, 4])
    b = frozen_core.fold(U2, h2, [1, 4])
    ab = frozen_core.fold(r["dU"] + 0.3 * U2, r["dh"] + 0.3 * h2, [1, 4])
    assert np.abs(ab[0] - (a[0] + 0.3 * b[0])).max() < 1e-13 * (np.abs(ab[0]).max() + 1)
    assert abs(ab[1] - (a[1] + 0.3 * b[1])) < 1e-13 * (abs(ab[1]) + 1)
