"""Pins of the oracle for the two-body integrals K (Theory section) against facts from outside it:

* the Laplacian of u against central differences of u itself;
* the synthetic orbital gradients against differences of the orbitals;
* the whole of K against the similarity transformation it comes from: the operator
  nabla^2 u + (nabla u)^2 + 2 nabla u . nabla acting on f equals e^{-u} nabla^2 (e^{u} f) - nabla^2 f,
  so K can be formed from values of u and of analytic orbitals alone, with Laplacians taken by
  differences (no gradient formula, no orbital gradient, no index bookkeeping shared with the
  oracle);
* the coincident pair (j = i), which differences cannot reach, against a closed form of the
  reading on a one-point grid;
* the pair-swap symmetry that P12 gives, the split into the part linear and the part quadratic in
  the Jastrow coefficients, and K = 0 without a Jastrow factor;
* planted mistakes in the oracle's Jastrow derivatives fail the difference pin.
"""
import numpy as np
import pytest

import synth
from synth import molecules
from oracle import jastrow, two_body_k

TERMS_WITH_EN = np.array([(0, 2, 0), (1, 1, 0), (0, 1, 1), (1, 2, 1), (0, 0, 2), (2, 2, 2)])


def _random_jastrow(rng, terms, n_nuc=2, n_sets=2):
    nuc = rng.uniform(-1.2, 1.2, size=(n_nuc, 3))
    nuc_set = np.arange(n_nuc) % n_sets
    coef = rng.uniform(-0.15, 0.15, size=(n_sets, len(terms)))
    return nuc, nuc_set, np.asarray(terms), coef


# ------------------------------------------------------------------ Laplacian of u

@pytest.mark.parametrize("terms", [synth.CANONICAL_TERMS, TERMS_WITH_EN])
def test_lap1_matches_central_differences(terms):
    rng = np.random.default_rng(5)
    jas = _random_jastrow(rng, terms, n_nuc=3)
    r1 = rng.uniform(-3, 3, size=(60, 3))
    r2 = rng.uniform(-3, 3, size=(60, 3))

    def second_difference(h):
        out = -6.0 * jastrow.u_value(r1, r2, *jas)
        for x in range(3):
            e = np.zeros(3)
            e[x] = h
            out = out + jastrow.u_value(r1 + e, r2, *jas) + jastrow.u_value(r1 - e, r2, *jas)
        return out / h ** 2

    fd = (4.0 * second_difference(5e-4) - second_difference(1e-3)) / 3.0  # Richardson
    lap = jastrow.lap1(r1, r2, *jas)
    assert np.abs(lap - fd).max() < 1e-7 * max(1.0, np.abs(lap).max())


def test_synthetic_orbital_gradients_match_differences():
    p = synth.make_small(n_orb=5, n_rad=3, n_theta=2, n_phi=3, n_atoms=3, seed=2)
    d = synth.orbital_gradients(p)
    assert d.shape == (p.n_grid, p.n_orb, 3)
    chi = molecules.basis_values(p.grid, p.nuc_xyz, p.shells)
    assert np.abs(chi @ p.orb_coef - p.phi).max() < 1e-12 * np.abs(p.phi).max()
    h = 1e-5
    for x in range(3):
        e = np.zeros(3)
        e[x] = h
        fp = molecules.basis_values(p.grid + e, p.nuc_xyz, p.shells) @ p.orb_coef
        fm = molecules.basis_values(p.grid - e, p.nuc_xyz, p.shells) @ p.orb_coef
        assert np.abs((fp - fm) / (2 * h) - d[:, :, x]).max() < 1e-6 * max(1.0, np.abs(d).max())


# ------------------------------------------------------------------ K from the similarity transformation

class _Orbitals:
    """Analytic functions (r - C)^e exp(-alpha |r - C|^2) with their gradients."""

    def __init__(self, rng, n):
        self.C = rng.uniform(-1.0, 1.0, size=(n, 3))
        self.e = rng.integers(0, 2, size=(n, 3))
        self.alpha = rng.uniform(0.3, 0.8, size=n)

    def value(self, k, r):
        d = r - self.C[k]
        poly = np.prod(d ** self.e[k], axis=-1)
        return poly * np.exp(-self.alpha[k] * np.sum(d * d, axis=-1))

    def grad(self, k, r):
        d = r - self.C[k]
        g = np.exp(-self.alpha[k] * np.sum(d * d, axis=-1))
        out = []
        for x in range(3):
            ex = self.e[k, x]
            dx = (ex * d[..., x] ** (ex - 1) if ex > 0 else 0.0) - 2 * self.alpha[k] * d[..., x] ** (ex + 1)
            others = np.prod([d[..., y] ** self.e[k, y] for y in range(3) if y != x], axis=0)
            out.append(dx * others * g)
        return np.stack(out, axis=-1)


def _separated_points(rng, n, nuc, min_dist=0.3):
    pts = []
    while len(pts) < n:
        r = rng.uniform(-2.0, 2.0, size=3)
        if all(np.linalg.norm(r - q) > min_dist for q in pts) and all(np.linalg.norm(r - R) > min_dist for R in nuc):
            pts.append(r)
    return np.array(pts)


def _laplacian_by_differences(fun, r, h=1e-3):
    def second_difference(hh):
        out = -6.0 * fun(r)
        for x in range(3):
            e = np.zeros(3)
            e[x] = hh
            out = out + fun(r + e) + fun(r - e)
        return out / hh ** 2
    return (4.0 * second_difference(h / 2) - second_difference(h)) / 3.0


def _k_by_similarity_transform(grid, w, orbs, n_orb, jas):
    """K from values of u and of the orbitals only: the operator of K acting on f is
    e^{-u} nabla^2 (e^{u} f) - nabla^2 f, applied to electron 1 (f(1,2) of P12) and to electron 2
    (f(2,1)), with the Laplacians by Richardson-extrapolated second differences."""
    n = len(grid)
    ri = np.broadcast_to(grid[:, None, :], (n, n, 3)).copy()
    rj = np.broadcast_to(grid[None, :, :], (n, n, 3)).copy()
    eu = np.exp(-jastrow.u_value(ri, rj, *jas))
    phi = np.stack([orbs.value(k, grid) for k in range(n_orb)], axis=1)
    T1 = np.zeros((n, n, n_orb))  # operator on electron 1 (at r_i) acting on phi_q
    T2 = np.zeros((n, n, n_orb))  # operator on electron 2 (at r_j) acting on phi_s
    for k in range(n_orb):
        on1 = _laplacian_by_differences(lambda r: np.exp(jastrow.u_value(r, rj, *jas)) * orbs.value(k, r), ri)
        T1[:, :, k] = eu * on1 - _laplacian_by_differences(lambda r: orbs.value(k, r), ri)
        on2 = _laplacian_by_differences(lambda r: np.exp(jastrow.u_value(ri, r, *jas)) * orbs.value(k, r), rj)
        T2[:, :, k] = eu * on2 - _laplacian_by_differences(lambda r: orbs.value(k, r), rj)
    off = 1.0 - np.eye(n)  # coincident pairs contribute nothing
    W = np.outer(w, w) * off
    K = 0.5 * (np.einsum("ij,ip,jr,ijq,js->pqrs", W, phi, phi, T1, phi)
               + np.einsum("ij,ip,jr,iq,ijs->pqrs", W, phi, phi, phi, T2))
    return K, phi


def _case(seed, terms, n=18, n_orb=3):
    rng = np.random.default_rng(seed)
    jas = _random_jastrow(rng, terms)
    grid = _separated_points(rng, n, jas[0])
    w = rng.uniform(0.5, 1.5, size=n)
    orbs = _Orbitals(rng, n_orb)
    dphi = np.stack([orbs.grad(k, grid) for k in range(n_orb)], axis=1)
    return grid, w, orbs, n_orb, jas, dphi


def _fd_error(seed, terms):
    grid, w, orbs, n_orb, jas, dphi = _case(seed, terms)
    K_fd, phi = _k_by_similarity_transform(grid, w, orbs, n_orb, jas)
    K = two_body_k.k_integrals(grid, w, phi, dphi, *jas, coincident=False)
    return np.abs(K - K_fd).max() / np.abs(K_fd).max()


@pytest.mark.parametrize("seed,terms", [(1, synth.CANONICAL_TERMS), (2, TERMS_WITH_EN)])
def test_k_matches_similarity_transform_by_differences(seed, terms):
    assert _fd_error(seed, terms) < 1e-6


def test_k_pins_catch_planted_mistakes(monkeypatch):
    lap, grad = jastrow.lap1, jastrow.grad1
    assert _fd_error(1, synth.CANONICAL_TERMS) < 1e-6
    # the Laplacian at half its value
    monkeypatch.setattr(jastrow, "lap1", lambda *a: 0.5 * lap(*a))
    assert _fd_error(1, synth.CANONICAL_TERMS) > 1e-3
    monkeypatch.setattr(jastrow, "lap1", lap)
    # wrong sign of the gradient (the square is unchanged, the derivative term flips)
    monkeypatch.setattr(jastrow, "grad1", lambda *a: -grad(*a))
    assert _fd_error(1, synth.CANONICAL_TERMS) > 1e-3
    monkeypatch.setattr(jastrow, "grad1", grad)
    # the swapped term f(2,1) evaluated like f(1,2) (electron 1 in u's first slot both times)
    real = two_body_k._pair_fields
    calls = []

    def same_slot(first, second, jas):
        calls.append(1)
        return real(first, second, jas) if len(calls) % 2 == 1 else real(second, first, jas)
    monkeypatch.setattr(two_body_k, "_pair_fields", same_slot)
    assert _fd_error(1, synth.CANONICAL_TERMS) > 1e-3


def test_k_coincident_pair_reading_closed_form():
    """One grid point r, one nucleus at the origin, u = c1 (a1 + a2) + 2 c2 b (terms (0,1,0) and
    (0,0,1)).  At the coincident pair the electron-electron unit vector and 1/r12 are 0 while the
    rest is kept: grad_1 u = c1 a'(d) r/d, and with b = 0, b' = 1, b'' = -2,
        F = lap_1 u + |grad_1 u|^2 = c1 (a'' + 2 a'/d) - 4 c2 + c1^2 a'^2,
    so K[p,q,r,s] = w^2 phi_p phi_r [F phi_q phi_s + (g . dphi_q) phi_s + phi_q (g . dphi_s)]."""
    rng = np.random.default_rng(4)
    r = np.array([[0.48, 0.0, 0.64]])
    d = 0.8
    c1, c2, w = 0.13, -0.07, np.array([0.7])
    terms = np.array([(0, 1, 0), (0, 0, 1)])
    phi = rng.uniform(-1, 1, size=(1, 3))
    dphi = rng.uniform(-1, 1, size=(1, 3, 3))
    K = two_body_k.k_integrals(r, w, phi, dphi, np.zeros((1, 3)), [0], terms, np.array([[c1, c2]]))
    ap, app = 1 / (1 + d) ** 2, -2 / (1 + d) ** 3
    g = c1 * ap * r[0] / d
    F = c1 * (app + 2 * ap / d) - 4 * c2 + c1 ** 2 * ap ** 2
    f, gd = phi[0], dphi[0] @ g
    want = w[0] ** 2 * (F * np.einsum("p,q,r,s->pqrs", f, f, f, f)
                        + np.einsum("p,q,r,s->pqrs", f, gd, f, f) + np.einsum("p,q,r,s->pqrs", f, f, f, gd))
    assert np.abs(K - want).max() < 1e-14 * np.abs(want).max()
    assert np.all(two_body_k.k_integrals(r, w, phi, dphi, np.zeros((1, 3)), [0], terms, np.array([[c1, c2]]),
                                         coincident=False) == 0.0)


def test_k_symmetries_and_jastrow_dependence():
    grid, w, orbs, n_orb, jas, dphi = _case(3, synth.CANONICAL_TERMS, n=14, n_orb=3)
    phi = np.stack([orbs.value(k, grid) for k in range(n_orb)], axis=1)
    nuc, nuc_set, terms, coef = jas
    K = two_body_k.k_integrals(grid, w, phi, dphi, nuc, nuc_set, terms, coef)
    # P12 makes K symmetric under the exchange of the two electrons' index pairs ...
    assert np.abs(K - K.transpose(2, 3, 0, 1)).max() < 1e-13 * np.abs(K).max()
    # ... but not hermitian: the derivative term acts on the ket only
    assert np.abs(K - K.transpose(1, 0, 3, 2)).max() > 1e-3 * np.abs(K).max()
    # linear part (Laplacian, derivative) plus quadratic part (square) in the coefficients
    Km = two_body_k.k_integrals(grid, w, phi, dphi, nuc, nuc_set, terms, -coef)
    K2 = two_body_k.k_integrals(grid, w, phi, dphi, nuc, nuc_set, terms, 2 * coef)
    lin, quad = 0.5 * (K - Km), 0.5 * (K + Km)
    assert np.abs(K2 - (2 * lin + 4 * quad)).max() < 1e-12 * np.abs(K2).max()
    assert np.abs(quad).max() > 1e-4 * np.abs(lin).max()
    # no Jastrow factor, no K
    K0 = two_body_k.k_integrals(grid, w, phi, dphi, nuc, nuc_set, terms, 0 * coef)
    assert np.all(K0 == 0.0)
