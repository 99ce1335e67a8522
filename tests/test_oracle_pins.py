"""Pins of the CPU oracle against facts that do not come from the oracle itself:
calculus, the literal triple quadrature of the L definition, the paper's two
independent routes (explicit normal ordering vs. the Appendix B working
equations) and the identities it states between them, a closed form for a
separable Jastrow factor, and symmetry / homogeneity / covariance invariants."""
import numpy as np
import pytest

import synth
from oracle import bruteforce, direct, jastrow, spin


def _jas(p):
    return p.nuc_xyz, p.nuc_set, p.terms, p.coef


# ------------------------------------------------------------------ Jastrow gradient

@pytest.mark.parametrize("terms", [synth.CANONICAL_TERMS,
                                   np.array([(0, 2, 0), (1, 1, 0), (2, 2, 2), (0, 1, 1)])])
def test_grad1_matches_central_differences(terms):
    rng = np.random.default_rng(11)
    nuc = rng.uniform(-1.5, 1.5, size=(3, 3))
    nuc_set = np.array([0, 1, 0])
    coef = rng.uniform(-0.1, 0.1, size=(2, len(terms)))
    r1 = rng.uniform(-3, 3, size=(40, 3))
    r2 = rng.uniform(-3, 3, size=(40, 3))
    g = jastrow.grad1(r1, r2, nuc, nuc_set, terms, coef)
    h = 1e-5
    fd = np.zeros_like(g)
    for x in range(3):
        e = np.zeros(3)
        e[x] = h
        fd[:, x] = (jastrow.u_value(r1 + e, r2, nuc, nuc_set, terms, coef)
                    - jastrow.u_value(r1 - e, r2, nuc, nuc_set, terms, coef)) / (2 * h)
    assert np.abs(g - fd).max() < 1e-9 * max(1.0, np.abs(g).max())
    # u is symmetric in the two electrons
    assert np.allclose(jastrow.u_value(r1, r2, nuc, nuc_set, terms, coef),
                       jastrow.u_value(r2, r1, nuc, nuc_set, terms, coef), atol=1e-15)


def test_grad1_coincident_points_keep_only_electron_nucleus_part():
    nuc = np.array([[0.0, 0.0, 0.0]])
    r = np.array([0.3, -0.2, 0.5])
    ee = np.array([(0, 0, 1)])
    en = np.array([(0, 1, 0)])
    c = np.array([[0.07]])
    assert np.all(jastrow.grad1(r, r, nuc, [0], ee, c) == 0.0)
    # separable term c (a1 + a2): gradient a'(r) r_hat at coincidence as elsewhere
    d = np.linalg.norm(r)
    want = 0.07 / (1 + d) ** 2 * r / d
    assert np.allclose(jastrow.grad1(r, r, nuc, [0], en, c), want, rtol=1e-14)


# ------------------------------------------------------------------ L factorisation

def test_ldecomp_equals_literal_triple_quadrature():
    p = synth.make_small(n_orb=3, n_rad=3, n_theta=2, n_phi=3, n_atoms=2, seed=3)
    L1 = bruteforce.L_ldecomp(p)
    L2 = bruteforce.L_triple(p)
    assert np.abs(L1 - L2).max() < 1e-13 * np.abs(L2).max()
    # L is symmetric under permutations of the three electrons (pairs move together)
    assert np.allclose(L1, np.einsum("prtqsu->rptsqu", L1), atol=1e-16)
    assert np.allclose(L1, np.einsum("prtqsu->tpruqs", L1), atol=1e-16)


# ------------------------------------------------------------------ two routes

@pytest.mark.parametrize("dens", ["closed", "random"])
def test_route2_matches_explicit_normal_ordering(dens):
    p = synth.make_small(n_orb=4, n_rad=4, n_theta=3, n_phi=3, n_atoms=3, seed=21, n_occ=2)
    g = p.gamma if dens == "closed" else synth.random_density(4, 9)
    r1 = bruteforce.build(p, g)
    r2 = direct.build(p, g)
    scale = np.abs(r2["dU"]).max()
    assert scale > 1e-6
    assert np.abs(r1["dU"] - r2["dU"]).max() < 1e-12 * scale
    assert np.abs(r1["dh"] - r2["dh"]).max() < 1e-12 * scale
    assert abs(r1["e0"] - r2["e0"]) < 1e-12 * scale
    # the paper's identities inside Route 1
    assert np.abs(r1["dh_general"] - r1["dh"]).max() < 1e-12 * scale        # eq. (tcmf:1el)
    assert abs(r1["e0_rdm"] - r1["e0"]) < 1e-12 * scale                      # eq. (tcmf:0el)
    assert np.abs(r1["dU_ab"] - r1["dU"]).max() < 1e-14 * scale              # spin blocks agree
    assert np.abs(r1["dh_beta"] - r1["dh"]).max() < 1e-14 * scale


@pytest.mark.slow
def test_h2_config_routes_agree_to_1e10_hartree():
    p = synth.make_config("h2")
    r1 = bruteforce.build(p)
    r2 = direct.build(p)
    assert np.abs(r1["dU"] - r2["dU"]).max() < 1e-10
    assert np.abs(r1["dh"] - r2["dh"]).max() < 1e-10
    assert abs(r1["e0"] - r2["e0"]) < 1e-10
    assert abs(r1["e0_rdm"] - r2["e0"]) < 1e-10


# ------------------------------------------------------------------ closed form

def _separable_closed_form(p, g):
    """Separable u = g(r1) + g(r2) (terms (0, n, 0) only): nabla_1 u = nabla g(r1), so
    V_RS(i) = S_RS nabla g(r_i) with S the grid overlap, and eq. (Ldecomp) gives
    L = G_PQ S_RS S_TU + S_PQ G_RS S_TU + S_PQ S_RS G_TU, G_PQ = sum_i w phi_P phi_Q |nabla g|^2.
    Inserting this L in eq. (dU) and integrating over spin (closed shell, per-spin
    gamma) gives the expression below, derived by hand from eq. (dU)."""
    S = p.phi.T @ (p.weights[:, None] * p.phi)
    # nabla g(r) for g(r) = sum_I sum_t c (a^n) (+ a^0 a^n symmetrisation: c (a1^n + a2^n))
    grad = np.zeros((p.n_grid, 3))
    for I, R in enumerate(p.nuc_xyz):
        v = p.grid - R
        d = np.linalg.norm(v, axis=1)
        a = d / (1 + d)
        for t, (m, n, o) in enumerate(p.terms):
            assert m == 0 and o == 0
            c = p.coef[p.nuc_set[I], t]
            if n > 0:
                grad += (c * n * a ** (n - 1) / (1 + d) ** 2 / d)[:, None] * v
    G = p.phi.T @ ((p.weights * (grad ** 2).sum(1))[:, None] * p.phi)
    t = np.trace(S @ g)
    k = np.trace(G @ g)
    SgS, GgS, SgG = S @ g @ S, G @ g @ S, S @ g @ G
    E = np.einsum
    dU = -(2 * t * E("pq,rs->pqrs", G, S) + 2 * t * E("pq,rs->pqrs", S, G)
           + 2 * k * E("pq,rs->pqrs", S, S)
           - E("pq,rs->pqrs", G, SgS) - E("pq,rs->pqrs", SgS, G)
           - E("pq,rs->pqrs", S, GgS + SgG) - E("pq,rs->pqrs", GgS + SgG, S))
    return dU


def test_separable_jastrow_closed_form():
    terms = np.array([(0, 1, 0), (0, 2, 0)])
    p = synth.make_small(n_orb=5, n_rad=6, n_theta=3, n_phi=4, n_atoms=2, seed=4, terms=terms)
    g = synth.random_density(5, 3)
    want = _separable_closed_form(p, g)
    got = direct.build(p, g)["dU"]
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


# ------------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def small():
    p = synth.make_small(n_orb=5, n_rad=5, n_theta=3, n_phi=4, n_atoms=2, seed=8, n_occ=2)
    g = synth.random_density(5, 2)
    return p, g, direct.build(p, g)


def test_eightfold_symmetry_and_hermitian_onebody(small):
    _, _, r = small
    dU = r["dU"]
    s = np.abs(dU).max()
    for perm in ["qprs", "pqsr", "rspq", "srqp"]:
        assert np.abs(dU - np.einsum("pqrs->" + perm, dU)).max() < 1e-14 * s
    assert np.abs(r["dh"] - r["dh"].T).max() < 1e-14 * s


def test_homogeneity_and_zero_jastrow(small):
    p, g, r = small
    from dataclasses import replace
    r2 = direct.build(replace(p, coef=1.7 * p.coef), g)
    assert np.abs(r2["dU"] - 1.7 ** 2 * r["dU"]).max() < 1e-13 * np.abs(r["dU"]).max()
    r0 = direct.build(replace(p, coef=0 * p.coef), g)
    assert np.abs(r0["dU"]).max() == 0.0 and r0["e0"] == 0.0


def test_orbital_rotation_covariance(small):
    p, g, r = small
    from dataclasses import replace
    Q, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((p.n_orb, p.n_orb)))
    r2 = direct.build(replace(p, phi=p.phi @ Q), Q.T @ g @ Q)
    want = np.einsum("pqrs,pa,qb,rc,sd->abcd", r["dU"], Q, Q, Q, Q)
    assert np.abs(r2["dU"] - want).max() < 1e-13 * np.abs(want).max()
    assert np.abs(r2["dh"] - Q.T @ r["dh"] @ Q).max() < 1e-13 * np.abs(want).max()
    assert abs(r2["e0"] - r["e0"]) < 1e-13 * np.abs(want).max()


def test_grid_permutation_and_outer_split(small):
    p, g, r = small
    perm = np.random.default_rng(1).permutation(p.n_grid)
    r2 = direct.build(synth.permute_grid(p, perm), g)
    assert np.abs(r2["dU"] - r["dU"]).max() < 1e-14 * np.abs(r["dU"]).max() * 10
    half = p.n_grid // 3
    a = direct.build(p, g, outer=np.arange(half))
    b = direct.build(p, g, outer=np.arange(half, p.n_grid))
    assert np.abs(a["dU"] + b["dU"] - r["dU"]).max() < 1e-14 * np.abs(r["dU"]).max() * 10
    assert abs(a["e0"] + b["e0"] - r["e0"]) < 1e-15 + 1e-13 * abs(r["e0"])


# ------------------------------------------------------------------ planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped term, a wrong sign or a transposed operand in the Appendix B
    equations must break agreement with the explicit normal ordering."""
    p = synth.make_small(n_orb=3, n_rad=3, n_theta=2, n_phi=3, n_atoms=2, seed=3)
    g = synth.random_density(3, 6)
    want = bruteforce.build(p, g)["dU"]
    orig = direct.intermediates

    def dropped_Zt(V, w, phi, gamma):
        rho, A, B = orig(V, w, phi, gamma)
        Zt = np.einsum("ixru,ixus->irs", V, np.einsum("ixts,tu->ixus", V, gamma))
        return rho, A + Zt, B

    def wrong_half(V, w, phi, gamma):
        rho, A, B = orig(V, w, phi, gamma)
        Wt = 2.0 * np.einsum("i,ip,iq,pq->i", w, phi, phi, gamma)
        return rho, A, B + 0.5 * Wt[:, None, None, None] * V

    def transposed_product(V, w, phi, gamma):
        # Z_rs = rho_ru X_us + Y_rt rho_ts with the second product transposed
        rho, A, B = orig(V, w, phi, gamma)
        X = np.einsum("ixts,tu->ixus", V, gamma)
        Y = np.einsum("ixru,tu->ixrt", V, gamma)
        good = np.einsum("ixrt,its->ixrs", Y, rho)
        bad = np.einsum("its,ixrt->ixsr", rho, Y)
        return rho, A, B + good - bad

    for bad in (dropped_Zt, wrong_half, transposed_product):
        monkeypatch.setattr(direct, "intermediates", bad)
        got = direct.build(p, g)["dU"]
        assert np.abs(got - want).max() > 1e-6 * np.abs(want).max(), bad.__name__
    monkeypatch.setattr(direct, "intermediates", orig)
    assert np.abs(direct.build(p, g)["dU"] - want).max() < 1e-12 * np.abs(want).max()


# ------------------------------------------------------------------ two spin densities (Appendix A)

def _open_shell_densities(kind, n):
    if kind == "rohf":                       # 2 alpha, 1 beta occupied orbitals of one orbital set
        return np.diag([1.0, 1.0] + [0.0] * (n - 2)), np.diag([1.0] + [0.0] * (n - 1))
    return synth.random_density(n, 31), synth.random_density(n, 32, rank=2)


@pytest.mark.parametrize("kind", ["rohf", "random"])
def test_open_shell_route2_matches_explicit_normal_ordering(kind):
    """Appendix A against the spin-orbital definition (eq. dU, the general Delta h with the
    two-body density, the zero-body term with the three-body density) for unequal spin densities."""
    p = synth.make_small(n_orb=4, n_rad=4, n_theta=3, n_phi=3, n_atoms=3, seed=21)
    ga, gb = _open_shell_densities(kind, 4)
    r1 = bruteforce.build_spin(p, ga, gb)
    r2 = spin.build(p, ga, gb)
    scale = np.abs(r2["dU_aa"]).max()
    assert scale > 1e-6
    for k in ("dU_aa", "dU_ab", "dU_bb", "dh_a", "dh_b"):
        assert np.abs(r1[k] - r2[k]).max() < 1e-12 * scale, k
    assert abs(r1["e0"] - r2["e0"]) < 1e-12 * scale
    # the spin-summed one-body form equals the general one, and the constant its three-body form
    assert np.abs(r1["dh_general_a"] - r1["dh_a"]).max() < 1e-12 * scale
    assert np.abs(r1["dh_general_b"] - r1["dh_b"]).max() < 1e-12 * scale
    assert abs(r1["e0_rdm"] - r1["e0"]) < 1e-12 * scale
    assert np.abs(r1["dh_ab"]).max() == 0.0                                  # no spin-flip block
    assert np.abs(r1["dU_ba"] - r1["dU_ab"].transpose(2, 3, 0, 1)).max() < 1e-14 * scale
    # unequal densities give unequal blocks (the test would not see a spin mix-up otherwise)
    assert np.abs(r2["dU_aa"] - r2["dU_bb"]).max() > 1e-3 * scale
    assert np.abs(r2["dU_ab"] - r2["dU_aa"]).max() > 1e-3 * scale


def test_open_shell_equal_densities_reduce_to_closed_shell():
    """gamma^a = gamma^b: every block is the closed-shell Delta U of Appendix B."""
    p = synth.make_small(n_orb=4, n_rad=4, n_theta=3, n_phi=3, n_atoms=3, seed=21)
    g = synth.random_density(4, 9)
    c = direct.build(p, g)
    s2 = spin.build(p, g, g)
    scale = np.abs(c["dU"]).max()
    for k in ("dU_aa", "dU_ab", "dU_bb"):
        assert np.abs(s2[k] - c["dU"]).max() < 1e-13 * scale
    assert np.abs(s2["dh_a"] - c["dh"]).max() < 1e-13 * scale
    assert np.abs(s2["dh_b"] - c["dh"]).max() < 1e-13 * scale
    assert abs(s2["e0"] - c["e0"]) < 1e-13 * scale


def test_open_shell_blocks_average_to_closed_shell_of_mean_density():
    """Delta U is linear in the densities: (aa + bb) / 2 and the pair-symmetrised ab block both
    equal the closed-shell Delta U of the spin-averaged density (Appendix B as the spin average)."""
    p = synth.make_small(n_orb=4, n_rad=4, n_theta=3, n_phi=3, n_atoms=3, seed=21)
    ga, gb = synth.random_density(4, 9), synth.random_density(4, 10, rank=2)
    r = spin.build(p, ga, gb)
    c = direct.build(p, 0.5 * (ga + gb))
    scale = np.abs(c["dU"]).max()
    assert np.abs(0.5 * (r["dU_aa"] + r["dU_bb"]) - c["dU"]).max() < 1e-13 * scale
    assert np.abs(0.5 * (r["dU_ab"] + r["dU_ab"].transpose(2, 3, 0, 1)) - c["dU"]).max() < 1e-13 * scale
    assert np.abs(r["dU_ab"] - c["dU"]).max() > 1e-3 * scale       # the ab block alone is not


def test_open_shell_spin_flip(small):
    """Exchanging the two densities exchanges the spin labels of every output."""
    p, _, _ = small
    ga, gb = synth.random_density(p.n_orb, 41), synth.random_density(p.n_orb, 42, rank=1)
    r = spin.build(p, ga, gb)
    f = spin.build(p, gb, ga)
    scale = np.abs(r["dU_aa"]).max()
    assert np.abs(f["dU_aa"] - r["dU_bb"]).max() < 1e-13 * scale
    assert np.abs(f["dU_bb"] - r["dU_aa"]).max() < 1e-13 * scale
    assert np.abs(f["dU_ab"] - r["dU_ab"].transpose(2, 3, 0, 1)).max() < 1e-13 * scale
    assert np.abs(f["dh_a"] - r["dh_b"]).max() < 1e-13 * scale
    assert abs(f["e0"] - r["e0"]) < 1e-13 * scale


def test_open_shell_pins_catch_planted_mistakes(monkeypatch):
    """A direct term from one spin's density, the two spins' exchange terms interchanged, or a
    dropped half in B must break agreement with the spin-orbital definition."""
    p = synth.make_small(n_orb=3, n_rad=3, n_theta=2, n_phi=3, n_atoms=2, seed=3)
    ga, gb = synth.random_density(3, 6), synth.random_density(3, 7, rank=1)
    want = bruteforce.build_spin(p, ga, gb)
    orig = spin.intermediates

    def direct_from_alpha_only(V, w, phi, a, b):
        # exchange parts right, direct parts (W, Wt) from 2 gamma^a instead of gamma^a + gamma^b
        rho, good = orig(V, w, phi, a, b)
        Wd = np.einsum("ixtu,tu->ix", V, a - b)
        Wtd = np.einsum("itu,tu->i", rho, a - b)
        out = {}
        for s in ("a", "b"):
            A, B = good[s]
            out[s] = (A + np.einsum("ix,ixrs->irs", Wd, V), B + 0.5 * Wtd[:, None, None, None] * V)
        return rho, out

    def spins_interchanged(V, w, phi, a, b):
        rho, out = orig(V, w, phi, a, b)
        return rho, {"a": out["b"], "b": out["a"]}

    def dropped_half(V, w, phi, a, b):
        rho, out = orig(V, w, phi, a, b)
        Wt = np.einsum("itu,tu->i", rho, a + b)
        return rho, {s: (A, B + 0.5 * Wt[:, None, None, None] * V) for s, (A, B) in out.items()}

    for bad in (direct_from_alpha_only, spins_interchanged, dropped_half):
        monkeypatch.setattr(spin, "intermediates", bad)
        got = spin.build(p, ga, gb)
        worst = max(np.abs(got[k] - want[k]).max() / np.abs(want[k]).max() for k in ("dU_aa", "dU_ab", "dU_bb"))
        assert worst > 1e-6, bad.__name__
    monkeypatch.setattr(spin, "intermediates", orig)
    got = spin.build(p, ga, gb)
    assert max(np.abs(got[k] - want[k]).max() for k in ("dU_aa", "dU_ab", "dU_bb")) < 1e-12 * np.abs(want["dU_aa"]).max()


@pytest.mark.slow
def test_h2_config_open_shell_routes_agree_to_1e10_hartree():
    """The H2-like workload with one alpha and no beta electron: Appendix A against the
    spin-orbital definition (20 spin orbitals, 6.4e7 L entries)."""
    p = synth.make_config("h2")
    n = p.n_orb
    ga = np.diag([1.0] + [0.0] * (n - 1))
    gb = np.zeros((n, n))
    r1 = bruteforce.build_spin(p, ga, gb)
    r2 = spin.build(p, ga, gb)
    for k in ("dU_aa", "dU_ab", "dU_bb", "dh_a", "dh_b"):
        assert np.abs(r1[k] - r2[k]).max() < 1e-10, k
    assert abs(r1["e0"] - r2["e0"]) < 1e-10
    assert abs(r1["e0_rdm"] - r2["e0"]) < 1e-10
