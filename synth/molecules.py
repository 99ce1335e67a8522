"""Seeded synthetic molecules for the xTC grid build.

Each configuration gives nuclei, an atom-centred quadrature grid with Becke
partition weights, real molecular orbitals that are orthonormal on that grid,
a closed-shell per-spin density gamma and Jastrow parameters.  The recipes
follow the workloads the build is measured on:

* ``h2``    : 2 H at z = +-0.7 bohr, 16 Gaussians (per atom s: 13.0, 1.96,
              0.44, 0.12, 0.03; one p shell 0.73), N = 10, 2 x (20 radial x
              50 angular) = 2,000 points, one Jastrow centre set, 1 occupied.
* ``water`` : O at the origin, H at (0, +-1.43, 1.11), N = 58 from a 58-function
              s/p/d basis, 40,000 points, one centre set per nucleus, 5 occupied.
* ``n2``    : diatomic at 2.07 bohr, N = 120, 100,000 points, one centre set per
              nucleus, 7 occupied.
* ``large`` : 4 heavy nuclei on a square of side 2.8 bohr, each with an H 2.0 bohr
              further out on the diagonal; N = 200, 200,000 points, centre sets
              (heavy, H), 14 occupied.

Grids: Treutler-type radial map r = (xi/ln 2)(1+x)^0.6 ln(2/(1-x)) on
Gauss-Chebyshev (second kind) nodes, angular product of Gauss-Legendre nodes
in cos(theta) and uniform phi, Becke fuzzy-cell partition with three smoothing
iterations.  No radial node sits on a nucleus.  Orbitals are random U(-1,1)
combinations of the basis (numpy default_rng(seed)), Loewdin-orthonormalised in
the grid metric Phi^T W Phi.  Jastrow coefficients are U(-0.1, 0.1) from the same
generator.  Everything here is input generation; no part of the xTC method is
computed in this module.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
import math

import numpy as np

# Jastrow term set (m, n, o): c * (a1^m a2^n + a1^n a2^m) * b^o with m <= n <= 2,
# 1 <= o <= 2, m + n + o <= 4 -- nine terms per centre set.
CANONICAL_TERMS = np.array(
    [(0, 0, 1), (0, 1, 1), (0, 2, 1), (1, 1, 1), (1, 2, 1),
     (0, 0, 2), (0, 1, 2), (0, 2, 2), (1, 1, 2)], dtype=np.int32)

CONFIG_NAMES = ("h2", "water", "n2", "large")


@dataclass
class Problem:
    """One xTC build input.  Shapes: grid (n_grid, 3), weights (n_grid,),
    phi (n_grid, n_orb), gamma (n_orb, n_orb), nuc_xyz (n_nuc, 3),
    nuc_set (n_nuc,), terms (n_terms, 3), coef (n_sets, n_terms)."""
    name: str
    nuc_xyz: np.ndarray
    nuc_set: np.ndarray
    terms: np.ndarray
    coef: np.ndarray
    grid: np.ndarray
    weights: np.ndarray
    phi: np.ndarray
    gamma: np.ndarray
    n_occ: int
    seed: int
    # the basis (atom index, shell kind, exponent) and the orbital coefficients on the raw
    # Cartesian Gaussians: phi = basis_values(grid, nuc_xyz, shells) @ orb_coef up to rounding
    shells: list | None = None
    orb_coef: np.ndarray | None = None

    @property
    def n_grid(self) -> int:
        return self.grid.shape[0]

    @property
    def n_orb(self) -> int:
        return self.phi.shape[1]

    @property
    def n_sets(self) -> int:
        return self.coef.shape[0]

    @property
    def n_pair(self) -> int:
        return self.n_orb * (self.n_orb + 1) // 2


# ----------------------------------------------------------------------------- grid

def _radial(n: int, xi: float = 1.0):
    k = np.arange(1, n + 1)
    t = k * math.pi / (n + 1)
    x = np.cos(t)
    wx = math.pi / (n + 1) * np.sin(t) ** 2 / np.sqrt(1.0 - x * x)
    a = 0.6
    c = xi / math.log(2.0)
    r = c * (1.0 + x) ** a * np.log(2.0 / (1.0 - x))
    dr = c * (a * (1.0 + x) ** (a - 1.0) * np.log(2.0 / (1.0 - x)) + (1.0 + x) ** a / (1.0 - x))
    return r, wx * dr * r * r


def _angular(n_theta: int, n_phi: int):
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    ph = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    st = np.sqrt(1.0 - ct * ct)
    xyz = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                    np.outer(ct, np.ones_like(ph))], axis=-1).reshape(-1, 3)
    w = np.outer(wt, np.full(n_phi, 2.0 * math.pi / n_phi)).reshape(-1)
    return xyz, w


def _becke(points: np.ndarray, centres: np.ndarray, owner: int) -> np.ndarray:
    n_at = centres.shape[0]
    if n_at == 1:
        return np.ones(points.shape[0])
    d = np.linalg.norm(points[:, None, :] - centres[None, :, :], axis=-1)
    cell = np.ones((points.shape[0], n_at))
    for a in range(n_at):
        for b in range(n_at):
            if a == b:
                continue
            mu = (d[:, a] - d[:, b]) / np.linalg.norm(centres[a] - centres[b])
            f = mu
            for _ in range(3):
                f = 1.5 * f - 0.5 * f ** 3
            cell[:, a] *= 0.5 * (1.0 - f)
    return cell[:, owner] / cell.sum(axis=1)


def make_grid(centres: np.ndarray, spec):
    """spec: per atom (n_rad, n_theta, n_phi)."""
    pts, wts = [], []
    for a, (nr, nt, nph) in enumerate(spec):
        r, wr = _radial(nr)
        ang, wa = _angular(nt, nph)
        p = (r[:, None, None] * ang[None, :, :]).reshape(-1, 3) + centres[a]
        w = (wr[:, None] * wa[None, :]).reshape(-1)
        w = w * _becke(p, centres, a)
        pts.append(p)
        wts.append(w)
    return np.concatenate(pts), np.concatenate(wts)


# ----------------------------------------------------------------------------- basis

_HEAVY = {"s": [5.0, 1.5, 15.0, 0.5, 50.0, 0.18, 170.0, 0.07, 600.0, 2000.0, 0.03, 6000.0],
          "p": [1.2, 0.4, 4.0, 0.15, 13.0, 40.0, 0.06],
          "d": [0.8, 2.5, 0.3, 8.0]}
_HYDRO = {"s": [1.0, 0.3, 3.5, 0.1, 12.0, 40.0, 0.04, 130.0],
          "p": [0.8, 0.25, 2.5, 0.09],
          "d": [1.0, 0.35]}
_PATTERN = ["s", "p", "s", "d", "s", "p", "s", "p", "d", "s", "s", "p", "d", "s", "p", "s", "d", "s"]
_NCART = {"s": 1, "p": 3, "d": 6}
_CART = {"s": [(0, 0, 0)], "p": [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
         "d": [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]}


def _choose_shells(kinds, n_func):
    """Round-robin over atoms, each taking its next shell of a fixed pattern while
    it fits, then s functions with further exponents until exactly n_func."""
    shells = []
    ptr = [0] * len(kinds)
    used = [{"s": 0, "p": 0, "d": 0} for _ in kinds]
    total = 0
    progress = True
    while total < n_func and progress:
        progress = False
        for a, kind in enumerate(kinds):
            table = _HEAVY if kind == "X" else _HYDRO
            while ptr[a] < len(_PATTERN):
                L = _PATTERN[ptr[a]]
                ptr[a] += 1
                if used[a][L] < len(table[L]) and total + _NCART[L] <= n_func:
                    shells.append((a, L, table[L][used[a][L]]))
                    used[a][L] += 1
                    total += _NCART[L]
                    progress = True
                    break
            if total >= n_func:
                break
    extra = 0
    while total < n_func:
        a = extra % len(kinds)
        shells.append((a, "s", 0.02 * (2.7 ** (extra // len(kinds)))))
        extra += 1
        total += 1
    return shells


def basis_values(points, centres, shells):
    cols = []
    for a, L, alpha in shells:
        d = points - centres[a]
        r2 = np.einsum("ij,ij->i", d, d)
        g = np.exp(-alpha * r2)
        for (i, j, k) in _CART[L]:
            cols.append(d[:, 0] ** i * d[:, 1] ** j * d[:, 2] ** k * g)
    return np.stack(cols, axis=1)


def basis_gradients(points, centres, shells):
    """d/dr of every Cartesian Gaussian of basis_values: shape (n_points, n_functions, 3)."""
    cols = []
    for a, L, alpha in shells:
        d = points - centres[a]
        r2 = np.einsum("ij,ij->i", d, d)
        g = np.exp(-alpha * r2)
        for ijk in _CART[L]:
            mono = [d[:, x] ** ijk[x] for x in range(3)]
            grad = []
            for x in range(3):
                k = ijk[x]
                # d/dx (x^k e^{-alpha r^2}) = (k x^(k-1) - 2 alpha x^(k+1)) e^{-alpha r^2}
                dk = (k * d[:, x] ** (k - 1) if k > 0 else 0.0) - 2.0 * alpha * d[:, x] ** (k + 1)
                others = [mono[y] for y in range(3) if y != x]
                grad.append(dk * others[0] * others[1] * g)
            cols.append(np.stack(grad, axis=1))
    return np.stack(cols, axis=1)


def orthonormal_orbitals(chi, weights, n_orb, rng):
    """Returns (phi, C) with phi = chi @ C up to rounding."""
    norms = np.sqrt(np.einsum("gm,g,gm->m", chi, weights, chi))
    chi = chi / norms
    c = rng.uniform(-1.0, 1.0, size=(chi.shape[1], n_orb))
    phi = chi @ c
    C = c / norms[:, None]
    for _ in range(3):  # repeated symmetric orthonormalisation (converges to Loewdin)
        s = phi.T @ (weights[:, None] * phi)
        ev, U = np.linalg.eigh(s)
        T = U @ np.diag(ev ** -0.5) @ U.T
        phi = phi @ T
        C = C @ T
    return phi, C


def orbital_gradients(p: Problem) -> np.ndarray:
    """Analytic gradients of the orbitals at the grid points, shape (n_grid, n_orb, 3), C-contiguous:
    the inputs of the two-body integrals K (nabla phi on the grid)."""
    if p.shells is None or p.orb_coef is None:
        raise ValueError("problem carries no basis description")
    dchi = basis_gradients(p.grid, p.nuc_xyz, p.shells)
    return np.ascontiguousarray(np.einsum("gmx,mo->gox", dchi, p.orb_coef))


# ----------------------------------------------------------------------------- configs

def _closed_shell_gamma(n_orb, n_occ):
    g = np.zeros((n_orb, n_orb))
    g[np.arange(n_occ), np.arange(n_occ)] = 1.0
    return g


def _build(name, centres, kinds, grid_spec, n_orb, n_occ, nuc_set, n_sets, seed,
           shells=None, terms=CANONICAL_TERMS):
    rng = np.random.default_rng(seed)
    centres = np.asarray(centres, dtype=np.float64)
    grid, w = make_grid(centres, grid_spec)
    if shells is None:
        shells = _choose_shells(kinds, n_orb)
    chi = basis_values(grid, centres, shells)
    phi, C = orthonormal_orbitals(chi, w, n_orb, rng)
    coef = rng.uniform(-0.1, 0.1, size=(n_sets, terms.shape[0]))
    return Problem(name=name, nuc_xyz=centres, nuc_set=np.asarray(nuc_set, dtype=np.int32),
                   terms=np.ascontiguousarray(terms, dtype=np.int32), coef=coef,
                   grid=np.ascontiguousarray(grid), weights=np.ascontiguousarray(w),
                   phi=np.ascontiguousarray(phi), gamma=_closed_shell_gamma(n_orb, n_occ),
                   n_occ=n_occ, seed=seed, shells=list(shells), orb_coef=C)


def make_config(name: str) -> Problem:
    """The four measured workloads (see module docstring)."""
    if name == "h2":
        c = [[0, 0, -0.7], [0, 0, 0.7]]
        sh = []
        for a in range(2):
            sh += [(a, "s", e) for e in (13.0, 1.96, 0.44, 0.12, 0.03)] + [(a, "p", 0.73)]
        return _build("h2", c, "HH", [(20, 5, 10)] * 2, 10, 1, [0, 0], 1, 0, shells=sh)
    if name == "water":
        c = [[0, 0, 0], [0, 1.43, 1.11], [0, -1.43, 1.11]]
        return _build("water", c, "XHH", [(50, 20, 20), (40, 10, 25), (40, 10, 25)],
                      58, 5, [0, 1, 2], 3, 2)
    if name == "n2":
        c = [[0, 0, -1.035], [0, 0, 1.035]]
        return _build("n2", c, "XX", [(100, 20, 25)] * 2, 120, 7, [0, 1], 2, 3)
    if name == "large":
        h = 1.4
        heavy = [[h, h, 0], [-h, h, 0], [-h, -h, 0], [h, -h, 0]]
        hyd = [[x + 2.0 * np.sign(x) / math.sqrt(2), y + 2.0 * np.sign(y) / math.sqrt(2), 0]
               for x, y, _ in heavy]
        spec = [(100, 10, 25)] * 4 + [(50, 20, 25)] * 4
        return _build("large", heavy + hyd, "XXXXHHHH", spec, 200, 14,
                      [0, 0, 0, 0, 1, 1, 1, 1], 2, 5)
    raise ValueError(f"unknown config {name!r}")


def make_batched(n_inst: int = 32, seed: int = 4, scale: float = 1.0, n_orb_range=(20, 90)) -> list:
    """Instances of uneven size for the batched build: N uniform in [20, 90] (``n_orb_range``),
    grid uniform in [10k, 60k] points (times ``scale``; smaller ranges serve quick tests), 1-4
    nuclei uniformly in a ball of radius
    3 bohr (the first heavy, the rest H), one Jastrow centre set per nucleus, n_occ = max(1, N/10).
    Sizes and positions come from default_rng(seed); instance k draws its orbitals and Jastrow
    coefficients from default_rng(1000 + k)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        n_orb = int(rng.integers(n_orb_range[0], n_orb_range[1] + 1))
        n_grid = int(rng.integers(10000, 60001) * scale)
        n_nuc = int(rng.integers(1, 5))
        centres = []
        while len(centres) < n_nuc:
            p = rng.uniform(-3.0, 3.0, size=3)
            if np.linalg.norm(p) <= 3.0 and all(np.linalg.norm(p - q) > 1.0 for q in centres):
                centres.append(p)
        kinds = "X" + "H" * (n_nuc - 1)
        per_atom = max(n_grid // n_nuc, 200)
        n_theta, n_phi = 10, 20
        spec = [(max(per_atom // (n_theta * n_phi), 2), n_theta, n_phi)] * n_nuc
        out.append(_build(f"batched{k}", centres, kinds, spec, n_orb, max(1, n_orb // 10),
                          list(range(n_nuc)), n_nuc, 1000 + k))
    return out


def make_small(n_orb: int = 4, n_rad: int = 6, n_theta: int = 3, n_phi: int = 4,
               n_atoms: int = 2, seed: int = 7, n_occ: int = 1, separate_sets: bool = True,
               terms=CANONICAL_TERMS) -> Problem:
    """A small molecule for tests: n_atoms nuclei on a bent chain, heavy first."""
    base = [[0.0, 0.0, -0.7], [0.0, 0.0, 0.7], [0.0, 1.3, 1.2], [1.1, -0.9, 0.4]]
    centres = base[:n_atoms]
    kinds = "X" + "H" * (n_atoms - 1)
    n_sets = n_atoms if separate_sets else 1
    nuc_set = list(range(n_atoms)) if separate_sets else [0] * n_atoms
    return _build(f"small{n_orb}", centres, kinds, [(n_rad, n_theta, n_phi)] * n_atoms,
                  n_orb, n_occ, nuc_set, n_sets, seed, terms=np.asarray(terms, dtype=np.int32))


def random_density(n_orb: int, seed: int, rank: int | None = None) -> np.ndarray:
    """A random symmetric density with eigenvalues in [0, 1] and a random
    (non-diagonal) eigenbasis; rank = number of non-zero occupations."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n_orb, n_orb)))
    occ = rng.uniform(0.05, 1.0, size=n_orb)
    if rank is not None:
        occ[rank:] = 0.0
    g = (q * occ) @ q.T
    return 0.5 * (g + g.T)


def permute_grid(p: Problem, perm: np.ndarray) -> Problem:
    """The same problem with its grid points reordered."""
    return replace(p, grid=np.ascontiguousarray(p.grid[perm]),
                   weights=np.ascontiguousarray(p.weights[perm]),
                   phi=np.ascontiguousarray(p.phi[perm]))
