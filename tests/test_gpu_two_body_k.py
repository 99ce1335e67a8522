"""GPU parity of the two-body integrals K (xtc_two_body_K) against the CPU oracle
(two_body_k.k_integrals, pinned to the similarity transformation by differences), through the C ABI.

The Laplacian table, its product with the pair densities and the contraction are FP64 on the GPU;
V comes from steps (a)+(b) in the context's precision, so the mixed paths carry V's split error
(measured 2.2e-7 for fp16x2 and 9.5e-8 for bf16x3 of max |K| on the 13-orbital case; the tests allow
2e-6, and 1e-11 in FP64).  The cases span several 64-wide tiles of every GEMM dimension with ragged
tails (N = 13: N^2 = 169 rows, 91 pairs; 210 and 600 grid points)."""
import numpy as np
import pytest

import synth
from oracle import two_body_k

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-11, "fp16x2": 2e-6, "bf16x3": 2e-6}


def ctx_for(p, prec, **kw):
    from paper_2304_07006_gb300 import Context
    c = Context(prec, **kw)
    c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    return c


def oracle_k(p, dphi):
    return two_body_k.k_integrals(p.grid, p.weights, p.phi, dphi, p.nuc_xyz, p.nuc_set, p.terms, p.coef)


@pytest.fixture(scope="module")
def small():
    p = synth.make_small(n_orb=13, n_rad=7, n_theta=3, n_phi=5, n_atoms=2, seed=5)   # 210 points
    d = synth.orbital_gradients(p)
    return p, d, oracle_k(p, d)


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_two_body_K_matches_oracle(small, prec):
    p, d, ref = small
    with ctx_for(p, prec) as c:
        K = c.two_body_K(p.grid, p.weights, p.phi, d)
    err = np.abs(K - ref).max() / np.abs(ref).max()
    assert err < REL[prec], err


def test_two_body_K_three_centres_more_orbitals():
    """Three nuclei with their own centre sets, N = 10, 600 points, electron-nucleus-only terms
    (o = 0) beside the canonical ones."""
    terms = np.concatenate([synth.CANONICAL_TERMS, np.array([(0, 2, 0), (1, 1, 0)], dtype=np.int32)])
    p = synth.make_small(n_orb=10, n_rad=5, n_theta=5, n_phi=8, n_atoms=3, seed=9, terms=terms)
    d = synth.orbital_gradients(p)
    ref = oracle_k(p, d)
    with ctx_for(p, "fp64") as c:
        K = c.two_body_K(p.grid, p.weights, p.phi, d)
    assert np.abs(K - ref).max() < REL["fp64"] * np.abs(ref).max()


def test_two_body_K_chunks_ranges_and_device_buffers(small):
    """Chunks of 128 outer points give the one-chunk result; disjoint outer ranges add up to the
    whole grid; an empty range gives zeros; device inputs and output give the host result; K has
    the pair-swap symmetry and is not hermitian."""
    import torch
    p, d, _ = small
    with ctx_for(p, "fp64") as c:
        full = c.two_body_K(p.grid, p.weights, p.phi, d)
        c.set_outer_range(0, 77)
        a = c.two_body_K(p.grid, p.weights, p.phi, d)
        c.set_outer_range(77, -1)
        b = c.two_body_K(p.grid, p.weights, p.phi, d)
        c.set_outer_range(5, 5)
        z = c.two_body_K(p.grid, p.weights, p.phi, d)
        c.set_outer_range(0, -1)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")
        dev = torch.empty(full.shape, dtype=torch.float64, device="cuda:0")
        c.two_body_K(t(p.grid), t(p.weights), t(p.phi), t(d), out=dev)
        torch.cuda.synchronize()
    with ctx_for(p, "fp64", grid_chunk=128) as c:
        chunked = c.two_body_K(p.grid, p.weights, p.phi, d)
    scale = np.abs(full).max()
    assert np.abs(chunked - full).max() < 1e-13 * scale
    assert np.abs(a + b - full).max() < 1e-13 * scale
    assert np.all(z == 0.0)
    assert np.array_equal(dev.cpu().numpy(), full)
    assert np.abs(full - full.transpose(2, 3, 0, 1)).max() < 1e-13 * scale
    assert np.abs(full - full.transpose(1, 0, 3, 2)).max() > 1e-3 * scale


def test_two_body_K_argument_errors(small):
    from paper_2304_07006_gb300 import Context, XtcError
    p, d, _ = small
    with ctx_for(p, "fp64") as c:
        bad = d.copy()
        bad[3, 2, 1] = np.nan
        with pytest.raises(XtcError) as e:
            c.two_body_K(p.grid, p.weights, p.phi, bad)
        assert e.value.code == -3
        with pytest.raises(XtcError) as e:
            c.two_body_K(p.grid, p.weights, np.zeros((p.n_grid, 201)), np.zeros((p.n_grid, 201, 3)))
        assert e.value.code == -1
        # the library still works after the refused calls
        K = c.two_body_K(p.grid, p.weights, p.phi, d)
        assert np.isfinite(K).all()
    with Context("fp64") as c:
        with pytest.raises(XtcError) as e:
            c.two_body_K(p.grid, p.weights, p.phi, d)
        assert e.value.code == -7
