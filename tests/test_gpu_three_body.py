"""GPU parity of the explicit three-body tensor of eq. Ldecomp (xtc_three_body_L) against the
CPU oracle's Route 1 tensor (bruteforce.L_ldecomp, itself pinned to the literal triple quadrature
of the L definition), through the C ABI.  The products and sums of L are FP64 on both sides; V
comes from steps (a)+(b) in the context's precision, so the mixed paths carry V's split error
(tolerance 1e-5 of max |L|)."""
import numpy as np
import pytest

import synth
from oracle import bruteforce

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-12, "fp16x2": 1e-5, "bf16x3": 1e-5}


def ctx_for(p, prec, **kw):
    from paper_2304_07006_gb300 import Context
    c = Context(prec, **kw)
    c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    return c


@pytest.fixture(scope="module")
def tiny():
    p = synth.make_small(n_orb=4, n_rad=5, n_theta=3, n_phi=4, n_atoms=2, seed=7)   # 120 points
    return p, bruteforce.L_ldecomp(p)


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_three_body_L_matches_oracle(tiny, prec):
    p, ref = tiny
    with ctx_for(p, prec) as c:
        L = c.three_body_L(p.grid, p.weights, p.phi)
    err = np.abs(L - ref).max() / np.abs(ref).max()
    assert err < REL[prec], err


def test_three_body_L_symmetries_and_outer_ranges(tiny):
    """Permuting the electrons (pairs moving together) leaves L unchanged; disjoint outer ranges
    add up to the whole grid; an empty range gives zeros; device output equals host output."""
    import torch
    p, _ = tiny
    with ctx_for(p, "fp64") as c:
        full = c.three_body_L(p.grid, p.weights, p.phi)
        c.set_outer_range(0, 50)
        a = c.three_body_L(p.grid, p.weights, p.phi)
        c.set_outer_range(50, -1)
        b = c.three_body_L(p.grid, p.weights, p.phi)
        c.set_outer_range(7, 7)
        z = c.three_body_L(p.grid, p.weights, p.phi)
        c.set_outer_range(0, -1)
        dev = torch.empty(full.shape, dtype=torch.float64, device="cuda:0")
        c.three_body_L(p.grid, p.weights, p.phi, out=dev)
        torch.cuda.synchronize()
    scale = np.abs(full).max()
    assert np.abs(full - np.einsum("prtqsu->rptsqu", full)).max() < 1e-13 * scale
    assert np.abs(full - np.einsum("prtqsu->tpruqs", full)).max() < 1e-13 * scale
    assert np.abs(a + b - full).max() < 1e-13 * scale
    assert np.all(z == 0.0)
    assert np.array_equal(dev.cpu().numpy(), full)


def test_three_body_L_h2_workload():
    """The H2-like workload (N=10, 2,000 points, the paper-sized minimal case) in FP64."""
    p = synth.make_config("h2")
    ref = bruteforce.L_ldecomp(p)
    with ctx_for(p, "fp64") as c:
        L = c.three_body_L(p.grid, p.weights, p.phi)
    assert np.abs(L - ref).max() < 1e-12 * np.abs(ref).max()


def test_three_body_L_rejects_large_orbital_sets(tiny):
    from paper_2304_07006_gb300 import XtcError
    p, _ = tiny
    phi = np.zeros((p.n_grid, 25))
    with ctx_for(p, "fp64") as c:
        with pytest.raises(XtcError) as e:
            c.three_body_L(p.grid, p.weights, phi)
        assert e.value.code == -1
