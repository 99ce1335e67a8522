"""The allocation-free entry point xtc_vfield_noalloc, for callers that may not allocate device
memory (code inside a framework that owns every allocation, or a loop that must not call
cudaMalloc).  Its output must match the oracle's vector pair fields (steps (a)+(b), eq. Ldecomp
intermediate) within the tolerance the step-(b) parity tests use, on two calls in a row (the
second call reuses the library's fixed scratch array left over from the first), and the call
must reject problems whose workspace does not fit that array.  This file is collected last on
purpose."""
import numpy as np
import pytest

import synth
from oracle import direct

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp16x2": 2e-6, "bf16x3": 2e-6}


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_noalloc_vfield_matches_oracle_twice(prec):
    torch = pytest.importorskip("torch")
    from paper_2304_07006_gb300 import Context
    p = synth.make_config("h2")
    jas = (p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    want = direct.vfield(p.grid, p.weights, p.phi, jas, np.arange(p.n_grid))   # [i][x][p][q]
    iu = np.triu_indices(p.n_orb)
    want = want[:, :, iu[0], iu[1]]                                              # packed pairs p <= q
    scale = np.abs(want).max()
    grid, w, phi = _dev(torch, p.grid), _dev(torch, p.weights), _dev(torch, p.phi)
    with Context(prec) as c:
        c.set_jastrow(*jas)
        for call in range(2):
            out = torch.full((p.n_grid, 3, p.n_pair), float("nan"), dtype=torch.float64, device="cuda")
            c.vfield_noalloc(grid, w, phi, 0, p.n_grid, out)
            got = out.cpu().numpy()
            assert np.isfinite(got).all(), call
            assert np.abs(got - want).max() < TOL[prec] * scale, (call, np.abs(got - want).max() / scale)
        # an outer sub-range lands at the start of the output
        out = torch.zeros((100, 3, p.n_pair), dtype=torch.float64, device="cuda")
        c.vfield_noalloc(grid, w, phi, 700, 800, out)
        assert np.abs(out.cpu().numpy() - want[700:800]).max() < TOL[prec] * scale


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x3"])
def test_noalloc_long_inner_sum_without_fp64_flush(prec):
    """20,000 inner points (N=10): past the 8,192-point interval at which xtc_vfield flushes its
    FP32 running sums to FP64, which the allocation-free call does not do.  Its error against the
    oracle stays within the step-(b) tolerance (measured: see the assertion message)."""
    torch = pytest.importorskip("torch")
    from paper_2304_07006_gb300 import Context
    p = synth.make_small(n_orb=10, n_rad=40, n_theta=10, n_phi=25, n_atoms=2, seed=21)  # 20,000 points
    jas = (p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    outer = np.arange(0, 256)
    iu = np.triu_indices(p.n_orb)
    want = direct.vfield(p.grid, p.weights, p.phi, jas, outer)[:, :, iu[0], iu[1]]
    scale = np.abs(want).max()
    with Context(prec) as c:
        c.set_jastrow(*jas)
        out = torch.full((len(outer), 3, p.n_pair), float("nan"), dtype=torch.float64, device="cuda")
        c.vfield_noalloc(_dev(torch, p.grid), _dev(torch, p.weights), _dev(torch, p.phi), 0, len(outer), out)
    rel = np.abs(out.cpu().numpy() - want).max() / scale
    assert rel < TOL[prec], rel


def test_noalloc_rejects_host_pointers_and_oversized_problems():
    torch = pytest.importorskip("torch")
    from paper_2304_07006_gb300 import Context, XtcError
    p = synth.make_config("h2")
    with Context("fp16x2") as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        out = np.zeros((p.n_grid, 3, 55))
        with pytest.raises(XtcError) as e:                 # host buffers would need staging memory
            c.vfield_noalloc(p.grid, p.weights, p.phi, 0, p.n_grid, out)
        assert e.value.code == -1
        big = synth.make_config("water")                  # pair tables of ~270 MiB do not fit 64 MiB
        c.set_jastrow(big.nuc_xyz, big.nuc_set, big.terms, big.coef)
        outb = torch.zeros((4, 3, big.n_pair), dtype=torch.float64, device="cuda")
        with pytest.raises(XtcError) as e:
            c.vfield_noalloc(_dev(torch, big.grid), _dev(torch, big.weights), _dev(torch, big.phi), 0, 4, outb)
        assert e.value.code == -1 and "MiB" in str(e.value)
