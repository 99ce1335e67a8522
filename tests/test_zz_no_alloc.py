"""The allocation-free entry point xtc_vfield_noalloc, for callers that may not allocate device
memory (code inside a framework that owns every allocation, or a loop that must not call
cudaMalloc).  It must reproduce xtc_vfield (the allocating entry point of the same steps) within
the tolerance the step-(b) parity tests use, on two calls in a row (the second call reuses the
library's fixed scratch array left over from the first), and reject problems whose workspace
does not fit that array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp16x2": 2e-6, "bf16x3": 2e-6}


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_noalloc_vfield_matches_allocating_entry_point_twice(prec):
    torch = pytest.importorskip("torch")
    from paper_2304_07006_gb300 import Context
    p = synth.make_config("h2")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    grid, w, phi = dev(p.grid), dev(p.weights), dev(p.phi)
    n_pair = p.n_orb * (p.n_orb + 1) // 2
    with Context(prec) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        want = c.vfield(p.grid, p.weights, p.phi, 0, p.n_grid)
        scale = np.abs(want).max()
        for call in range(2):
            out = torch.full((p.n_grid, 3, n_pair), float("nan"), dtype=torch.float64, device="cuda")
            c.vfield_noalloc(grid, w, phi, 0, p.n_grid, out)
            got = out.cpu().numpy()
            assert np.isfinite(got).all(), call
            assert np.abs(got - want).max() < TOL[prec] * scale, (call, np.abs(got - want).max() / scale)
        # an outer sub-range lands at the start of the output
        out = torch.zeros((100, 3, n_pair), dtype=torch.float64, device="cuda")
        c.vfield_noalloc(grid, w, phi, 700, 800, out)
        assert np.abs(out.cpu().numpy() - want[700:800]).max() < TOL[prec] * scale


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
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        outb = torch.zeros((4, 3, big.n_pair), dtype=torch.float64, device="cuda")
        with pytest.raises(XtcError) as e:
            c.vfield_noalloc(dev(big.grid), dev(big.weights), dev(big.phi), 0, 4, outb)
        assert e.value.code == -1 and "MiB" in str(e.value)
