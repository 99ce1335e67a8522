"""Failure handling on the GPU without faulting it: a bounded device wait that runs out reports
XTC_ERR_TIMEOUT and leaves the context usable; a caller allocator supplies and takes back the
whole device workspace, and one that refuses a request makes the build fail with XTC_ERR_OOM."""
import numpy as np
import pytest

import synth
from oracle import direct

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    p = synth.make_small(n_orb=5, n_rad=6, n_theta=3, n_phi=4, n_atoms=2, seed=4)
    return p, direct.build(p)


def _err(out, ref):
    return max(float(np.abs(np.asarray(out[k]) - np.asarray(ref[k])).max()) for k in ("dU", "dh", "e0"))


def test_bounded_wait_times_out_and_the_context_stays_usable(small):
    from paper_2304_07006_gb300 import Context
    p, ref = small
    with Context("fp16x2") as c:
        assert c.selftest_wait_timeout(50) == -6               # XTC_ERR_TIMEOUT
        assert c.selftest_wait_timeout(0) == -1                # limit out of range
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        assert _err(c.build(p.grid, p.weights, p.phi, p.gamma), ref) < 1e-6


def _torch_allocator(limit=None):
    import torch
    live, log = {}, []

    def alloc(n):
        if limit is not None and n > limit:
            return 0
        t = torch.empty(n, dtype=torch.uint8, device="cuda:0")
        live[t.data_ptr()] = t
        log.append(n)
        return t.data_ptr()

    def release(ptr):
        del live[ptr]

    return (alloc, release), live, log


def test_caller_allocator_supplies_and_takes_back_the_workspace(small):
    from paper_2304_07006_gb300 import Context
    p, ref = small
    with Context("fp16x2") as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        want = c.build(p.grid, p.weights, p.phi, p.gamma)
    allocator, live, log = _torch_allocator()
    with Context("fp16x2", allocator=allocator) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        got = c.build(p.grid, p.weights, p.phi, p.gamma)
        got2 = c.build(p.grid, p.weights, p.phi, p.gamma)      # reuses the workspace
        assert len(log) > 10 and live
    assert not live                                            # everything went back
    for k in ("dU", "dh", "e0"):
        assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), k
        assert np.array_equal(np.asarray(got2[k]), np.asarray(want[k])), k


def test_caller_allocator_refusal_is_reported_as_out_of_memory(small):
    from paper_2304_07006_gb300 import Context, XtcError
    p, _ = small
    allocator, live, _ = _torch_allocator(limit=1 << 16)     # refuses anything above 64 KiB
    with Context("fp16x2", allocator=allocator) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        with pytest.raises(XtcError) as e:
            c.build(p.grid, p.weights, p.phi, p.gamma)
        assert e.value.code == -4                              # XTC_ERR_OOM
    assert not live


def test_refined_reciprocals_are_within_one_ulp_and_unbiased():
    """Step (a) of the tensor-core precisions takes 1/sqrt(x) and 1/x as the hardware approximation
    plus one Newton-Raphson step.  Against correctly rounded FP32 values (from FP64): at most one
    ulp off, and the signed errors average out (a one-signed error would bias the gradient, and
    with it every output, by the same relative amount)."""
    from paper_2304_07006_gb300 import Context
    rng = np.random.default_rng(3)
    # squared distances and 1 + distances as the gradient meets them: 1e-20 .. 1e4 bohr^2, 1 .. 100
    x = np.concatenate([10.0 ** rng.uniform(-20, 4, 2_000_000), rng.uniform(1.0, 100.0, 2_000_000)]).astype(np.float32)
    with Context("fp16x2") as c:
        ys, yr = c.selftest_reciprocals(x)
    assert np.isfinite(ys).all() and np.isfinite(yr).all()        # packed and scalar forms agree
    xd = x.astype(np.float64)
    for got, exact in ((ys, 1.0 / np.sqrt(xd)), (yr, 1.0 / xd)):
        want = exact.astype(np.float32)                           # correctly rounded
        ulp = np.spacing(np.abs(want)).astype(np.float64)
        err = (got.astype(np.float64) - exact) / ulp
        assert (np.abs(got.astype(np.float64) - want.astype(np.float64)) <= ulp).all(), "more than one ulp"
        assert abs(err.mean()) < 0.01, err.mean()                 # no systematic part
