"""GPU parity of the frozen-core folding (xTC-FC, xtc_frozen_core_fold) against the CPU oracle
(oracle/frozen_core.py, pinned to Fock-space matrix elements), through the C ABI.

The fold itself runs in FP64 on identical inputs, so it must agree with the oracle to rounding
(1e-13 relative).  End to end (GPU build, then GPU fold, against oracle build and oracle fold) the
build's tolerances hold: 1e-8 Eh for FP64, 1e-6 Eh for the mixed precisions."""
import numpy as np
import pytest

import synth
from oracle import direct, frozen_core

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp16x2": 1e-6}


def ctx_for(p, prec, **kw):
    from paper_2304_07006_gb300 import Context
    c = Context(prec, **kw)
    if p is not None:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    return c


def _pair_symmetric(n, seed):
    """Random integrals with only the pair symmetry U(pq|rs) = U(rs|pq) (non-hermitian, like a
    caller's V - K) and a non-symmetric one-body matrix."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n,) * 4)
    return 0.5 * (a + a.transpose(2, 3, 0, 1)), rng.standard_normal((n, n))


@pytest.fixture(scope="module")
def small():
    p = synth.make_small(n_orb=7, n_rad=8, n_theta=4, n_phi=5, n_atoms=2, seed=5)   # 320 points
    g = synth.random_density(7, 61)
    return p, g, direct.build(p, g)


@pytest.mark.parametrize("core", [[0], [1, 4], [0, 2, 3, 6], []])
def test_fold_of_oracle_integrals_matches_oracle(small, core):
    _, _, ref = small
    with ctx_for(None, "fp64") as c:
        out = c.frozen_core_fold(ref["dU"], ref["dh"], core, want_dU=True)
    h_fc, e_core, act = frozen_core.fold(ref["dU"], ref["dh"], core)
    s = np.abs(ref["dU"]).max()
    assert np.abs(out["dh_fc"] - h_fc).max() < 1e-13 * s
    assert abs(out["e_core"][0] - e_core) < 1e-13 * s
    assert np.array_equal(out["dU_act"], ref["dU"][np.ix_(act, act, act, act)])


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_build_then_fold_matches_oracle(small, prec):
    p, g, ref = small
    core = [0, 3]
    with ctx_for(p, prec) as c:
        b = c.build(p.grid, p.weights, p.phi, g)
        out = c.frozen_core_fold(b["dU"], b["dh"], core, want_dU=True)
    h_fc, e_core, act = frozen_core.fold(ref["dU"], ref["dh"], core)
    assert np.abs(out["dh_fc"] - h_fc).max() < TOL[prec]
    assert abs(out["e_core"][0] - e_core) < TOL[prec]
    assert np.abs(out["dU_act"] - ref["dU"][np.ix_(act, act, act, act)]).max() < TOL[prec]


def test_freezing_occupied_orbitals_negates_delta_h():
    """Core = the occupied orbitals of a projector density: dh_fc = -Delta h, e_core = 0."""
    p = synth.make_small(n_orb=6, n_rad=8, n_theta=4, n_phi=5, n_atoms=2, seed=9)
    g = np.diag([1.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    with ctx_for(p, "fp64") as c:
        b = c.build(p.grid, p.weights, p.phi, g)
        out = c.frozen_core_fold(b["dU"], b["dh"], [0, 1])
    s = np.abs(b["dh"]).max()
    assert np.abs(out["dh_fc"] + b["dh"][2:, 2:]).max() < 1e-12 * s
    assert abs(out["e_core"][0]) < 1e-12 * s


def test_device_buffers_all_core_and_bad_indices():
    torch = pytest.importorskip("torch")
    from paper_2304_07006_gb300 import XtcError
    n = 9
    U, h = _pair_symmetric(n, 3)
    core = [8, 1, 5]
    with ctx_for(None, "fp64") as c:
        dU, dh = torch.tensor(U, device="cuda"), torch.tensor(h, device="cuda")
        dh_fc = torch.empty((6, 6), dtype=torch.float64, device="cuda")
        dU_act = torch.empty((6,) * 4, dtype=torch.float64, device="cuda")
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        c.frozen_core_fold(dU, dh, core, dh_fc=dh_fc, dU_act=dU_act, e_core=e)
        h_fc, e_core, act = frozen_core.fold(U, h, core)
        assert np.abs(dh_fc.cpu().numpy() - h_fc).max() < 1e-13 * np.abs(U).max()
        assert abs(e.item() - e_core) < 1e-13 * np.abs(U).max()
        assert np.array_equal(dU_act.cpu().numpy(), U[np.ix_(act, act, act, act)])
        # every orbital frozen: only the core energy
        out = c.frozen_core_fold(U, h, list(range(n)))
        assert abs(out["e_core"][0] - frozen_core.fold(U, h, list(range(n)))[1]) < 1e-12 * np.abs(U).max()
        for bad in ([1, 1], [n], [-1]):
            with pytest.raises(XtcError):
                c.frozen_core_fold(U, h, bad)


def test_full_size_fold():
    """120 orbitals (the headline orbital count), two core orbitals, non-hermitian integrals
    made on the device: the fold against the oracle on the same values."""
    torch = pytest.importorskip("torch")
    n, core = 120, [0, 61]
    gen = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randn((n,) * 4, dtype=torch.float64, device="cuda", generator=gen)
    dU = (a + a.permute(2, 3, 0, 1)) * 0.5
    del a
    dh = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=gen)
    with ctx_for(None, "fp64") as c:
        dU_act = torch.empty((n - 2,) * 4, dtype=torch.float64, device="cuda")
        out = c.frozen_core_fold(dU, dh, core, dU_act=dU_act)
    U, h = dU.cpu().numpy(), dh.cpu().numpy()
    h_fc, e_core, act = frozen_core.fold(U, h, core)
    assert np.abs(out["dh_fc"] - h_fc).max() < 1e-12
    assert abs(out["e_core"][0] - e_core) < 1e-12
    got = dU_act.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n - 2, size=(4096, 4))
    want = U[act[idx[:, 0]], act[idx[:, 1]], act[idx[:, 2]], act[idx[:, 3]]]
    assert np.array_equal(got[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]], want)
    assert np.array_equal(got[:, 5, 60, :], U[np.ix_(act, [act[5]], [act[60]], act)][:, 0, 0, :])
