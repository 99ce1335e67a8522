"""GPU parity of the spin-resolved build (Appendix A, xtc_build_1b2b_rohf) against the CPU
oracle's restricted open-shell equations (oracle/spin.py, itself pinned to the spin-orbital
definition), through the C ABI.  Tolerances as in test_gpu_parity, absolute in Hartree on every
entry of every output: FP64 1e-8 Eh, mixed 1e-6 Eh."""
import numpy as np
import pytest

import synth
from oracle import spin

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp16x2": 1e-6, "bf16x3": 1e-6}
KEYS = ("dU_aa", "dU_ab", "dU_bb", "dh_a", "dh_b", "e0")


def ctx_for(p, prec, **kw):
    from paper_2304_07006_gb300 import Context
    c = Context(prec, **kw)
    c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    return c


def max_err(out, ref, keys=KEYS):
    errs = []
    for k in keys:
        a = np.asarray(out[k], dtype=np.float64).reshape(-1)
        b = np.asarray(ref[k], dtype=np.float64).reshape(-1)
        errs.append(np.abs(a - b).max())
    return max(errs)


@pytest.fixture(scope="module")
def small():
    p = synth.make_small(n_orb=6, n_rad=8, n_theta=4, n_phi=5, n_atoms=2, seed=5)   # 320 points
    ga, gb = synth.random_density(6, 51), synth.random_density(6, 52, rank=3)
    return p, ga, gb, spin.build(p, ga, gb)


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_rohf_build_small_random_densities(small, prec):
    p, ga, gb, ref = small
    with ctx_for(p, prec) as c:
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
    err = max_err(out, ref)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_rohf_chunks_and_ragged_tail(small, prec):
    """Several outer chunks (128 points each, the last one partial) and a rank-1 beta density."""
    p, ga, _, _ = small
    gb = synth.random_density(6, 53, rank=1)
    ref = spin.build(p, ga, gb)
    with ctx_for(p, prec, grid_chunk=128) as c:
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
    assert max_err(out, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_rohf_equal_densities_match_closed_shell_build(small, prec):
    """gamma^a = gamma^b: every block is the closed-shell build's Delta U (Appendix B)."""
    p, ga, _, _ = small
    with ctx_for(p, prec) as c:
        closed = c.build(p.grid, p.weights, p.phi, ga)
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, ga)
    ref = {"dU_aa": closed["dU"], "dU_ab": closed["dU"], "dU_bb": closed["dU"], "dh_a": closed["dh"],
           "dh_b": closed["dh"], "e0": closed["e0"]}
    assert max_err(out, ref) < TOL[prec]


def test_rohf_beta_density_zero_and_empty_outer_range(small):
    """A fully polarised density (gamma^b = 0) against the oracle, then an empty outer range."""
    p, ga, _, _ = small
    gb = np.zeros_like(ga)
    ref = spin.build(p, ga, gb)
    with ctx_for(p, "fp16x2") as c:
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
        assert max_err(out, ref) < TOL["fp16x2"]
        c.set_outer_range(5, 5)
        empty = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
    for k in KEYS:
        assert np.all(np.asarray(empty[k]) == 0.0), k


def test_rohf_device_outputs_match_host_outputs_bitwise(small):
    import torch
    p, ga, gb, _ = small
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n = p.n_orb
    outs = {k: torch.empty((n,) * 4, dtype=torch.float64, device=dev) for k in ("dU_aa", "dU_ab", "dU_bb")}
    outs.update({k: torch.empty((n, n), dtype=torch.float64, device=dev) for k in ("dh_a", "dh_b")})
    outs["e0"] = torch.empty(1, dtype=torch.float64, device=dev)
    with ctx_for(p, "fp16x2") as c:
        host = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
        c.build_rohf(t(p.grid), t(p.weights), t(p.phi), t(ga), t(gb), **outs)
        torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(outs[k].cpu().numpy().reshape(-1), np.asarray(host[k]).reshape(-1)), k


def test_rohf_error_statuses(small):
    from paper_2304_07006_gb300 import XtcError
    p, ga, gb, _ = small
    with ctx_for(p, "fp16x2") as c:
        bad = gb.copy()
        bad[0, 1] += 1e-3
        with pytest.raises(XtcError) as e:
            c.build_rohf(p.grid, p.weights, p.phi, ga, bad)
        assert e.value.code == -2                              # gamma_b not symmetric
        bad = ga.copy()
        bad[2, 2] = np.inf
        with pytest.raises(XtcError) as e:
            c.build_rohf(p.grid, p.weights, p.phi, bad, gb)
        assert e.value.code == -3                              # non-finite gamma_a
        c.build_rohf(p.grid, p.weights, p.phi, ga, gb)         # still usable


@pytest.mark.parametrize("prec", ["fp64", "fp16x2", "bf16x3"])
def test_rohf_water_workload_sampled_outer_points(prec):
    """The water workload with an open-shell density (5 alpha, 4 beta occupied orbitals), on 48
    sampled outer points (full inner sums)."""
    p = synth.make_config("water")
    perm = np.random.default_rng(11).permutation(p.n_grid)
    p = synth.permute_grid(p, perm)
    n = p.n_orb
    ga = np.diag([1.0] * 5 + [0.0] * (n - 5))
    gb = np.diag([1.0] * 4 + [0.0] * (n - 4))
    ref = spin.build(p, ga, gb, outer=np.arange(48))
    with ctx_for(p, prec) as c:
        c.set_outer_range(0, 48)
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
    assert max_err(out, ref) < TOL[prec]


@pytest.fixture(scope="module")
def n2_open_shell():
    """The N=120 workload with 8 alpha and 7 beta occupied orbitals."""
    p = synth.make_config("n2")
    n = p.n_orb
    return p, np.diag([1.0] * 8 + [0.0] * (n - 8)), np.diag([1.0] * 7 + [0.0] * (n - 7))


def test_rohf_n2_workload_sampled_outer_points(n2_open_shell):
    """16 sampled outer points of the N=120 workload (full inner sums), fp16x2, against the oracle."""
    p, ga, gb = n2_open_shell
    perm = np.random.default_rng(12).permutation(p.n_grid)
    q = synth.permute_grid(p, perm)
    ref = spin.build(q, ga, gb, outer=np.arange(16))
    with ctx_for(q, "fp16x2") as c:
        c.set_outer_range(0, 16)
        out = c.build_rohf(q.grid, q.weights, q.phi, ga, gb)
    err = max_err(out, ref)
    assert err < TOL["fp16x2"], err


def test_rohf_n2_workload_whole_grid_blocks_average_to_closed_shell(n2_open_shell):
    """Every outer point of the N=120 workload, fp16x2.  Delta U is linear in the two densities,
    so (aa + bb) / 2 and the pair-symmetrised ab block equal the closed-shell build's Delta U for
    the spin-averaged density (checked on the oracle in the CPU pins); this exercises the spin
    passes, the ab cross block and the unpacking at full size."""
    p, ga, gb = n2_open_shell
    with ctx_for(p, "fp16x2") as c:
        out = c.build_rohf(p.grid, p.weights, p.phi, ga, gb)
        closed = c.build(p.grid, p.weights, p.phi, 0.5 * (ga + gb))
    ref = np.asarray(closed["dU"])
    tol = TOL["fp16x2"] * max(1.0, np.abs(ref).max())
    assert np.abs(0.5 * (out["dU_aa"] + out["dU_bb"]) - ref).max() < tol
    assert np.abs(0.5 * (out["dU_ab"] + out["dU_ab"].transpose(2, 3, 0, 1)) - ref).max() < tol
    assert np.all(np.isfinite(out["dh_a"])) and np.all(np.isfinite(out["dh_b"])) and np.isfinite(out["e0"][0])
