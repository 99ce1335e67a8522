"""Benchmark of the xTC one-/two-body build (steps a-d) on one GB300.

One step = one complete xTC build of the N2/CO-like workload (N = 120 orbitals, 100,000
grid points, 7 doubly occupied orbitals, 2 Jastrow centre sets x 9 terms): Delta U, Delta h and
the constant, in the mixed-precision path.  The metric is algorithmic TFLOP/s of the build,

    F = F_b + F_c + F_d,  F_b = 2*3*N_g^2*N_pair,  F_c = 12*N_g*N^3,  F_d = 2*4*N_g*N_pair^2,

divided by the device time of one build (inputs resident in HBM).  The per-step working set
(pair-product tables of several GB) is far larger than L2, so no flush is needed between steps.

Also reported: the same metric end to end through the C ABI with host buffers (``e2e``), the
roofline of the dominant kernel (step b on the tensor cores), the FP64 GPU path timed on
sampled outer points (time is linear in the outer sum) with the mixed/FP64 speed ratio, the
mixed-vs-FP64 error in Hartree on those points, and the CPU oracle timed on a bounded sample.

``--impl reference`` times the CPU oracle (the plain FP64 numpy restatement of the paper) on
the same workload and metric instead.  With several GPUs (torchrun) every rank runs an
independent replica (the build does not shard in this version) and the value is the sum.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "n2"
METRIC = "xTC 2-body build TFLOP/s & seconds at N=120 (mixed vs FP64, same GB300) at stated Eh error"


def job_throughput(ms_local: float, steps: int, world: int, flops_per_step: float, dist=None, device=None):
    """Milliseconds per step of the slowest rank and the whole-job TFLOP/s.  Every rank runs the
    same build on its own GPU (replicas), so the job does world x the per-step work in the slowest
    rank's time.  dist: torch.distributed (initialised) or None for one process."""
    ms = float(ms_local)
    if dist is not None:
        import torch
        tt = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_step = ms / steps
    return ms_step, world * flops_per_step / (ms_step * 1e-3) / 1e12


def flops(n_orb: int, n_grid: int, n_outer: int | None = None) -> dict:
    n_outer = n_grid if n_outer is None else n_outer
    npair = n_orb * (n_orb + 1) // 2
    fb = 2.0 * 3 * n_outer * n_grid * npair
    fc = 12.0 * n_outer * n_orb ** 3
    fd = 2.0 * 4 * n_outer * npair * npair
    return {"b": fb, "c": fc, "d": fd, "total": fb + fc + fd}


def config_dict(p, prec):
    return {"workload": f"{WORKLOAD}: N2/CO-like diatomic at 2.07 bohr, N={p.n_orb} orbitals, "
                        f"{p.n_grid} grid points, {p.n_occ} doubly occupied, {p.n_sets} Jastrow centre sets x "
                        f"{p.terms.shape[0]} terms",
            "n_orb": p.n_orb, "n_grid": p.n_grid, "n_occ": p.n_occ, "precision": prec,
            "l2": "per-step working set (rho split tables, several GB) >> 129 MB L2; no flush needed"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.send_signal(signal.SIGTERM)
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# dram__bytes_read.sum + dram__bytes_write.sum of one step (b) GEMM launch (fp16x2) captured with
# ncu on the first VFIELD_CAPTURE_OUTER outer points of the workload (`--ncu-case`), for GEMM
# engine revision VFIELD_CAPTURE_REVISION; with another revision the traffic is reported as null
VFIELD_CAPTURE_REVISION = 5
VFIELD_DRAM_BYTES_CAPTURED = 21_219_623_424 + 2_889_048_320
VFIELD_CAPTURE_OUTER = 1184


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def oracle_sample(p, n_sample: int, seed: int = 0):
    """Times the CPU oracle on n_sample outer points (full inner sum)."""
    from oracle import direct
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(p.n_grid, size=n_sample, replace=False))
    t0 = time.perf_counter()
    direct.build(p, outer=idx, i_block=n_sample)
    dt = time.perf_counter() - t0
    f = flops(p.n_orb, p.n_grid, n_sample)["total"]
    return {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "seconds": dt,
            "sample": f"{n_sample} random outer grid points of the {WORKLOAD} workload with the full inner sum "
                      f"(the build is linear in the outer sum); numpy FP64, BLAS threads = all host cores"}


def run_reference(args):
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = synth.make_config(WORKLOAD)
    n_sample = 2
    for _ in range(args.warmup):
        oracle_sample(p, n_sample)
    times, vals = [], []
    for s in range(args.steps):
        r = oracle_sample(p, n_sample, seed=s + 1)
        times.append(r["seconds"])
        vals.append(r["value"])
    value = float(np.mean(vals))
    cpu = {"value": value, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": r["sample"].replace(f"{n_sample} random", f"{n_sample} random")}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(p, "fp64 (CPU oracle)"), "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_measure(args, torch, dev, local):
    """The batched workload (uneven instances: N in [20, 90], 10k-60k points, 1-4 nuclei): one
    xtc_build_1b2b_batched call against a loop of xtc_build_1b2b calls on one context, inputs
    resident on the device, after one warm-up of each.  Delta U is formed (it feeds Delta h and
    the constant) but not unpacked into dense N^4 outputs."""
    import synth
    from paper_2304_07006_gb300 import Context

    probs = synth.make_batched(args.batched)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    inst = [{"nuc_xyz": q.nuc_xyz, "nuc_set": q.nuc_set, "terms": q.terms, "coef": q.coef, "grid": t(q.grid),
             "weights": t(q.weights), "phi": t(q.phi), "gamma": t(q.gamma),
             "dh": torch.empty((q.n_orb, q.n_orb), dtype=torch.float64, device=dev),
             "e0": torch.empty(1, dtype=torch.float64, device=dev)} for q in probs]
    total = sum(flops(q.n_orb, q.n_grid)["total"] for q in probs)

    def loop(c):
        for d in inst:
            c.set_jastrow(d["nuc_xyz"], d["nuc_set"], d["terms"], d["coef"])
            c.build(d["grid"], d["weights"], d["phi"], d["gamma"], dh=d["dh"], e0=d["e0"], want_dU=False)

    res = {}
    with Context(args.precision, device=local) as c:
        loop(c)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        loop(c)
        torch.cuda.synchronize(dev)
        res["loop_s"] = time.perf_counter() - t0
    with Context(args.precision, device=local) as c:
        c.build_batched(inst, want_dU=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c.build_batched(inst, want_dU=False)
        torch.cuda.synchronize(dev)
        res["batched_s"] = time.perf_counter() - t0
    return {"instances": len(probs), "n_orb_range": [min(q.n_orb for q in probs), max(q.n_orb for q in probs)],
            "n_grid_range": [min(q.n_grid for q in probs), max(q.n_grid for q in probs)],
            "algorithmic_flops": total, "loop_s": res["loop_s"], "batched_s": res["batched_s"],
            "tflops_batched": total / res["batched_s"] / 1e12, "tflops_loop": total / res["loop_s"] / 1e12,
            "speedup_vs_loop": res["loop_s"] / res["batched_s"], "lanes": 4,
            "note": "wall time of one call (host + device), inputs on the device, dU not unpacked"}


def rohf_measure(args, torch, dev, local, p, s_closed):
    """The spin-resolved build (Appendix A) on the same workload with 8 alpha and 7 beta occupied
    orbitals: inputs and outputs on the device, Delta U formed but not unpacked, one warm-up and
    two timed builds (CUDA events).  Algorithmic work: step (b) once, steps (c) and (d) once per
    spin of electron 2."""
    from paper_2304_07006_gb300 import Context
    from paper_2304_07006_gb300.xtc import KERNEL_NAMES

    N, NG = p.n_orb, p.n_grid
    F = flops(N, NG)
    total = F["b"] + 2 * F["c"] + 2 * F["d"]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ga = t(np.diag([1.0] * 8 + [0.0] * (N - 8)))
    gb = t(np.diag([1.0] * 7 + [0.0] * (N - 7)))
    grid, w, phi = t(p.grid), t(p.weights), t(p.phi)
    outs = {k: torch.empty((N, N), dtype=torch.float64, device=dev) for k in ("dh_a", "dh_b")}
    outs["e0"] = torch.empty(1, dtype=torch.float64, device=dev)
    steps = 2
    with Context(args.precision, device=local, timing=True) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.build_rohf(grid, w, phi, ga, gb, want_dU=False, **outs)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        per = {k: 0.0 for k in KERNEL_NAMES}
        for _ in range(steps):
            c.build_rohf(grid, w, phi, ga, gb, want_dU=False, **outs)
            for k, (ms, _) in c.timings().items():
                per[k] += ms / steps
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sec = e0.elapsed_time(e1) / 1e3 / steps
    return {"densities": "8 alpha, 7 beta occupied orbitals (diagonal)", "seconds_per_build": sec,
            "algorithmic_flops": total, "tflops": total / sec / 1e12, "time_vs_closed_shell_build": sec / s_closed,
            "per_kernel_ms": per, "note": "inputs and outputs on the device; Delta U not unpacked"}


def fullrank_measure(args, torch, dev, local, p, per_kernel_closed):
    """The N=120 workload with a random full-rank density (eigenvalues in [0.05, 1], a random
    eigenbasis: a correlated-density stand-in): one warm-up and one timed build, inputs and outputs
    on the device, Delta U formed but not unpacked; step (d) time against the rank-7 build's."""
    import synth
    from paper_2304_07006_gb300 import Context

    N = p.n_orb
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grid, w, phi = t(p.grid), t(p.weights), t(p.phi)
    gam = t(synth.random_density(N, 120))
    dh = torch.empty((N, N), dtype=torch.float64, device=dev)
    e0 = torch.empty(1, dtype=torch.float64, device=dev)
    with Context(args.precision, device=local, timing=True) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.build(grid, w, phi, gam, dh=dh, e0=e0, want_dU=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c.build(grid, w, phi, gam, dh=dh, e0=e0, want_dU=False)
        torch.cuda.synchronize(dev)
        sec = time.perf_counter() - t0
        tm = c.timings()
    # the step (d) GEMM alone: the row splits and adds into M are timed with step (b)'s V writes
    # under "aux", which the next chunk's step (a) on the second stream overlaps
    d_ms = tm["assemble"][0]
    d_closed = per_kernel_closed["assemble"]["ms_per_step"]
    return {"density": f"random, rank {N} ({(N + 15) // 16} groups of factors in step (c))", "seconds_per_build": sec,
            "fields_ms": tm["fields"][0], "step_d_gemm_ms": d_ms, "step_d_gemm_vs_rank7_build": d_ms / d_closed,
            "note": "wall time of one build, inputs on the device, Delta U not unpacked; step_d_gemm_ms = the "
                    "step (d) GEMM launches (one per chunk for any density rank)"}


def large_measure(args, torch, dev, local):
    """The large workload (4 heavy atoms + 4 H, N=200, 200,000 grid points, 8 Jastrow centres in
    2 sets, 14 doubly occupied orbitals): one warm-up and one timed build (CUDA events), inputs and
    outputs on the device, Delta U formed but not unpacked."""
    from paper_2304_07006_gb300 import Context

    p = synth_config("large")
    F = flops(p.n_orb, p.n_grid)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grid, w, phi, gam = t(p.grid), t(p.weights), t(p.phi), t(p.gamma)
    dh = torch.empty((p.n_orb, p.n_orb), dtype=torch.float64, device=dev)
    e0 = torch.empty(1, dtype=torch.float64, device=dev)
    with Context(args.precision, device=local) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.build(grid, w, phi, gam, dh=dh, e0=e0, want_dU=False)
        stream = torch.cuda.current_stream(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        c.build(grid, w, phi, gam, dh=dh, e0=e0, want_dU=False)
        b.record(stream)
        torch.cuda.synchronize(dev)
        sec = a.elapsed_time(b) / 1e3
    return {"workload": f"large: N={p.n_orb}, {p.n_grid} grid points, {len(p.nuc_xyz)} Jastrow centres",
            "seconds_per_build": sec, "algorithmic_flops": F["total"], "tflops": F["total"] / sec / 1e12,
            "note": "inputs and outputs on the device; Delta U not unpacked"}


def three_body_measure(args, torch, dev, local):
    """The explicit three-body tensor of eq. Ldecomp on the H2-like workload (N=10, 2,000 grid
    points, FP64 path): one warm-up and three timed calls, output on the device."""
    from paper_2304_07006_gb300 import Context

    p = synth_config("h2")
    N, NP = p.n_orb, p.n_orb * (p.n_orb + 1) // 2
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grid, w, phi = t(p.grid), t(p.weights), t(p.phi)
    L = torch.empty((N,) * 6, dtype=torch.float64, device=dev)
    with Context("fp64", device=local) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.three_body_L(grid, w, phi, out=L)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            c.three_body_L(grid, w, phi, out=L)
        torch.cuda.synchronize(dev)
        sec = (time.perf_counter() - t0) / 3
    flops_t = 2.0 * NP ** 3 * p.n_grid + 6.0 * NP ** 2 * p.n_grid
    return {"workload": f"h2: N={N}, {p.n_grid} grid points, FP64", "seconds_per_call": sec,
            "elements": N ** 6, "t_flops": flops_t,
            "note": "wall time per call with steps (a)+(b) in FP64; L is written densely on the device"}


def two_body_k_measure(args, torch, dev, local):
    """The two-body integrals K (Theory section) on the H2-like workload (N=10, 2,000 grid points,
    FP64 path): one warm-up and three timed calls, inputs and output on the device.  FP64 FLOPs of
    the two contractions: W = (w F) P (2 n_grid^2 n_pair) and S (2 x 4 n_grid x N^2 x n_pair)."""
    import synth
    from paper_2304_07006_gb300 import Context

    p = synth_config("h2")
    N, NP, NG = p.n_orb, p.n_orb * (p.n_orb + 1) // 2, p.n_grid
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grid, w, phi, dphi = t(p.grid), t(p.weights), t(p.phi), t(synth.orbital_gradients(p))
    K = torch.empty((N,) * 4, dtype=torch.float64, device=dev)
    with Context("fp64", device=local) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.two_body_K(grid, w, phi, dphi, out=K)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            c.two_body_K(grid, w, phi, dphi, out=K)
        torch.cuda.synchronize(dev)
        sec = (time.perf_counter() - t0) / 3
    flops = 2.0 * NG * NG * NP + 8.0 * NG * N * N * NP
    return {"workload": f"h2: N={N}, {NG} grid points, FP64", "seconds_per_call": sec,
            "contraction_flops": flops, "gflops": flops / sec / 1e9,
            "note": "wall time per call: steps (a)+(b) for V, the Laplacian table (n_grid^2 pairs), the two "
                    "FP64 contractions and the unpack into K[p][q][r][s]"}


def frozen_core_measure(args, torch, dev, local, peaks):
    """The xTC-FC folding at N=120 (two core orbitals, the 1s pair of the N2-like workload) of
    device-resident Delta U / Delta h: one warm-up and five timed calls.  The fold is a gather of
    the active block (8 B read + 8 B written per element) plus O(N^2 n_core) sums."""
    from paper_2304_07006_gb300 import Context

    N, core = 120, [0, 1]
    n_act = N - len(core)
    gen = torch.Generator(device=dev).manual_seed(11)
    a = torch.randn((N,) * 4, dtype=torch.float64, device=dev, generator=gen)
    dU = (a + a.permute(2, 3, 0, 1)) * 0.5
    del a
    dh = torch.randn((N, N), dtype=torch.float64, device=dev, generator=gen)
    dh_fc = torch.empty((n_act, n_act), dtype=torch.float64, device=dev)
    dU_act = torch.empty((n_act,) * 4, dtype=torch.float64, device=dev)
    e = torch.empty(1, dtype=torch.float64, device=dev)
    with Context(args.precision, device=local) as c:
        c.frozen_core_fold(dU, dh, core, dh_fc=dh_fc, dU_act=dU_act, e_core=e)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(5):
            c.frozen_core_fold(dU, dh, core, dh_fc=dh_fc, dU_act=dU_act, e_core=e)
        torch.cuda.synchronize(dev)
        sec = (time.perf_counter() - t0) / 5
    nbytes = 16.0 * n_act ** 4
    hbm = peaks.get("hbm_gbs", 6800.0)
    return {"workload": f"N={N}, core {core}, Delta U and Delta h on the device", "seconds_per_call": sec,
            "achieved_gbs": nbytes / sec / 1e9, "frac_hbm": nbytes / sec / 1e9 / hbm,
            "note": "wall time per C-ABI call (three kernels, synchronous); bytes = 16 x n_act^4"}


def synth_config(name):
    import synth
    return synth.make_config(name)


def run_ncu_case(args):
    """A small, quick build (same workload, outer sum restricted to P points) for kernel captures."""
    import synth
    from paper_2304_07006_gb300 import Context

    p = synth.make_config(WORKLOAD)
    with Context(args.precision) as c:
        c.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
        c.set_outer_range(0, args.ncu_case)
        for _ in range(2):
            out = c.build(p.grid, p.weights, p.phi, p.gamma, want_dU=False)
    print(f"ncu case: {WORKLOAD}, {args.precision}, outer points [0, {args.ncu_case}), e0 {float(out['e0'][0]):.12e}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x2", choices=["fp16x2", "bf16x3"])
    ap.add_argument("--fp64-sample", type=int, default=1024, help="outer points for the FP64 GPU comparison")
    ap.add_argument("--cpu-sample", type=int, default=4, help="outer points for the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--batched", type=int, default=32, metavar="N",
                    help="also time the batched workload of N uneven instances (0: skip)")
    ap.add_argument("--rohf", type=int, default=1, help="also time the spin-resolved build (0: skip)")
    ap.add_argument("--large", type=int, default=1, help="also time one build of the N=200 workload (0: skip)")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="P",
                    help="profiling aid: run one warm-up and one build of the workload restricted to the first P "
                         "outer points, print a one-line summary and exit (no benchmark line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.ncu_case > 0:
        run_ncu_case(args)
        return

    import torch
    import synth
    from paper_2304_07006_gb300 import Context
    from paper_2304_07006_gb300.xtc import KERNEL_NAMES

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    p = synth.make_config(WORKLOAD)
    N, NG = p.n_orb, p.n_grid
    F = flops(N, NG)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grid, w, phi, gamma = t(p.grid), t(p.weights), t(p.phi), t(p.gamma)
    dU = torch.empty((N,) * 4, dtype=torch.float64, device=dev)
    dh = torch.empty((N, N), dtype=torch.float64, device=dev)
    e0 = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = Context(args.precision, device=local, stream=stream.cuda_stream, timing=True)
    ctx.set_jastrow(p.nuc_xyz, p.nuc_set, p.terms, p.coef)
    run = lambda: ctx.build(grid, w, phi, gamma, dU=dU, dh=dh, e0=e0)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms = np.zeros(len(KERNEL_NAMES))
    kern_n = np.zeros(len(KERNEL_NAMES), dtype=np.int64)
    ev0.record(stream)
    for _ in range(args.steps):
        run()
        tm = ctx.timings()
        kern_ms += np.array([v[0] for v in tm.values()])
        kern_n += np.array([v[1] for v in tm.values()])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms_step, value = job_throughput(ev0.elapsed_time(ev1), args.steps, world, F["total"], dist, dev)

    # roofline of the dominant kernel: step (b), per-launch algorithmic flops / mean launch time
    per_kernel = {name: {"ms_per_step": kern_ms[k] / args.steps, "launches_per_step": int(kern_n[k] // args.steps)}
                  for k, name in enumerate(KERNEL_NAMES)}
    # one gradient-table launch per chunk; "vfield" and "assemble" time the step (b) and step (d)
    # GEMMs alone, "aux" the kernels around them (V and M from the FP64 tile sums, row splits)
    n_vf = kern_n[KERNEL_NAMES.index("grad")] / args.steps
    vf_ms = kern_ms[1] / args.steps / n_vf
    vf_flops_launch = F["b"] / n_vf
    peaks, peak_src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    achieved = vf_flops_launch / (vf_ms * 1e-3) / 1e12
    issued_factor = 3 if args.precision == "fp16x2" else 6
    # DRAM bytes of the step (b) kernel from the ncu capture (fp16x2, VFIELD_CAPTURE_OUTER outer
    # points), scaled by the outer points of a launch (traffic grows with the row tiles); only for
    # the engine revision that was captured
    from paper_2304_07006_gb300.xtc import engine_revision
    traffic = None
    if (args.precision == "fp16x2" and VFIELD_DRAM_BYTES_CAPTURED
            and engine_revision() == VFIELD_CAPTURE_REVISION):
        traffic = VFIELD_DRAM_BYTES_CAPTURED * (NG / n_vf) / VFIELD_CAPTURE_OUTER
    roofline = {"kernel": "vfield_tc (step b: tcgen05 split-fp16 GEMM V = G rho^T)",
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_src} bf16 dense sustained (fp16 nominal ratio 1:1)",
                "issued_tflops": achieved * issued_factor,
                "issued_frac": achieved * issued_factor / peak,
                "ms_per_chunk": vf_ms, "algorithmic_flops_per_chunk": vf_flops_launch}
    asm_ms = kern_ms[3] / args.steps / n_vf
    asm_ach = F["d"] / n_vf / (asm_ms * 1e-3) / 1e12
    # fp16x2 issues three split products per algorithmic one in both GEMMs (hi x hi, hi x lo,
    # lo x fp16(B)); bf16x3 six
    asm_factor = 3 if args.precision == "fp16x2" else 6
    aux_ms = kern_ms[KERNEL_NAMES.index("aux")] / args.steps / n_vf
    assemble = {"kernel": "step d GEMM per chunk (fp16x2: vfield_tc in mode 1 on the split rows of L and R)",
                "bound": "tensor", "achieved": asm_ach, "issued_tflops": asm_ach * asm_factor,
                "frac": asm_ach / peak, "issued_frac": asm_ach * asm_factor / peak, "ms_per_chunk": asm_ms,
                "aux_ms_per_chunk": aux_ms,
                "note": "aux = the row splits of L and R, the add into M and the V write of step (b)"}

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "seconds_per_build": ms_step / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x2 split (steps b and d), f32 tensor accumulate, f64 flushes and chunk sums"
            if args.precision == "fp16x2" else "bf16x3 split (steps b and d), f32 tensor accumulate, f64 sums",
            "data": "synthetic", "config": config_dict(p, args.precision),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "algorithmic_flops_per_build": F, "roofline": roofline, "assemble_roofline": assemble,
            "per_kernel": per_kernel, "clocks": clk,
            "gpu_launches": int(kern_n.sum())}

    if rank == 0:
        # FP64 GPU path and the mixed error, on sampled outer points (same kernels, outer range)
        rng = np.random.default_rng(7)
        perm = rng.permutation(NG)
        ps = synth.permute_grid(p, perm)
        S = args.fp64_sample
        res = {}
        for prec in ("fp64", args.precision):
            with Context(prec, device=local, timing=True) as c:
                c.set_jastrow(ps.nuc_xyz, ps.nuc_set, ps.terms, ps.coef)
                c.set_outer_range(0, S)
                c.build(ps.grid, ps.weights, ps.phi, ps.gamma, want_dU=False)  # warm-up
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                out = c.build(ps.grid, ps.weights, ps.phi, ps.gamma)
                dt = time.perf_counter() - t0
                tm = c.timings()
                dev_ms = sum(v[0] for k, v in tm.items() if k != "prep")
                res[prec] = (out, dt, dev_ms, tm)
        full_fp64_s = res["fp64"][2] / 1e3 * NG / S
        err = {k: float(np.abs(np.asarray(res[args.precision][0][k]) - np.asarray(res["fp64"][0][k])).max())
               for k in ("dU", "dh", "e0")}
        line["fp64_path"] = {"sample_outer_points": S, "device_ms_on_sample": res["fp64"][2],
                             "seconds_per_build_extrapolated": full_fp64_s,
                             "tflops_extrapolated": F["total"] / full_fp64_s / 1e12,
                             "mixed_speedup_vs_fp64": full_fp64_s / (ms_step / 1e3)}
        # the outputs are sums over outer points: an error that grows with the outer sum (a
        # one-signed bias) reaches NG / S times the sample's on the whole grid; random errors less
        line["error_eh_vs_fp64_gpu"] = {
            "sample": {k: v for k, v in err.items()},
            "whole_grid_extrapolated": {k: v * NG / S for k, v in err.items()},
            "note": f"max |mixed - FP64 GPU| over every Delta U / Delta h entry and the constant on {S} random outer "
                    f"points (full inner sum); whole_grid_extrapolated = sample x {NG}/{S}, the bound for an error "
                    f"that grows linearly with the outer sum"}

        # end to end through the C ABI with pinned host buffers (copies inside the timed region)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hg, hw, hphi, hgam = pin(p.grid), pin(p.weights), pin(p.phi), pin(p.gamma)
        hdU = torch.empty((N,) * 4, dtype=torch.float64).pin_memory()
        hdh = torch.empty((N, N), dtype=torch.float64).pin_memory()
        he0 = torch.empty(1, dtype=torch.float64).pin_memory()
        ctx.build(hg, hw, hphi, hgam, dU=hdU, dh=hdh, e0=he0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.build(hg, hw, hphi, hgam, dU=hdU, dh=hdh, e0=he0)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        h2d = sum(int(a.numel()) * 8 for a in (hg, hw, hphi, hgam))
        d2h = sum(int(a.numel()) * 8 for a in (hdU, hdh, he0))
        line["e2e"] = {"value": F["total"] / dt / 1e12, "unit": "TFLOP/s", "seconds_per_build": dt,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        if args.batched:
            line["batched"] = batched_measure(args, torch, dev, local)
        if args.rohf:
            line["rohf"] = rohf_measure(args, torch, dev, local, p, ms_step / 1e3)
        line["three_body_L"] = three_body_measure(args, torch, dev, local)
        line["two_body_K"] = two_body_k_measure(args, torch, dev, local)
        line["full_rank_density"] = fullrank_measure(args, torch, dev, local, p, per_kernel)
        line["frozen_core_fold"] = frozen_core_measure(args, torch, dev, local, peaks)
        if args.large:
            free, _ = torch.cuda.mem_get_info(dev)
            line["large"] = (large_measure(args, torch, dev, local) if free > 100e9
                             else {"skipped": f"{free / 1e9:.0f} GB free on the device, 100 GB wanted"})
        line["cpu_baseline"] = oracle_sample(p, args.cpu_sample)
        line["cpu_baseline"].pop("seconds", None)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
