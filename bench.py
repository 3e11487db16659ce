"""Benchmark: deflated Hutchinson samples/s at true relative residual 1e-8.

Default workload (the mixed-precision estimator configuration of the
metric): Wilson-Dirac operator on a 16^3 x 32 periodic lattice
(N = 1,572,864), random SU(3) links exp(i 0.2 H) (seed 3), m0 = -0.8;
three-level multigrid (2^4 then 2^4 aggregates, 12 and 16 null vectors per
chirality, FP32 null-vector iterations; level-1 GCR of 6 iterations, one
minimal-residual smoothing step on the coarse levels, dense coarsest inverse
applied on tensor cores); Algorithm 2 deflation of rank 24 on the coarsest
level; 128 real Rademacher samples per step solved together, each to
||b - A x|| <= 1e-8 ||b|| on the FP64 residual.  The path: FP32 flexible
GCR(4) on the odd-site Schur complement (even-odd solve) and the FP32
V-cycle (two-layer learned smoother on the fine level with no MR step after
it, tensor-core coarse stencil and restriction) inside FP64 residual
refinement.  The plain FP64 form (full-lattice FP64 GCR(16) and V-cycle,
plain minimal-residual smoother) is timed on the same lattice
("fp64_path").

A step = one batch through the whole sample path: Rademacher noise (a1),
deflation projection (a8, with the Wilson and transfer kernels), the
multigrid-preconditioned solves (a2-a6) and the trace statistics (a9).  The
adaptive setup, the smoother training and the deflation space (a7, a10) are
built once before timing and reported as setup_s; the end-to-end number
repeats them every step.

Errors against the FP64 oracle ("errors"): the true residual of
mixed-precision solutions recomputed with the oracle's operator; and, on the
unit-link twin of the workload (same lattice and path, links = 1), the
estimate against the oracle's closed-form tr A^{-1} in standard errors and
the undeflated sample variance against the oracle's closed-form exact
variance, with the variance reduction from deflation.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) each rank takes its own sample range (replicas: the
samples are independent); the per-sample values are gathered on the host and
rank 0 reports the whole run's estimate.
"""

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Config 3: 16^3 x 32, eps 0.2 (seed 3), m0 -0.8, three levels, 128 samples
# per step, mixed precision with the learned smoother (the metric's form).
CONFIG3 = dict(
    workload="wilson-dirac 16^3x32 eps0.2 seed3 m0=-0.8, 3-level MG (2^4, 2^4; nv 12, 16; level-1 GCR 6 its; "
             "coarse MR 1), Algorithm 2 k=24 on the coarsest level, 128 Rademacher samples/step, two-layer learned "
             "smoother, even-odd (odd-site Schur complement) FP32 GCR(4) inner solves with FP64 refinement to true "
             "rel. residual 1e-8",
    dims=(16, 16, 16, 32), eps=0.2, link_seed=3, m0=-0.8, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvs=[12, 16],
    k=24, guard=16, s=128, tol=1e-8, noise_seed=103, restart=4, maxit=500, inner_tol=1e-5, schur=1,
    mg_kw={"coarse_tol": 0.0, "coarse_maxit": 6, "coarse_smoother_steps": 1, "null_f32": 1},
    learned=1, learned_mr=0, layers=2, eig_maxit=30, fp64_samples=16,
)
# Config 2: 8^4 lattice, two-level multigrid, kept for comparison with
# earlier numbers.
CONFIG2 = dict(
    workload="wilson-dirac 8^4 eps0.3 seed2 m0=-0.8, 2-level MG (2^4 blocks, nv 12; learned smoother + 1 MR), "
             "Algorithm 2 k=24, 64 Rademacher samples/step, true FP64 rel. residual 1e-8",
    dims=(8, 8, 8, 8), eps=0.3, link_seed=2, m0=-0.8, blocks=[(2, 2, 2, 2)], nvs=[12], k=24, guard=16,
    s=64, tol=1e-8, noise_seed=102, restart=16, maxit=500, inner_tol=1e-5, learned=1, eig_maxit=30,
    fp64_samples=64,
)
WORKLOADS = {"config3": CONFIG3, "config2": CONFIG2}
WL = dict(CONFIG3)
# Config 4: an uneven batch solved concurrently (qd_hutchinson_batch):
# (lattice, m0, samples) = (8^4, -0.6, 16), (12^4, -0.75, 48), (16^4, -0.8,
# 96); eps 0.2 links (seeds 4, 5, 6), three-level MG (2^4, 2^4; nv 12, 16)
# with a fixed 6-iteration level-1 GCR so that each V-cycle is one graph,
# Algorithm 2 k = 24, mixed precision to a true FP64 residual 1e-8.
BATCH = dict(
    workload="uneven batch: wilson-dirac 8^4 m0=-0.6 x16, 12^4 m0=-0.75 x48, 16^4 m0=-0.8 x96 samples; eps0.2 "
             "seeds 4-6; 3-level MG (2^4, 2^4; nv 12, 16; level-1 GCR 6 its); Algorithm 2 k=24; true FP64 rel. "
             "residual 1e-8; one concurrent batch per step",
    problems=[((8, 8, 8, 8), 4, -0.6, 16), ((12, 12, 12, 12), 5, -0.75, 48), ((16, 16, 16, 16), 6, -0.8, 96)],
    eps=0.2, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvs=[12, 16], mg_kw={"coarse_tol": 0.0, "coarse_maxit": 6},
    k=24, guard=16, tol=1e-8, restart=16, maxit=500, inner_tol=1e-5,
)
HERE = os.path.dirname(os.path.abspath(__file__))
METRIC = "deflated Hutchinson samples/s @res 1e-8"
UNIT = "samples/s"
# Recipe peaks (MEASURED_PEAKS.json holds HBM and bf16; FP64 is the recipe's
# nominal 1.25 TFLOP/s, matching the 1.20 TFLOP/s an FMA-chain probe measured).
FP64_PEAK_TFLOPS = 1.25
# Outer GCR iterations per sample of the plain FP64 path on the config-3
# workload (the fp64_path leg measures 49-50); the oracle arm's time per
# iteration is scaled by it when the run itself has no FP64 leg.
# FP32 CUDA-core peak from the unit counts and the maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_ITERS_CONFIG3 = 50


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic(workload, kind):
    """DRAM bytes per launch of `kind` on `workload` from the committed ncu
    summary, if the kernel's source is unchanged since it was taken."""
    import hashlib
    path = os.path.join(HERE, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            entries = json.load(f)["entries"]
    except (OSError, ValueError, KeyError):
        return None
    for e in entries:
        if e.get("workload") == workload and e.get("kind") == kind:
            try:
                with open(os.path.join(HERE, e["source"]), "rb") as f:
                    if hashlib.sha256(f.read()).hexdigest() != e["sha256"]:
                        return None
            except OSError:
                return None
            return e["bytes_per_launch"]
    return None


def _mg_params(qd, wl=None):
    wl = WL if wl is None else wl
    return qd.mg_params(len(wl["blocks"]), wl["blocks"], wl["nvs"], **wl.get("mg_kw", {}))


def _learned_mr(wl):
    """Minimal-residual steps after the learned smoother."""
    return wl.get("learned_mr", wl.get("learned", 0))


def _setup(qd, ctx, U, wl=None):
    """Gauge, hierarchy, learned smoother, deflation space for the workload."""
    wl = WL if wl is None else wl
    g = qd.Gauge(ctx, wl["dims"], U)
    mg = qd.Multigrid(ctx, g, wl["m0"], 0.0, _mg_params(qd, wl))
    judge = None
    if wl.get("learned"):
        judge = qd.smoother_train(mg, nsamples=4, solve_tol=1e-3, mr_steps=_learned_mr(wl),
                                  layers=wl.get("layers", 1))
        qd.smoother_enable(mg, True, _learned_mr(wl))
    d = qd.Deflation(ctx, g, mg, wl["m0"], 0.0,
                     qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, wl["k"], guard=wl["guard"], eig_tol=1e-6,
                                    solve_tol=1e-10, maxit=wl.get("eig_maxit", 60)))
    return g, mg, d, judge


def _batch(qd, ctx, g, mg, d, offset, precision, nsamples=None, wl=None, plain=False):
    """One estimator batch; plain=True: full-lattice GCR(16) (the plain FP64
    path), whatever the workload's even-odd and restart settings."""
    wl = WL if wl is None else wl
    if plain:
        wl = dict(wl, restart=16, schur=0)
    return qd.hutchinson_trace(ctx, g, mg, d, wl["m0"], 0.0, seed=wl["noise_seed"], sample_offset=offset,
                               nsamples=wl["s"] if nsamples is None else nsamples, tol=wl["tol"], maxit=wl["maxit"],
                               restart=wl["restart"], precision=precision, inner_tol=wl["inner_tol"], max_refine=10,
                               **({"schur": wl["schur"]} if wl.get("schur") else {}))


def _oracle_iteration_seconds(dims, eps, link_seed, m0, blocks, nvs, mg_kw, noise_seed, iters=1):
    """Seconds of one outer V-cycle-preconditioned FP64 GCR iteration of the
    oracle on the workload's lattice (the same operator sizes, transfers and
    V-cycle shape as the plain FP64 path: fine MR(4), coarse MR steps and
    fixed coarse GCR iterations as the workload sets them).  The oracle's
    null-vector iteration is capped at 2 steps: its setup (single-threaded
    sparse products, ~15 min at 16^3 x 32 for 200 steps) is untimed and the
    per-iteration cost does not depend on the null vectors' quality."""
    from oracle import krylov, philox
    from oracle import multigrid as omg
    from paper_1909_12234_gb300 import synth
    U = synth.random_su3_links(dims, eps, link_seed)
    H = omg.setup(U, m0, dims, blocks, nvs, seed=7, null_maxit=2, smoother_steps=4,
                  coarse_tol=mg_kw.get("coarse_tol", 0.1), coarse_maxit=mg_kw.get("coarse_maxit", 256),
                  coarse_smoother_steps=mg_kw.get("coarse_smoother_steps"))
    lev = H.levels[0]
    z = philox.rademacher(lev.n, noise_seed, range(1)).astype(np.complex128)[:, 0]
    t = time.perf_counter()
    krylov.gcr(lev.matvec, z, 0.0, maxit=iters, restart=16, precond=lambda r: H.vcycle(0, r))
    return (time.perf_counter() - t) / iters


def cpu_baseline(iters_per_sample):
    """The FP64 oracle on this host's cores, on a bounded sample of the
    workload: one outer iteration of one sample, scaled to samples/s by the
    outer iterations a sample of the plain FP64 algorithm takes."""
    kw = {k: WL[k] for k in ("dims", "eps", "link_seed", "m0", "blocks", "nvs", "noise_seed")}
    sec = _oracle_iteration_seconds(mg_kw=WL.get("mg_kw", {}), **kw)
    return {"value": 1.0 / (sec * iters_per_sample), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one outer V-cycle-preconditioned FP64 GCR iteration of one sample on the workload lattice "
                      f"({sec:.1f} s, oracle setup untimed, null-vector steps capped at 2), times "
                      f"{iters_per_sample} iterations per sample (the plain FP64 path's count); numpy/scipy FP64, "
                      f"sparse products single-threaded"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    kw = {k: WL[k] for k in ("dims", "eps", "link_seed", "m0", "blocks", "nvs", "noise_seed")}
    iters_per_sample = FP64_ITERS_CONFIG3 if WL["dims"] == CONFIG3["dims"] else 28
    from oracle import krylov, philox
    from oracle import multigrid as omg
    from paper_1909_12234_gb300 import synth
    U = synth.random_su3_links(WL["dims"], WL["eps"], WL["link_seed"])
    mg_kw = WL.get("mg_kw", {})
    H = omg.setup(U, WL["m0"], WL["dims"], WL["blocks"], WL["nvs"], seed=7, null_maxit=2, smoother_steps=4,
                  coarse_tol=mg_kw.get("coarse_tol", 0.1), coarse_maxit=mg_kw.get("coarse_maxit", 256),
                  coarse_smoother_steps=mg_kw.get("coarse_smoother_steps"))
    lev = H.levels[0]
    Z = philox.rademacher(lev.n, WL["noise_seed"], range(args.warmup + args.steps)).astype(np.complex128)

    def step(i):  # one outer iteration of sample i
        krylov.gcr(lev.matvec, Z[:, i], 0.0, maxit=1, restart=16, precond=lambda r: H.vcycle(0, r))

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = (time.perf_counter() - t) / args.steps
    value = 1.0 / (dt * iters_per_sample)
    sample = (f"each step one outer V-cycle-preconditioned FP64 GCR iteration of one sample ({dt:.1f} s); "
              f"samples/s = 1 / (seconds per iteration x {iters_per_sample} iterations per sample of the plain "
              f"FP64 algorithm); oracle setup untimed with null-vector steps capped at 2")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt * iters_per_sample,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WL["workload"] + "; reference = the FP64 oracle (numpy/scipy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def stencil_roofline(qd, ctx, reps=20):
    """The Wilson stencil alone (FP32 and FP64) on the 16^3 x 32 lattice with
    64 right-hand sides: every field is larger than L2, so no flush is needed.
    Algorithmic bytes per launch: spinor in + out once, links once,
    V (24 nrhs + 36) complex words; flops 1368 per site and right-hand side."""
    import torch
    from paper_1909_12234_gb300 import synth
    dims, nrhs = (16, 16, 16, 32), 64
    U = synth.random_su3_links(dims, 0.2, 3)
    g = qd.Gauge(ctx, dims, U)
    V = g.V
    hbm = _peaks().get("hbm_gbs", 6800.0)
    out = {"lattice": "16^3x32", "nrhs": nrhs, "peak_gbs": hbm, "l2": "fields 0.8-1.6 GB > L2"}
    for name, dt, fn, cb in (("f32", torch.complex64, qd.dirac_apply_f32, 8),
                             ("f64", torch.complex128, qd.dirac_apply, 16)):
        x = torch.randn((V, 12, nrhs), dtype=dt, device=f"cuda:{ctx.device}")
        y = torch.empty_like(x)
        for _ in range(3):
            fn(ctx, g, -0.8, 0.0, False, nrhs, x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(reps):
            fn(ctx, g, -0.8, 0.0, False, nrhs, x, y)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = V * (24.0 * cb * nrhs + 36.0 * cb)
        gbs = nbytes / (ms / 1e3) / 1e9
        out[name] = {"ms_per_launch": ms, "achieved_gbs": gbs, "frac": gbs / hbm,
                     "tflops": 1368.0 * V * nrhs / (ms / 1e3) / 1e12}
        del x, y
    g.close()
    return out


def kernel_only(qd, ctx, names, reps=20):
    """Hot kernels alone on the shapes of the 16^3 x 32 workload (a profiling
    target): the FP32 V-cycle's level-1 stencil on tensor cores (8192 sites,
    D = 24, split pass included), the restriction fine -> level 1 on tensor
    cores, the FP32 prolongation level 1 -> fine and level 2 -> level 1, and
    the FP32 Wilson stencil (A x, the residual b - A x, and the odd-site
    Schur complement through the parity-restricted hops); 128 right-hand
    sides.  The hierarchy takes
    random blocked vectors (no null-vector iteration: the kernels' cost does
    not depend on W) and no dense coarsest inverse.  Algorithmic bytes as in
    the bench's per-kernel table; every field is larger than L2 except the
    level-2 field."""
    import torch
    from paper_1909_12234_gb300 import synth
    dims, s = (16, 16, 16, 32), 128
    U = synth.random_su3_links(dims, 0.2, 3)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.8, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], null_maxit=0,
                                                       seed=5, coarsest_direct=0))
    dev = f"cuda:{ctx.device}"
    hbm = _peaks().get("hbm_gbs", 6800.0)
    V = g.V
    n1, n2 = 8192 * 24, 512 * 32
    x0 = torch.randn((V * 12, s), dtype=torch.complex64, device=dev)
    y0 = torch.empty_like(x0)
    b0 = torch.randn((V * 12, s), dtype=torch.complex64, device=dev) if "wilson_resid_f32" in names else None
    xh = torch.randn((V // 2 * 12, s), dtype=torch.complex64, device=dev) if "schur_f32" in names else None
    yh = torch.empty_like(xh) if xh is not None else None
    x1 = torch.randn((n1, s), dtype=torch.complex64, device=dev)
    y1 = torch.empty_like(x1)
    x2 = torch.randn((n2, s), dtype=torch.complex64, device=dev)
    cases = {
        "coarse_tc": (lambda: qd.coarse_apply_tc(mg, 1, s, x1, y1), 8192 * (9 * 24 * 24 * 8.0 + 2 * 24 * 8.0 * s)),
        "restrict_tc": (lambda: qd.restrict_tc(mg, 0, s, x0, x1),
                        8.0 * (V * 12 * 12 + V * 12 * s + 8192 * 24 * s)),
        "prolong_l1": (lambda: qd.prolongate_f32(mg, 0, s, x1, y0), 8.0 * (V * 12 * 12 + V * 12 * s + n1 * s)),
        "prolong_l2": (lambda: qd.prolongate_f32(mg, 1, s, x2, y1), 8.0 * (8192 * 24 * 16 + n1 * s + n2 * s)),
        "wilson_f32": (lambda: qd.dirac_apply_f32(ctx, g, -0.8, 0.0, False, s, x0, y0), V * (24.0 * 8 * s + 36.0 * 8)),
        "wilson_resid_f32": (lambda: qd.dirac_residual_f32(ctx, g, -0.8, 0.0, False, s, b0, x0, y0),
                             V * (36.0 * 8 * s + 36.0 * 8)),
        # the entry point also allocates its half-field scratch and synchronises
        "schur_f32": (lambda: qd.dirac_schur_apply_f32(ctx, g, -0.8, 0.0, s, xh, yh),
                      (V // 2) * (60.0 * 8 * s + 144.0 * 8)),
        "smoother_f32": (lambda: qd.smoother_apply_f32(mg, s, x0, y0), V * (24.0 * 8 * s + 36.0 * 8)),
    }
    if "smoother_f32" in names:
        rng = np.random.default_rng(1)
        qd.smoother_set_weights(mg, 0.1 * (rng.standard_normal((9, 4, 4)) + 1j * rng.standard_normal((9, 4, 4))))
    out = {"lattice": "16^3x32", "nrhs": s, "peak_gbs": hbm}
    for name in names:
        fn, nbytes = cases[name]
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(reps):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes / (ms / 1e3) / 1e9
        out[name] = {"ms_per_launch": ms, "alg_bytes": nbytes, "achieved_gbs": gbs, "frac": gbs / hbm}
    out["autotune"] = qd.autotune_report()
    for o in (mg, g):
        o.close()
    return out


def errors_against_oracle(qd, ctx, U, g, mg, d):
    """Errors of the GPU path against the FP64 oracle (see the module docstring)."""
    import torch
    from oracle import lattice, wilson
    from paper_1909_12234_gb300 import synth
    out = {}
    dims, m0, tol = WL["dims"], WL["m0"], WL["tol"]
    # (1) mixed-precision solutions of two deflated samples: true residual
    # with the oracle's (matrix-free) operator, and the FP64 path's solution
    ncol = 2
    z = torch.empty((g.V, 12, ncol), dtype=torch.complex128, device=f"cuda:{ctx.device}")
    qd.rademacher(ctx, g, WL["noise_seed"], 10 ** 6, ncol, z)
    b = torch.empty_like(z)
    d.project(ncol, z, b)
    xm, x64 = torch.empty_like(b), torch.empty_like(b)
    qd.solve(ctx, g, mg, m0, 0.0, ncol, b, xm, tol, maxit=WL["maxit"], restart=WL["restart"],
             precision=qd.QD_PREC_MIXED, inner_tol=WL["inner_tol"], max_refine=10, schur=WL.get("schur", 0))
    qd.solve(ctx, g, mg, m0, 0.0, ncol, b, x64, tol, maxit=WL["maxit"])
    torch.cuda.synchronize()
    eo = lattice.eo_index(dims)
    bl = b.cpu().numpy()[eo].reshape(-1, 4, 3, ncol)
    res = {}
    for name, x in (("mixed", xm), ("fp64", x64)):
        xl = x.cpu().numpy()[eo].reshape(-1, 4, 3, ncol)
        r = bl - wilson.dirac_apply(U, xl, m0, dims)
        res[name] = (np.linalg.norm(r.reshape(-1, ncol), axis=0) / np.linalg.norm(bl.reshape(-1, ncol), axis=0))
    dx = (torch.linalg.vector_norm(xm - x64, dim=(0, 1)) / torch.linalg.vector_norm(x64, dim=(0, 1))).cpu().numpy()
    out["solution"] = {"samples": ncol, "tol": tol,
                       "oracle_true_rel_residual_mixed": float(res["mixed"].max()),
                       "oracle_true_rel_residual_fp64": float(res["fp64"].max()),
                       "rel_diff_mixed_vs_fp64": float(dx.max()),
                       "scope": "two deflated samples of the workload, GPU solutions, residual b - A x computed by "
                                "the oracle's operator on the host"}
    # (2) the unit-link twin: same lattice, hierarchy, smoother, deflation and
    # precisions, links = 1; exact trace and variance from the oracle
    Ut = synth.random_su3_links(dims, 0.0, 0, unit=True)
    gt, mgt, dt, _ = _setup(qd, ctx, Ut)
    s = WL["s"]
    _batch(qd, ctx, gt, mgt, dt, 0, qd.QD_PREC_MIXED)  # warm-up (graphs)
    rd = _batch(qd, ctx, gt, mgt, dt, 0, qd.QD_PREC_MIXED)
    ru = _batch(qd, ctx, gt, mgt, None, 0, qd.QD_PREC_MIXED)
    exact = wilson.free_field_trace_inverse(dims, m0)
    var_exact = wilson.free_field_variance_real_rademacher(dims, m0)
    out["unit_link_twin"] = {
        "samples": s, "exact_trace": exact, "estimate": rd["estimate"].real, "stderr": rd["stderr"],
        "deviation_in_stderr": (rd["estimate"].real - exact) / rd["stderr"],
        "undeflated_estimate": ru["estimate"].real, "undeflated_stderr": ru["stderr"],
        "undeflated_deviation_in_stderr": (ru["estimate"].real - exact) / ru["stderr"],
        "undeflated_var": ru["var"], "undeflated_var_jackknife_err": ru["var_jackknife_err"],
        "oracle_exact_undeflated_var": var_exact,
        "undeflated_var_over_exact": ru["var"] / var_exact,
        "deflated_var": rd["var"], "variance_reduction": ru["var"] / rd["var"],
        "max_true_rel_residual": max(rd["max_true_rel_residual"], ru["max_true_rel_residual"]),
        "scope": "exact tr A^-1 and exact Var of the undeflated estimator: oracle closed forms (free field)"}
    for o in (dt, mgt, gt):
        o.close()
    return out


def run_ours(args):
    import torch
    from paper_1909_12234_gb300 import parallel
    from paper_1909_12234_gb300 import qdtrace as qd
    from paper_1909_12234_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    qd.load()
    ctx = qd.Context(local)
    stream = ctx.stream
    U = synth.random_su3_links(WL["dims"], WL["eps"], WL["link_seed"])
    torch.cuda.synchronize()
    t = time.perf_counter()
    g, mg, d, judge = _setup(qd, ctx, U)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    s = WL["s"]

    def offset(i):
        return parallel.sample_offset(rank, world, s, i)

    prec = qd.QD_PREC_MIXED if args.precision == "mixed" else qd.QD_PREC_F64
    for i in range(args.warmup):
        _batch(qd, ctx, g, mg, d, offset(i), prec)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = qd.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    results = []
    for i in range(args.steps):
        results.append(_batch(qd, ctx, g, mg, d, offset(args.warmup + i), prec))
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = qd.launch_count() - launches0
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    if dist:
        tt = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
    # the whole run's per-sample values (all ranks), statistics on rank 0
    t_local = np.concatenate([r["t"] for r in results])
    idx_local = np.concatenate([np.arange(s) + offset(args.warmup + i) for i in range(args.steps)])
    t_all = parallel.gather_samples(t_local, idx_local)[1] if dist else t_local
    run_stats = qd.trace_stats(ctx, t_all, results[-1]["t0"]) if rank == 0 else None

    # per-kernel device time: separate steps with the library's CUDA-event
    # profiling on (graph replay is off while profiling, so these steps run
    # the same kernels launched one by one)
    qd.prof_enable(ctx, True)
    for k in qd.PROF_KINDS:
        qd.prof_read(ctx, k, reset=True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(args.prof_steps):
        _batch(qd, ctx, g, mg, d, offset(3000 + i), prec)
    p1.record(stream)
    torch.cuda.synchronize()
    qd.prof_enable(ctx, False)
    ms_prof = p0.elapsed_time(p1)
    prof = {k: qd.prof_read(ctx, k) for k in qd.PROF_KINDS}
    value = args.steps * s * world / (ms_total / 1e3)
    iters = [r["iterations"] for r in results]
    worst = max(r["max_true_rel_residual"] for r in results)

    # roofline of the dominant kernel (largest summed device time)
    top = max(prof, key=lambda k: prof[k]["ms"])
    pt = prof[top]
    if pt["ms"] <= 0.0:  # no profiled steps
        pt = {"ms": float("nan"), "flops": float("nan"), "bytes": float("nan"), "launches": 0}
    peaks = _peaks()
    if top in ("direct_f32", "coarse_f32", "smoother_f32"):
        # FP32 CUDA-core contractions
        fp32_peak = FP32_PEAK_TFLOPS
        achieved = pt["flops"] / (pt["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None, "kernel": top, "launches": pt["launches"],
                "ms_per_launch": pt["ms"] / max(pt["launches"], 1),
                "peak_source": "FP32 CUDA cores from unit counts and clock: 152 SMs x 128 lanes x 2 flops x 2.07 GHz "
                               "(an FMA-chain probe reached 70 TFLOP/s)"}
    elif top.endswith("f64"):
        achieved = pt["flops"] / (pt["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": top, "launches": pt["launches"], "ms_per_launch": pt["ms"] / max(pt["launches"], 1),
                "peak_source": "recipe nominal FP64 (1.25 TFLOP/s); FMA probe measured 1.20"}
    else:
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = pt["bytes"] / (pt["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": top, "launches": pt["launches"],
                "ms_per_launch": pt["ms"] / max(pt["launches"], 1),
                "peak_source": "measured (burst copy)" if "hbm_gbs" in peaks else "fallback"}
    roof["traffic"] = _traffic(args.workload, top)
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share_of_step": round(v["ms"] / ms_prof, 4),
                   "alg_gbs": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                   "alg_tflops": round(v["flops"] / (v["ms"] / 1e3) / 1e12, 2) if v["ms"] > 0 else None}
               for k, v in prof.items() if v["launches"]}
    kernels["_profiled_steps"] = {"steps": args.prof_steps, "ms_per_step": round(ms_prof / max(args.prof_steps, 1), 3)}

    # end to end through the public API: links from pinned host memory,
    # setup, one batch, results read back, per step
    e2e_steps = args.e2e_steps
    pinned = torch.from_numpy(synth.links_to_canonical(U).view(np.float64).reshape(-1)).pin_memory()
    h2d = pinned.numel() * 8
    torch.cuda.synchronize()
    t = time.perf_counter()
    phases = {"gauge": 0.0, "mg_setup": 0.0, "smoother_train": 0.0, "deflation": 0.0, "batch": 0.0}

    def lap(key, t_prev):
        torch.cuda.synchronize()
        now = time.perf_counter()
        phases[key] += now - t_prev
        return now

    for i in range(e2e_steps):
        tp = time.perf_counter()
        g2 = qd.Gauge.from_host_buffer(ctx, WL["dims"], pinned)
        tp = lap("gauge", tp)
        mg2 = qd.Multigrid(ctx, g2, WL["m0"], 0.0, _mg_params(qd))
        tp = lap("mg_setup", tp)
        if WL.get("learned"):
            qd.smoother_train(mg2, nsamples=4, solve_tol=1e-3, mr_steps=_learned_mr(WL), layers=WL.get("layers", 1))
            qd.smoother_enable(mg2, True, _learned_mr(WL))
        tp = lap("smoother_train", tp)
        d2 = qd.Deflation(ctx, g2, mg2, WL["m0"], 0.0,
                          qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, WL["k"], guard=WL["guard"], eig_tol=1e-6,
                                         solve_tol=1e-10, maxit=WL.get("eig_maxit", 60)))
        tp = lap("deflation", tp)
        _batch(qd, ctx, g2, mg2, d2, offset(1000 + i), prec)
        tp = lap("batch", tp)
        d2.close()
        mg2.close()
        g2.close()
    torch.cuda.synchronize()
    e2e_dt = (time.perf_counter() - t) / max(e2e_steps, 1) if e2e_steps else float("nan")
    if dist:
        tt = torch.tensor([e2e_dt], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_dt = float(tt.item())
    e2e = None if not e2e_steps else {"value": s * world / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": s * 16 + 6 * 8,
           "phases_s": {k: round(v / max(e2e_steps, 1), 4) for k, v in phases.items()},
           "scope": f"per step: link upload from pinned host memory, adaptive MG setup, learned-smoother "
                    f"training, Algorithm 2 deflation space, one {s}-sample batch, per-sample t_j and statistics "
                    f"read back"}

    # the plain FP64 path on the same workload (the other side of the
    # metric), on a block of fp64_samples samples per step
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        sf = WL.get("fp64_samples", s)
        if WL.get("learned"):
            qd.smoother_enable(mg, False, _learned_mr(WL))  # the plain FP64 form
        _batch(qd, ctx, g, mg, d, offset(2000), qd.QD_PREC_F64, nsamples=sf, plain=True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        fres = [_batch(qd, ctx, g, mg, d, offset(2001 + i), qd.QD_PREC_F64, nsamples=sf, plain=True)
                for i in range(args.fp64_steps)]
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        if dist:
            tt = torch.tensor([fms], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            fms = float(tt.item())
        if WL.get("learned"):
            qd.smoother_enable(mg, True, _learned_mr(WL))
        fp64 = {"value": args.fp64_steps * sf * world / (fms / 1e3), "unit": UNIT, "steps": args.fp64_steps,
                "samples_per_step": sf, "ms_per_step": fms / args.fp64_steps, "dtype": "f64",
                "smoother": "plain MR (4 fine, coarse as the workload)", "solver": "full-lattice FP64 GCR(16)",
                "outer_iterations": [r["iterations"] for r in fres],
                "max_true_rel_residual": max(r["max_true_rel_residual"] for r in fres),
                "mixed_over_fp64": value / (args.fp64_steps * sf * world / (fms / 1e3))}

    errors = None
    if rank == 0 and not args.no_errors:
        errors = errors_against_oracle(qd, ctx, U, g, mg, d)

    stencil = stencil_roofline(qd, ctx) if rank == 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        its = max(fp64["outer_iterations"]) if fp64 else FP64_ITERS_CONFIG3
        try:
            cpu = cpu_baseline(its)
        except Exception as exc:  # report, never hide the GPU line
            cpu = {"value": None, "unit": UNIT, "error": repr(exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 inner solves + f64 refinement" + (" (FP16 smoother weights)" if WL.get("learned") else ""))
            if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": WL["workload"], "precision": args.precision,
                       "parallelism": f"replicas x{world} (independent samples)",
                       "l2": "working set > L2 (fine fields 1.6 GB each)",
                       "setup_s": round(setup_s, 3), "outer_iterations": iters,
                       "max_true_rel_residual": worst,
                       "estimate": [run_stats["estimate"].real, run_stats["stderr"]],
                       "estimate_samples": int(run_stats["s"]),
                       "mg_overrides": WL.get("mg_kw", {}),
                       "learned_smoother": ({"layers": WL.get("layers", 1), "mr_steps": _learned_mr(WL), "judge": judge}
                                            if WL.get("learned") else None)},
            "errors": errors,
            "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "fp64_path": fp64, "stencil": stencil, "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    for o in (d, mg, g, ctx):
        o.close()
    if dist:
        dist.destroy_process_group()
    return 0


# Config 5: 24^3 x 48, eps 0.15 (seed 5), m0 -0.8, three-level MG (2^4 then
# 3^4 blocks, nv 12 on both: the coarsest level has 512 sites x 24 dofs and a
# dense inverse), Algorithm 2 k = 24, 256 samples per step solved in blocks
# of 64 right-hand sides, mixed precision to a true FP64 residual 1e-8, with
# the learned smoother against the plain minimal-residual smoother.
LEARNED = dict(
    workload="wilson-dirac 24^3x48 eps0.15 seed5 m0=-0.8, 3-level MG (2^4, 3^4; nv 12, 12; level-1 GCR 6 its), "
             "Algorithm 2 k=24, 256 Rademacher samples/step in 4 blocks of 64, learned smoother (S + 2 MR) vs "
             "plain MR(4), true FP64 rel. residual 1e-8",
    dims=(24, 24, 24, 48), eps=0.15, link_seed=5, m0=-0.8, blocks=[(2, 2, 2, 2), (3, 3, 3, 3)], nvs=[12, 12],
    mg_kw={"coarse_tol": 0.0, "coarse_maxit": 6}, k=24, guard=16, s=256, rhs_block=64, tol=1e-8,
    noise_seed=105, restart=16, maxit=500, inner_tol=1e-5,
)


def run_learned(args):
    """Config 5: samples/s and iterations with the learned smoother and with
    the plain smoother on the same samples."""
    import torch
    from paper_1909_12234_gb300 import qdtrace as qd
    from paper_1909_12234_gb300 import synth

    if int(os.environ.get("WORLD_SIZE", "1")) != 1 or args.gpus != 1:
        raise SystemExit("the learned-smoother workload runs on one GPU")
    L = dict(LEARNED)
    if args.small:
        # the learned-vs-plain comparison on the 16^3 x 32 lattice of the
        # mixed-precision workload (eps 0.2, seed 3, 2^4 then 2^4 blocks, nv
        # 12 then 16), 128 samples in 2 blocks of 64
        L.update(dims=(16, 16, 16, 32), eps=0.2, link_seed=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvs=[12, 16],
                 s=128, rhs_block=64, noise_seed=103,
                 workload="wilson-dirac 16^3x32 eps0.2 seed3 m0=-0.8, 3-level MG (2^4, 2^4; nv 12, 16; level-1 GCR "
                          "6 its), Algorithm 2 k=24, 128 Rademacher samples/step in 2 blocks of 64, learned smoother "
                          "(S + 2 MR) vs plain MR(4), true FP64 rel. residual 1e-8")
    T0 = time.perf_counter()

    def log(msg):
        sys.stderr.write(f"[{time.perf_counter() - T0:8.1f}s] {msg}\n")
        sys.stderr.flush()
    qd.load()
    ctx = qd.Context(0)
    U = synth.random_su3_links(L["dims"], L["eps"], L["link_seed"])
    torch.cuda.synchronize()
    t = time.perf_counter()
    g = qd.Gauge(ctx, L["dims"], U)
    del U
    mg = qd.Multigrid(ctx, g, L["m0"], 0.0, qd.mg_params(2, L["blocks"], L["nvs"], **L["mg_kw"]))
    log("multigrid built")
    d = qd.Deflation(ctx, g, mg, L["m0"], 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, L["k"], guard=L["guard"],
                                                               eig_tol=1e-6, solve_tol=1e-10, maxit=60))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    log(f"setup done ({setup_s:.1f} s)")
    t = time.perf_counter()
    info = qd.smoother_train(mg, nsamples=8, solve_tol=1e-6, mr_steps=2)
    train_s = time.perf_counter() - t
    log(f"smoother trained ({train_s:.1f} s): {info}")
    s, sb = L["s"], L["rhs_block"]

    def step(i, learned):
        qd.smoother_enable(mg, learned, 2)
        ts, its, worst = [], [], 0.0
        for b0 in range(0, s, sb):
            r = qd.hutchinson_trace(ctx, g, mg, d, L["m0"], 0.0, L["noise_seed"], 100000 * i + b0, min(sb, s - b0),
                                    L["tol"], maxit=L["maxit"], restart=L["restart"], precision=qd.QD_PREC_MIXED,
                                    inner_tol=L["inner_tol"], max_refine=10)
            ts.append(r["t"])
            its.append(r["iterations"])
            worst = max(worst, r["max_true_rel_residual"])
            log(f"step {i} learned={learned} block {b0}: {r['iterations']} its, res {r['max_true_rel_residual']:.2e}")
        t0 = r["t0"]
        st = qd.trace_stats(ctx, np.concatenate(ts), t0)
        return st, its, worst

    def timed(learned, nsteps, first):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        out = [step(first + i, learned) for i in range(nsteps)]
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    for i in range(args.warmup):
        step(i, True)
        step(i, False)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qd.launch_count()
    ms, res = timed(True, args.steps, args.warmup)
    launches = qd.launch_count() - l0
    clk = clocks.stop()
    ms_plain, res_plain = timed(False, args.steps, args.warmup)

    qd.smoother_enable(mg, True, 2)
    qd.prof_enable(ctx, True)
    for k in qd.PROF_KINDS:
        qd.prof_read(ctx, k, reset=True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(ctx.stream)
    qd.hutchinson_trace(ctx, g, mg, d, L["m0"], 0.0, L["noise_seed"], 9000000, sb, L["tol"], maxit=L["maxit"],
                        restart=L["restart"], precision=qd.QD_PREC_MIXED, inner_tol=L["inner_tol"], max_refine=10)
    p1.record(ctx.stream)
    torch.cuda.synchronize()
    qd.prof_enable(ctx, False)
    ms_prof = p0.elapsed_time(p1)
    prof = {k: qd.prof_read(ctx, k) for k in qd.PROF_KINDS}
    top = max(prof, key=lambda k: prof[k]["ms"])
    pt = prof[top]
    hbm = _peaks().get("hbm_gbs", 6800.0)
    if top.endswith("f64") or top in ("direct_f32", "coarse_f32"):
        peak = FP64_PEAK_TFLOPS if top.endswith("f64") else FP32_PEAK_TFLOPS
        ach = pt["flops"] / (pt["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak}
    else:
        ach = pt["bytes"] / (pt["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm}
    roof.update({"traffic": None, "kernel": top, "launches": pt["launches"],
                 "ms_per_launch": pt["ms"] / max(pt["launches"], 1)})
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share_of_step": round(v["ms"] / ms_prof, 4)}
               for k, v in prof.items() if v["launches"]}

    def summary(ms_, rr):
        st, its, worst = rr[-1]
        return {"value": args.steps * s / (ms_ / 1e3), "ms_per_step": ms_ / args.steps, "outer_iterations": its,
                "max_true_rel_residual": max(r[2] for r in rr), "estimate": [st["estimate"].real, st["stderr"]],
                "var": st["var"], "var_jackknife_err": st["var_jackknife_err"]}

    learned, plain = summary(ms, res), summary(ms_plain, res_plain)
    line = {
        "metric": METRIC, "value": learned["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": learned["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 inner solves (FP16 smoother weights) + f64 refinement", "data": "synthetic",
        "config": {"workload": L["workload"], "precision": "mixed", "parallelism": "replicas x1",
                   "l2": "fields 2-8 GB per block exceed L2", "setup_s": round(setup_s, 3),
                   "smoother_train_s": round(train_s, 3), "smoother_judge": info,
                   "learned": learned, "plain": plain},
        "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": None, "gpu_launches": launches,
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    for o in (d, mg, g, ctx):
        o.close()
    return 0


def run_batch(args):
    """Config 4: the uneven batch, concurrent (one qd_hutchinson_batch call
    per step) against the same problems solved one after another."""
    import torch
    from paper_1909_12234_gb300 import qdtrace as qd
    from paper_1909_12234_gb300 import synth

    if int(os.environ.get("WORLD_SIZE", "1")) != 1 or args.gpus != 1:
        raise SystemExit("the batch workload runs on one GPU")
    qd.load()
    ctx = qd.Context(0)
    B = BATCH

    def setup(pinned=None):
        probs = []
        for i, (dims, seed, m0, s) in enumerate(B["problems"]):
            if pinned is None:
                g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, B["eps"], seed))
            else:
                g = qd.Gauge.from_host_buffer(ctx, dims, pinned[i])
            mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, B["blocks"], B["nvs"], **B["mg_kw"]))
            d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, B["k"], guard=B["guard"],
                                                                 eig_tol=1e-6, solve_tol=1e-10, maxit=60))
            probs.append(dict(gauge=g, mg=mg, defl=d, m0=m0, tau=0.0, seed=100 + seed, sample_offset=0, nsamples=s,
                              tol=B["tol"], maxit=B["maxit"], restart=B["restart"], precision=qd.QD_PREC_MIXED,
                              inner_tol=B["inner_tol"], max_refine=10))
        return probs

    def close(probs):
        for p in probs:
            for key in ("defl", "mg", "gauge"):
                p[key].close()

    torch.cuda.synchronize()
    t = time.perf_counter()
    probs = setup()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t
    total = sum(p["nsamples"] for p in probs)

    def step(i, concurrent):
        for p in probs:
            p["sample_offset"] = 1000 * i
        if concurrent:
            return qd.hutchinson_batch(ctx, probs, nstreams=len(probs))
        keys = ("gauge", "mg", "defl", "m0", "tau", "seed", "sample_offset", "nsamples", "tol")
        return [qd.hutchinson_trace(ctx, p["gauge"], p["mg"], p["defl"], p["m0"], 0.0, p["seed"], p["sample_offset"],
                                    p["nsamples"], p["tol"], **{k: v for k, v in p.items() if k not in keys})
                for p in probs]

    def timed(concurrent, nsteps, first):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        res = [step(first + i, concurrent) for i in range(nsteps)]
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    for i in range(args.warmup):
        step(i, True)
        step(i, False)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = qd.launch_count()
    ms, res = timed(True, args.steps, args.warmup)
    launches = qd.launch_count() - l0
    clk = clocks.stop()
    ms_seq, res_seq = timed(False, args.steps, args.warmup)
    # the concurrent and the sequential runs solve the same samples: identical
    same = all(np.array_equal(a["t"], b["t"]) for ra, rb in zip(res, res_seq) for a, b in zip(ra, rb))
    worst = max(r["max_true_rel_residual"] for rr in res for r in rr)

    # per-kernel device time of the sequential form (profiling is per context)
    qd.prof_enable(ctx, True)
    for k in qd.PROF_KINDS:
        qd.prof_read(ctx, k, reset=True)
    ms_prof, _ = timed(False, 1, 5000)
    qd.prof_enable(ctx, False)
    prof = {k: qd.prof_read(ctx, k) for k in qd.PROF_KINDS}
    top = max(prof, key=lambda k: prof[k]["ms"])
    pt = prof[top]
    hbm = _peaks().get("hbm_gbs", 6800.0)
    if top.endswith("f64") or top in ("direct_f32", "coarse_f32"):
        peak = FP64_PEAK_TFLOPS if top.endswith("f64") else FP32_PEAK_TFLOPS
        ach = pt["flops"] / (pt["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak}
    else:
        ach = pt["bytes"] / (pt["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm}
    roof.update({"traffic": None, "kernel": top, "launches": pt["launches"],
                 "ms_per_launch": pt["ms"] / max(pt["launches"], 1)})
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share_of_step": round(v["ms"] / ms_prof, 4)}
               for k, v in prof.items() if v["launches"]}
    # what a single persistent launch over the batch could gain: its step
    # cannot take less than the device time of the same kernels (summed
    # CUDA-event time of every instrumented kernel of one sequential step);
    # the rest of a step is launch gaps, host synchronisation and the small
    # uninstrumented kernels
    busy = sum(v["ms"] for v in prof.values())
    persistent_bound = {"device_busy_ms": round(busy, 3), "sequential_ms": round(ms_seq / args.steps, 3),
                        "concurrent_ms": round(ms / args.steps, 3),
                        "sequential_idle_fraction": round(1.0 - busy / (ms_seq / args.steps), 4),
                        "concurrent_over_busy": round((ms / args.steps) / busy, 4)}

    # end to end: links from pinned host memory, setup of all three, one batch
    pinned = []
    for dims, seed, m0, s in B["problems"]:
        U = synth.random_su3_links(dims, B["eps"], seed)
        canon = np.ascontiguousarray(np.transpose(U, (1, 0, 2, 3)))
        pinned.append(torch.from_numpy(canon.view(np.float64).reshape(-1)).pin_memory())
    e2e = None
    if args.e2e_steps:
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(args.e2e_steps):
            pr2 = setup(pinned)
            for p in pr2:
                p["sample_offset"] = 7000 + 1000 * i
            qd.hutchinson_batch(ctx, pr2, nstreams=len(pr2))
            close(pr2)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t) / args.e2e_steps
        e2e = {"value": total / dt, "unit": UNIT, "h2d_bytes_per_step": sum(p.numel() * 8 for p in pinned),
               "d2h_bytes_per_step": total * 16 + 6 * 8 * len(probs),
               "scope": "per step: link upload of the three lattices, their setups, one concurrent batch"}
    tune = qd.autotune_report()
    line = {
        "metric": METRIC, "value": args.steps * total / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 inner solves + f64 refinement", "data": "synthetic",
        "config": {"workload": B["workload"], "precision": "mixed", "parallelism": "one batch, 3 worker streams",
                   "l2": "16^4 fields (0.8-1.6 GB) exceed L2", "setup_s": round(setup_s, 3),
                   "max_true_rel_residual": worst, "bit_identical_to_sequential": same,
                   "sequential": {"value": args.steps * total / (ms_seq / 1e3), "ms_per_step": ms_seq / args.steps},
                   "persistent_launch_bound": persistent_bound,
                   "estimates": [[r["estimate"].real, r["stderr"]] for r in res[-1]],
                   "autotune": {k: v[0] for k, v in tune.items()}},
        "roofline": roof, "kernels": kernels, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    close(probs)
    ctx.close()
    return 0


# Smoother depth at equal cost (scope row f3): on the 16^3 x 32 workload,
# the plain MR smoother, the one-layer learned smoother with 1 or 2 MR steps
# after it, and stacks of 2 and 3 layers (S = S_L ... S_1, each layer the
# one-hop form, trained layer by layer) with 0 or 1 MR steps.  Cost is what
# samples/s measures: every variant runs the same 128-sample batches.
SMOOTHER_DEPTH = [(0, 0), (1, 0), (1, 1), (1, 2), (2, 0), (2, 1), (3, 0)]  # (layers, MR steps); layers 0 = plain MR


def run_smoother_depth(args):
    import torch
    from paper_1909_12234_gb300 import qdtrace as qd
    from paper_1909_12234_gb300 import synth

    if int(os.environ.get("WORLD_SIZE", "1")) != 1 or args.gpus != 1:
        raise SystemExit("the smoother-depth comparison runs on one GPU")
    WL.clear()
    WL.update(CONFIG3)
    qd.load()
    ctx = qd.Context(0)
    U = synth.random_su3_links(WL["dims"], WL["eps"], WL["link_seed"])
    wl = dict(WL, learned=0)
    g, mg, d, _ = _setup(qd, ctx, U, wl)
    s = WL["s"]
    rows = []
    for layers, mr in SMOOTHER_DEPTH:
        info = None
        if layers:
            t = time.perf_counter()
            info = qd.smoother_train(mg, nsamples=4, solve_tol=1e-3, mr_steps=mr, layers=layers)
            train_s = time.perf_counter() - t
            qd.smoother_enable(mg, True, mr)  # measured whatever the held-out judge said
        else:
            train_s = 0.0
            if qd.smoother_layers(mg):
                qd.smoother_enable(mg, False, 0)
        for i in range(args.warmup):
            _batch(qd, ctx, g, mg, d, 5000 * i, qd.QD_PREC_MIXED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        res = [_batch(qd, ctx, g, mg, d, 100000 + 1000 * i, qd.QD_PREC_MIXED) for i in range(args.steps)]
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        row = {"layers": layers, "mr_steps": mr if layers else "plain MR(%d)" % _mg_params(qd).smoother_steps,
               "samples_per_s": s / (ms / 1e3), "ms_per_step": ms,
               "outer_iterations": [r["iterations"] for r in res],
               "max_true_rel_residual": max(r["max_true_rel_residual"] for r in res), "train_s": train_s}
        if info:
            row.update(held_out_err_learned=info["err_learned"], held_out_err_plain=info["err_plain"],
                       judge_enables=info["enabled"])
        rows.append(row)
        sys.stderr.write(json.dumps(row) + "\n")
    print(json.dumps({"workload": "smoother depth at equal cost: " + WL["workload"], "unit": UNIT, "rows": rows}))
    for o in (d, mg, g, ctx):
        o.close()
    return 0


# Algorithm 1 against Algorithm 2 on the 8^4 lattice (Sec. 2.2, Sec. 4.1):
# the a-posteriori variance of the deflated estimator as a function of the
# rank, from one set of undeflated solves, with jackknife errors, and the
# sines of the angles between the Algorithm 1 vectors and range(W) (Fig. 3).
DEFL_CMP = dict(
    workload="deflation comparison: wilson-dirac 8^4 eps0.3 seed2 m0=-0.8, 2-level MG (2^4, nv 12); Algorithm 1 "
             "(24 smallest eigenvectors of A gamma5, GPU eigensolver with MG solves) vs Algorithm 2 (24 coarse "
             "eigenvectors); a-posteriori variance vs rank from 64 undeflated samples solved to 1e-8",
    dims=(8, 8, 8, 8), eps=0.3, link_seed=2, m0=-0.8, blocks=[(2, 2, 2, 2)], nvs=[12], k=24, guard=16, s=64,
    tol=1e-8, noise_seed=102, ranks=[0, 2, 4, 8, 12, 16, 20, 24],
)


def run_deflation_compare(args):
    import torch
    from paper_1909_12234_gb300 import qdtrace as qd
    from paper_1909_12234_gb300 import synth
    C = DEFL_CMP
    qd.load()
    ctx = qd.Context(0)
    U = synth.random_su3_links(C["dims"], C["eps"], C["link_seed"])
    g = qd.Gauge(ctx, C["dims"], U)
    mg = qd.Multigrid(ctx, g, C["m0"], 0.0, qd.mg_params(1, C["blocks"], C["nvs"]))
    torch.cuda.synchronize()
    t = time.perf_counter()
    d2 = qd.Deflation(ctx, g, mg, C["m0"], 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, C["k"], guard=C["guard"],
                                                               eig_tol=1e-6, solve_tol=1e-10, maxit=60))
    torch.cuda.synchronize()
    t_alg2 = time.perf_counter() - t
    t = time.perf_counter()
    d1 = qd.Deflation(ctx, g, mg, C["m0"], 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, C["k"], guard=C["guard"],
                                                               eig_tol=1e-6, solve_tol=1e-10, maxit=60))
    torch.cuda.synchronize()
    t_alg1 = time.perf_counter() - t
    s, k = C["s"], C["k"]
    res0 = qd.hutchinson_trace(ctx, g, mg, None, C["m0"], 0.0, seed=C["noise_seed"], sample_offset=0, nsamples=s,
                               tol=C["tol"], maxit=500, precision=qd.QD_PREC_MIXED, inner_tol=1e-5, max_refine=10)
    z = torch.empty((g.V, 12, s), dtype=torch.complex128, device="cuda:0")
    qd.rademacher(ctx, g, C["noise_seed"], 0, s, z)
    zhv1, uhz1 = d1.coeffs(s, z)
    zhv2, uhkz2 = d2.coeffs(s, z)
    G = d2.gram()
    rows = []
    for r in C["ranks"]:
        row = {"rank": r}
        for name, d in (("alg1", d1), ("alg2", d2)):
            if r == 0:
                tr, t0 = res0["t"], 0j
            else:
                t0 = d.set_rank(r)
                if name == "alg1":
                    corr = np.einsum("ji,ij->j", zhv1[:, :r], uhz1[:r])
                else:
                    corr = np.einsum("ji,ij->j", zhv2[:, :r], np.linalg.solve(G[:r, :r], uhkz2[:r]))
                tr = res0["t"] - corr
            st = qd.trace_stats(ctx, tr, t0)
            row[name] = {"estimate": st["estimate"].real, "stderr": st["stderr"], "var": st["var"],
                         "var_jackknife_err": st["var_jackknife_err"], "t0": t0.real}
        rows.append(row)
    # check the a-posteriori values against real deflated runs at full rank
    check = {}
    for name, d in (("alg1", d1), ("alg2", d2)):
        d.set_rank(k)
        rr = qd.hutchinson_trace(ctx, g, mg, d, C["m0"], 0.0, seed=C["noise_seed"], sample_offset=0, nsamples=s,
                                 tol=C["tol"], maxit=500, precision=qd.QD_PREC_MIXED, inner_tol=1e-5, max_refine=10)
        if name == "alg1":
            post = res0["t"] - np.einsum("ji,ij->j", zhv1, uhz1)
        else:
            post = res0["t"] - np.einsum("ji,ij->j", zhv2, np.linalg.solve(G, uhkz2))
        check[name] = {"max_abs_diff_posteriori_vs_run": float(np.abs(post - rr["t"]).max()),
                       "max_abs_t": float(np.abs(rr["t"]).max()), "var_run": rr["var"]}
    # Fig. 3 (right): sin of the angle between each Algorithm 1 vector and range(W)
    V = torch.empty((g.V, 12, k), dtype=torch.complex128, device="cuda:0")
    d1.basis(V)
    sines = qd.mg_subspace_sines(mg, 1, V)
    mu1, _, its1 = d1.info()
    mu2, _, its2 = d2.info()
    tau, nrs = d1.shift_info()
    line = {"analysis": "deflation rank sweep (Algorithm 1 vs Algorithm 2)", "workload": C["workload"],
            "build_s": {"alg1": round(t_alg1, 3), "alg2": round(t_alg2, 3)},
            "eigensolver": {"alg1_iterations": its1, "alg2_iterations": its2, "alg1_shift": tau,
                            "alg1_restarts": nrs, "alg1_mu": [round(float(x), 6) for x in mu1],
                            "alg2_mu": [round(float(x), 6) for x in mu2]},
            "undeflated": {"estimate": res0["estimate"].real, "var": res0["var"],
                           "var_jackknife_err": res0["var_jackknife_err"]},
            "rank_sweep": rows, "check_full_rank": check,
            "sin_angle_alg1_vectors_to_W": [round(float(x), 5) for x in sines]}
    print(json.dumps(line))
    for o in (d1, d2, mg, g, ctx):
        o.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-errors", action="store_true", help="skip the errors-against-the-oracle leg")
    ap.add_argument("--prof-steps", type=int, default=2)
    ap.add_argument("--workload", default="config3",
                    choices=sorted(WORKLOADS) + ["config4", "config5", "deflation", "smoother-depth"])
    ap.add_argument("--stencil-only", action="store_true",
                    help="only the Wilson stencil alone on 16^3 x 32 (a profiling target)")
    ap.add_argument("--small", action="store_true",
                    help="config5: the learned-vs-plain comparison on the 16^3 x 32 lattice")
    ap.add_argument("--smoother-steps", type=int, default=0, help="> 0: MR post-smoothing steps (default 4)")
    ap.add_argument("--coarse-smoother-steps", type=int, default=-1,
                    help=">= 0: MR post-smoothing steps on the coarse levels (default: as the fine level)")
    ap.add_argument("--learned", type=int, default=-1,
                    help=">= 1: train the learned smoother and use it with this many MR steps after it; "
                         "0: plain smoother; default: the workload's setting")
    ap.add_argument("--fixed-coarse", type=int, default=0,
                    help="> 0: level-1 GCR of a three-level hierarchy runs exactly this many iterations")
    ap.add_argument("--restart", type=int, default=0, help="> 0: restart length of the fine-level GCR")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="> 0: tolerance of the FP32 inner solves")
    ap.add_argument("--schur", type=int, default=-1,
                    help="1: even-odd fine solves (GCR on the odd-site Schur complement); 0: full lattice; "
                         "default: the workload's setting")
    ap.add_argument("--kernel", default="",
                    help="comma-separated hot kernels timed alone on the 16^3 x 32 shapes (a profiling target): "
                         "coarse_tc, restrict_tc, prolong_l1, prolong_l2, wilson_f32, wilson_resid_f32, schur_f32, "
                         "smoother_f32; 'all' for every one")
    ap.add_argument("--reps", type=int, default=20, help="launches timed per kernel with --kernel")
    ap.add_argument("--no-tune", action="store_true",
                    help="launch shapes fixed at their defaults (nothing timed by the autotuner)")
    ap.add_argument("--candidate", type=int, default=-1,
                    help=">= 0: with --kernel, launch shape k of every tunable kernel where it applies")
    args = ap.parse_args()
    if args.no_tune:
        from paper_1909_12234_gb300 import qdtrace as qd
        qd.load()
        qd.autotune_set(0)
    if args.kernel:
        from paper_1909_12234_gb300 import qdtrace as qd
        qd.load()
        ctx = qd.Context(0)
        names = (["coarse_tc", "restrict_tc", "prolong_l1", "prolong_l2", "wilson_f32", "wilson_resid_f32",
                  "schur_f32", "smoother_f32"]
                 if args.kernel == "all"
                 else args.kernel.split(","))
        if args.candidate >= 0:
            qd.autotune_force(args.candidate)
        print(json.dumps({"kernels_alone": kernel_only(qd, ctx, names, args.reps)}))
        ctx.close()
        return 0
    if args.stencil_only:
        from paper_1909_12234_gb300 import qdtrace as qd
        qd.load()
        ctx = qd.Context(0)
        print(json.dumps({"stencil": stencil_roofline(qd, ctx)}))
        ctx.close()
        return 0
    if args.workload in ("config4", "config5", "deflation", "smoother-depth"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-lattice workload"}))
            return 0
        if args.workload == "deflation":
            return run_deflation_compare(args)
        if args.workload == "smoother-depth":
            return run_smoother_depth(args)
        return run_batch(args) if args.workload == "config4" else run_learned(args)
    WL.clear()
    WL.update(WORKLOADS[args.workload])
    if args.fixed_coarse > 0:
        WL["mg_kw"] = dict(WL.get("mg_kw", {}), coarse_tol=0.0, coarse_maxit=args.fixed_coarse)
    if args.smoother_steps > 0:
        WL["mg_kw"] = dict(WL.get("mg_kw", {}), smoother_steps=args.smoother_steps)
    if args.coarse_smoother_steps >= 0:
        WL["mg_kw"] = dict(WL.get("mg_kw", {}), coarse_smoother_steps=args.coarse_smoother_steps)
    if args.learned >= 0:
        WL["learned"] = args.learned
        WL["learned_mr"] = args.learned
        WL["layers"] = 1
    if args.restart > 0:
        WL["restart"] = args.restart
    if args.inner_tol > 0:
        WL["inner_tol"] = args.inner_tol
    if args.schur >= 0:
        WL["schur"] = args.schur
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
