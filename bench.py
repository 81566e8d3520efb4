#!/usr/bin/env python3
"""Benchmark of the density-fitted PNOF7 energy+gradient evaluation on one GB300.

Metric: energy+gradient evaluations per second (one evaluation = the orbital transformation of
the RI tensor, J, K, the PNOF energy, the Lagrangian, the orbital and the occupation gradients at
fixed (C, gamma)), against the plain FP64 GPU path on the same inputs, at |dE| <= 1e-6 Ha.

Default line: the largest single-GPU system, the H1000 chain (spacing 1.8 bohr, one contracted s
function (STO-3G-like, zeta 1.24) and 3 aux s (alpha = 0.1 * 3^k) per H: nbf = 1000, naux = 3000,
nact = 1000, PNOF7, 500 pairs, N_g = 1), on the split-precision tensor-core path (5 BF16 digits
per operand element). C = S^{-1/2} Q for a seeded random orthogonal Q, gamma ~ U(0.1, 1.2). The K
timed steps are one region bracketed by CUDA events on the library's stream; every step reads
the 30 GB of B's digit planes from HBM (inputs larger than L2). The same line carries the other
workloads as extra keys under `configs`: the H200 lattice, the H50 chain and the 256-frame batch.

Under torchrun (N > 1) every rank evaluates its own independent instance (orbitals seeded by the
rank): the path has no exchange step, so the ranks are replicas and `value` sums their work.

`--impl reference` times the CPU FP64 oracle (test infrastructure) on a bounded sample of the same
workload: each step evaluates the oracle over a slice of the aux functions, scaled to whole
evaluations.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NOF energy+gradient evals/sec vs FP64 plain GPU path at |ΔE|≤1e-6 Ha"
ACC_GATE = 1e-6
L2_BYTES = 129 * 1000 * 1000  # GB300 L2

WORKLOADS = {
    "h1000": "H1000 chain, spacing 1.8 bohr, 1 contracted s/H (STO-3G-like, zeta 1.24) + 3 aux s/H (0.1*3^k): "
             "nbf=1000, naux=3000, nact=1000, PNOF7, 500 pairs, N_g=1",
    "h200": "H200 10x20 square lattice, spacing 2.0 bohr, 3 s/H (0.2*4^k) + 10 aux s/H (0.1*3^k): "
            "nbf=600, naux=2000, nact=200, PNOF7, 100 pairs, N_g=1",
    "h50": "H50 chain, spacing 1.8+U(-0.1,0.1) bohr, 3 s/H (0.2*4^k) + 10 aux s/H (0.1*3^k): "
           "nbf=150, naux=500, nact=50, PNOF7, 25 pairs, N_g=1",
}
HEADLINE = "h1000"
WORKLOAD = WORKLOADS["h50"]  # the nuclear-gradient workload's system


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=["split", "fp64"], default="split")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work (H50 sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="the headline workload only")
    ap.add_argument("--workload", choices=["default", "h1000", "h200", "h50", "batch", "nlop", "gradient",
                                           "dynamics", "optimize"], default="default",
                    help="default: H1000 headline line with H200, H50 and the batch as extra keys; h1000/h200/"
                         "h50: that system alone as the line; batch: many uneven H-chain frames evaluated "
                         "concurrently as one CUDA-graph launch; nlop: the finite-field polarizability and "
                         "hyperpolarizabilities of H2 (21 field instances stepped together); gradient: the "
                         "nuclear gradient of the H50 chain on the FP64 path; dynamics: velocity-Verlet steps "
                         "of H2 on converged states; optimize: the converged ON/NO loop of --opt-system from "
                         "its core guess")
    ap.add_argument("--opt-system", choices=["h1000", "h200", "h50"], default="h200")
    ap.add_argument("--opt-gtol", type=float, default=1e-5)
    ap.add_argument("--opt-etol", type=float, default=1e-8)
    ap.add_argument("--opt-maxit", type=int, default=2000)
    ap.add_argument("--opt-eps-rel", type=float, default=0.0)
    ap.add_argument("--opt-lr-grow", type=float, default=1.0)
    ap.add_argument("--opt-maxloop", type=int, default=10)
    ap.add_argument("--opt-orbopt", type=int, default=2, choices=[0, 1, 2])
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-max", type=int, default=64, help="largest chain length in the batch")
    ap.add_argument("--no-graph", action="store_true",
                    help="time plain API calls instead of CUDA-graph replays of one evaluation")
    ap.add_argument("--profile-evals", type=int, default=0,
                    help="profiling mode: build the --workload system (default: h1000), warm up, run this many "
                         "evaluations inside the NVTX range 'evals' (for ncu --nvtx --nvtx-include evals/) and exit")
    return ap.parse_args()


def workload(seed=2, name="h50"):
    """Geometry and basis pair of a named system (seed: the H50 chain's jitter)."""
    from paper_2512_13550_gb300 import inputs
    if name == "h1000":
        orb, aux = inputs.basis_h1000()
        return inputs.chain(1000, 1.8), orb, aux
    orb, aux = inputs.basis_3s_10aux()
    if name == "h200":
        return inputs.lattice(10, 20, 2.0), orb, aux
    return inputs.jittered_chain(50, seed), orb, aux


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 rate of the plain path: 2 FP64 FMA per clock per SM (the rate an FMA-throughput probe
# measured on GB300: 1.19 TFLOP/s), x 152 SMs x 2.07 GHz x 2 FLOP = 1.26 TFLOP/s.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12

# The three contractions of an evaluation (nof_profile selectors) with their algorithmic work
# per launch in the units of the system (X aux functions, n basis functions, a active orbitals):
# flops of the contraction and its minimum bytes (the operand streamed from HBM once at 4 bytes
# per element, the FP32 storage the work estimate assumes, and the output written once at 4
# bytes). The split path reads more than that (2 nd bytes per digit element, double-float
# outputs): those extra bytes are the price of its accuracy and count against it.
CONTRACTIONS = {
    1: ("half transform T = B C", lambda X, n, a: (2.0 * X * n * n * a, 4.0 * X * n * n + 4.0 * X * n * a)),
    2: ("full transform b = C^T T", lambda X, n, a: (2.0 * X * n * a * a, 4.0 * X * n * a + 4.0 * X * a * a)),
    3: ("Lagrangian contraction sum_P T W", lambda X, n, a: (2.0 * X * n * a * a, 4.0 * X * n * a + 4.0 * X * a * a)),
}


def eval_work(X, n, a):
    """Algorithmic work of one evaluation: flops of the three contractions (plus the J/K and D
    terms) and the minimum bytes (B once at 4 bytes per element, T and b/W' written and read once
    at 4 bytes)."""
    flops = 2.0 * X * n * n * a + 4.0 * X * n * a * a + 4.0 * X * a * a + 2.0 * X * a * a + 4.0 * n * n * a
    nbytes = 4.0 * X * n * n + 2 * 4.0 * X * n * a + 2 * 4.0 * X * a * a
    return flops, nbytes


def roofline(prec, sizes, which, ms_per_launch, name, nd=5, traffic=None):
    """Roofline of one contraction: achieved = its algorithmic flops (or bytes) per launch over
    the CUDA-event duration of a launch. The split path's arithmetic type is an exact BF16
    digit-plane product: nd (nd + 1) / 2 BF16 products per multiply-add, so its own peak is the
    measured BF16 peak divided by that count; the plain path's is the FP64 rate. The bound is the
    larger of flops / peak and bytes / HBM peak."""
    X, n, a = sizes["naux"], sizes["nbf"], sizes["nact"]
    peaks, src = _peaks()
    label, work = CONTRACTIONS[which]
    flops, nbytes = work(X, n, a)
    sec = ms_per_launch / 1e3
    base = {"kernel": name, "contraction": label, "algorithmic_flops": flops, "algorithmic_bytes": nbytes,
            "ms_per_launch": ms_per_launch, "traffic": traffic}
    if prec == 0:
        peak_t = FP64_PEAK_TFLOPS
        dtype_note = "FP64 SIMT: 2 FMA/clk/SM x 152 SMs x 2.07 GHz (probe-measured rate)"
        prods = 1
    else:
        prods = nd * (nd + 1) // 2
        bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        peak_t = bf16 / prods
        dtype_note = (f"{src} BF16 dense peak, sustained ({bf16:.1f} TFLOP/s; the kernel runs inside "
                      f"back-to-back evaluations) / {prods} BF16 digit products per multiply-add ({nd} digits)")
        base["digits"] = nd
        base["bf16_products_per_mac"] = prods
        # what the digit scheme actually moves: 2 nd bytes per element of the streamed operand
        base["digit_operand_bytes"] = nbytes * nd / 2.0
    t_tc = flops / (peak_t * 1e12)
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    if t_tc >= t_hbm:
        achieved = flops / sec / 1e12
        base.update({"bound": "tensor" if prec else "alu", "achieved": achieved, "peak": peak_t,
                     "unit": "TFLOP/s", "frac": achieved / peak_t, "peak_source": dtype_note})
        if prec:
            base["frac_of_bf16_peak_algorithmic"] = achieved / (peak_t * prods)  # no credit for the products
    else:
        achieved = nbytes / sec / 1e9
        base.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"],
                     "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"})
    return base


def eval_roofline(prec, sizes, ms_per_eval, nd=5):
    """Whole-evaluation fraction: t_roofline / t_measured with t_roofline the larger of the
    algorithmic flops over the arithmetic peak (BF16 / digit products, or FP64) and the algorithmic
    bytes over the HBM peak."""
    X, n, a = sizes["naux"], sizes["nbf"], sizes["nact"]
    peaks, src = _peaks()
    flops, nbytes = eval_work(X, n, a)
    if prec == 0:
        peak_t = FP64_PEAK_TFLOPS
    else:
        peak_t = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) / (nd * (nd + 1) // 2)
    t_tc = flops / (peak_t * 1e12)
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    t_roof = max(t_tc, t_hbm)
    return {"bound": ("tensor" if prec else "alu") if t_tc >= t_hbm else "hbm", "algorithmic_flops": flops,
            "algorithmic_bytes": nbytes, "t_roofline_ms": t_roof * 1e3, "ms_per_eval": ms_per_eval,
            "frac": t_roof * 1e3 / ms_per_eval, "arith_peak_tflops": peak_t, "hbm_peak_gbs": peaks["hbm_gbs"],
            "peak_source": src}


# ---------------------------------------------------------------------------------------
# the CPU FP64 oracle, timed on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------------------
def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class OracleSample:
    """The oracle's energy+gradient evaluation of a named system restricted to its first `xs` aux
    functions. Every term the evaluation spends its time on (the transforms, J, K, the Lagrangian
    contraction) is a sum over the aux index, so a slice of xs of the X aux functions is xs / X of
    one evaluation. The slice's three-centre integrals stand in for the fitted tensor's rows (the
    cost does not depend on the values), which keeps the sample's set-up to seconds."""

    def __init__(self, name: str, xs: int):
        from oracle import integrals, pnof, reference
        from paper_2512_13550_gb300 import inputs
        xyz, orb, aux = workload(2, name)
        if name == "h1000":  # the overlap stands in for h (1000 nuclei make V slow in numpy; the cost
            S = integrals.overlap(orb, xyz)  # of an evaluation does not depend on h's values)
            T, V = S, np.zeros_like(S)
        else:
            S, T, V = integrals.one_electron(orb, xyz)
        self.X = integrals.naux(aux, xyz)
        self.xs = min(xs, self.X)
        self.B = integrals.three_center(orb, aux, xyz, slice(0, self.xs))
        n = S.shape[0]
        self.pm = pnof.PairMap(xyz.shape[0], 1, n)
        self.C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 0))
        self.gam = inputs.random_gamma(self.pm.ngamma, 1)
        self.H = T + V
        self.vnn = integrals.nuclear_repulsion(xyz)

    def run(self):
        from oracle import pnof
        return pnof.energy_and_gradients(self.B, self.H, self.C, self.gam, self.pm, self.vnn)

    @property
    def fraction(self):
        return self.xs / self.X


def oracle_rate(name: str, xs: int, reps: int = 1):
    """(evaluations, seconds): `reps` sample evaluations of xs aux functions, as evaluations."""
    smp = OracleSample(name, xs)
    t0 = time.perf_counter()
    for _ in range(reps):
        smp.run()
    el = time.perf_counter() - t0
    return reps * smp.fraction, el


def cpu_baseline(name: str, xs: int):
    """The oracle with its BLAS on every core and, in a child process whose BLAS and OpenMP
    thread counts are set to 1, on one core."""
    evals, el = oracle_rate(name, xs)
    line = {"value": evals / el, "unit": "evals/s", "cores": _cores(), "kind": "oracle",
            "sample": f"the numpy FP64 oracle's energy+gradient evaluation of {WORKLOADS[name].split(':')[0]} "
                      f"over {xs} of its aux functions ({evals:.2e} evaluations) in {el:.1f} s, scaled by the aux "
                      f"count (every term it spends time on is a sum over the aux index); BLAS threads as configured"}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    xs1 = max(1, xs // 2)
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_rate({name!r}, {xs1})))")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        e1, t1 = json.loads(out.stdout.strip().splitlines()[-1])
        line["single_thread"] = {"value": e1 / t1, "unit": "evals/s", "cores": 1,
                                 "sample": f"{xs1} aux functions ({e1:.2e} evaluations) in {t1:.1f} s"}
        line["parallel_speedup"] = line["value"] / (e1 / t1)
    except (subprocess.SubprocessError, ValueError, IndexError) as exc:
        line["single_thread"] = {"value": None, "error": str(exc)[:200]}
    return line


def run_reference(args):
    """The oracle on the headline workload (or the --workload system): every step one sample of
    one aux function's share of an evaluation (about 4 s), rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = HEADLINE if args.workload == "default" else args.workload
    if name not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle sample for workload {name}"}))
        return 0
    xs = 1 if name == "h1000" else (4 if name == "h200" else 500)
    smp = OracleSample(name, xs)
    for _ in range(args.warmup):
        smp.run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.run()
    el = time.perf_counter() - t0
    v = args.steps * smp.fraction / el
    sample = (f"{args.steps} timed steps, each the numpy FP64 oracle's energy+gradient evaluation over {smp.xs} of "
              f"the {smp.X} aux functions ({smp.fraction:.2e} of an evaluation; every term it spends time on is a "
              f"sum over the aux index), set-up excluded")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# the native path
# ---------------------------------------------------------------------------------------
def _sizes_label(s):
    return {"nbf": s["nbf"], "naux": s["naux"], "nact": s["nact"]}


def run_system(name, args, stream, prec, rank=0, world=1, dist=None, steps=None, warmup=None, e2e=True,
               fp64=True, fp64_steps=1, clocks=False, local=0):
    """Time the energy+gradient evaluation of one named system: the timed region (K steps), the
    per-contraction CUDA-event profile, the end-to-end loop from host buffers, the plain FP64 path
    on the same inputs (rate and accuracy). Returns a dict; the contexts are freed on return."""
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    xyz, orb, aux = workload(2 + rank, name)

    def make_ctx(p):
        ctx = nof.Context(precision=p, stream=stream)
        ctx.build_B(xyz, orb, aux)
        return ctx

    t0 = time.perf_counter()
    ctx = make_ctx(prec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    s = ctx.sizes
    n = s["nbf"]
    nd = ctx.split_digits() if prec == nof.PREC_SPLIT_BF16 else 0
    tiles = None
    if prec == nof.PREC_SPLIT_BF16:
        t = ctx.tuned_tiles()
        tiles = {"gemm1_bn": t[0], "gemm2_bn": t[1], "gemm3_bn": t[2], "gemm3_chunk_atoms": t[3],
                 "picked_by": "autotuner (CUDA-event timing of candidate launch shapes at set-up; GEMM1 with L2 flushed)"}
    Q = torch.tensor(inputs.random_orthogonal(n, rank), dtype=torch.float64, device="cuda")
    C = ctx.lowdin(Q)
    gam = torch.tensor(inputs.random_gamma(s["ngamma"], 1), dtype=torch.float64, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(n, n, dtype=torch.float64, device="cuda")
    gg = torch.empty(s["ngamma"], dtype=torch.float64, device="cuda")
    # contexts that take the timed steps in turn: one when its B (digits or FP64) is more than twice
    # L2, else two with separate copies of B, so that every evaluation reads a B last touched two
    # steps earlier (inputs larger than L2 instead of a flush between steps)
    b_bytes = (2 * nd if nd else 8) * s["naux"] * n * n
    ctxs = [ctx] if b_bytes > 2 * L2_BYTES else [ctx, make_ctx(prec)]
    for c in ctxs:
        for _ in range(warmup):
            c.energy_grad(C, gam, E, g, gg)
    torch.cuda.synchronize()
    runs = [(lambda c=c: c.energy_grad(C, gam, E, g, gg)) for c in ctxs]
    per_eval = None
    if not args.no_graph:
        cgs = []
        l0 = nof.kernel_launches()
        for c in ctxs:
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, stream=stream):
                c.energy_grad(C, gam, E, g, gg)
            cgs.append(cg)
        per_eval = (nof.kernel_launches() - l0) // len(ctxs)
        torch.cuda.synchronize()
        for cg in cgs:
            cg.replay()
        torch.cuda.synchronize()
        runs = [cg.replay for cg in cgs]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        sampler.__enter__()
    l0 = nof.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        runs[i % len(runs)]()
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
    ms = e0.elapsed_time(e1)
    launches = nof.kernel_launches() - l0 if per_eval is None else per_eval * steps
    value, t_max = aggregate(ms, steps, world, dist, device="cuda")
    E_fast, g_fast = float(E.item()), g.clone()

    # each contraction timed with CUDA events inside the library (direct calls), ctx alternating
    # with the others as in the timed loop
    prof = {}
    pe = max(2, min(steps, 5))
    for which in ((1, 2, 3) if prec == nof.PREC_SPLIT_BF16 else (1,)):
        ctx.profile(which)
        for i in range(pe * len(ctxs)):
            ctxs[i % len(ctxs)].energy_grad(C, gam, E, g, gg)
        ms_w, cnt, kname = ctx.profile_read()
        ctx.profile(0)
        prof[which] = (ms_w / max(cnt, 1), kname)
    dom = max(prof, key=lambda w: prof[w][0])
    roof = roofline(prec, s, dom, prof[dom][0], prof[dom][1], nd=nd or 5)
    roof["all_contractions_ms_per_launch"] = {CONTRACTIONS[w][0]: prof[w][0] for w in prof}

    out = {"workload": WORKLOADS[name], "sizes": _sizes_label(s), "value": value, "ms_per_step": t_max / steps,
           "steps": steps, "warmup": warmup, "setup_s": round(setup_s, 2), "digits": nd or None, "tiles": tiles,
           "l2": ("inputs larger than L2: two contexts with separate copies of B's digits take the steps in turn"
                  if len(ctxs) == 2 else f"inputs larger than L2 (B: {b_bytes / 1e9:.2f} GB per context)"),
           "timing": ("CUDA-graph replay of one evaluation per step" if not args.no_graph else "one API call per step")
                     + ", one region bracketed by CUDA events on the library's stream",
           "gpu_launches": int(launches), "roofline": roof,
           "eval_roofline": eval_roofline(prec, s, t_max / steps, nd=nd or 5)}
    if sampler:
        out["clocks"] = sampler.summary()

    if e2e:
        out["e2e"] = e2e_loop(ctxs, C, gam, E, g, gg, stream, max(3, steps // 2), world, g_fast)
    for c in ctxs[1:]:
        c.close()

    # the plain FP64 GPU path on the same (C, gamma): its rate and the split path's accuracy
    if fp64 and prec == nof.PREC_SPLIT_BF16:
        ctx.close()
        torch.cuda.synchronize()
        c64 = make_ctx(nof.PREC_FP64)
        c64.energy_grad(C, gam, E, g, gg)  # warm-up (module loads, first launches)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(fp64_steps):
            c64.energy_grad(C, gam, E, g, gg)
        a1.record(stream)
        torch.cuda.synchronize()
        rate64 = fp64_steps / (a0.elapsed_time(a1) / 1e3)
        dE = abs(E_fast - float(E.item()))
        dg = float((g_fast - g).abs().max().item())
        out["fp64_plain_evals_per_s"] = rate64
        out["fp64_plain_steps"] = fp64_steps
        out["speedup_vs_fp64_plain"] = value / world / rate64
        out["accuracy"] = {"max_abs_dE_vs_fp64_gpu": dE, "max_abs_dg_vs_fp64_gpu": dg, "gate": ACC_GATE,
                           "pass": bool(dE <= ACC_GATE and dg <= ACC_GATE)}
        c64.close()
    else:
        ctx.close()
    torch.cuda.synchronize()
    return out


def e2e_loop(ctxs, C, gam, E, g, gg, stream, steps, world, g_ref):
    """End to end through the public API from pinned host buffers, pipelined the way a serving loop
    runs: every step uploads its own C and gamma and the host reads back every step's E and g. Two
    device buffer sets take the steps in turn (with two contexts, one per set); step i's upload (on
    a copy stream) and step i-1's readback (on a second copy stream) overlap evaluation i, and the
    evaluations stay serialised on the library's stream."""
    import torch
    n = C.shape[0]
    hC = C.cpu().pin_memory()
    hgam = gam.cpu().pin_memory()
    hE = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    hg = [torch.empty(n, n, dtype=torch.float64).pin_memory() for _ in range(2)]
    bC, bgam = [torch.empty_like(C) for _ in range(2)], [torch.empty_like(gam) for _ in range(2)]
    bE, bg, bgg = [torch.empty_like(E) for _ in range(2)], [torch.empty_like(g) for _ in range(2)], \
        [torch.empty_like(gg) for _ in range(2)]
    ectx = ctxs * 2 if len(ctxs) == 1 else ctxs
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("up", "done", "down")}
    # one untimed pass over both buffer sets (the library records their graphs on the second call)
    for k in range(2):
        for _ in range(2):
            ectx[k].energy_grad(bC[k].copy_(C), bgam[k].copy_(gam), bE[k], bg[k], bgg[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps + 1):
        if i < steps:
            k = i % 2
            with torch.cuda.stream(up):
                up.wait_event(ev["done"][k])
                bC[k].copy_(hC, non_blocking=True)
                bgam[k].copy_(hgam, non_blocking=True)
                ev["up"][k].record(up)
            with torch.cuda.stream(stream):
                stream.wait_event(ev["up"][k])
                stream.wait_event(ev["down"][k])
                ectx[k].energy_grad(bC[k], bgam[k], bE[k], bg[k], bgg[k])
                ev["done"][k].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev["done"][k])
                hE[k].copy_(bE[k], non_blocking=True)
                hg[k].copy_(bg[k], non_blocking=True)
                ev["down"][k].record(down)
        if i >= 1:
            ev["down"][(i - 1) % 2].synchronize()
    e2e_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    ok = bool(torch.equal(hg[(steps - 1) % 2], g_ref.cpu()))
    return {"value": world * steps / e2e_s, "unit": "evals/s", "steps": steps,
            "h2d_bytes_per_step": hC.numel() * 8 + hgam.numel() * 8,
            "d2h_bytes_per_step": hE[0].numel() * 8 + hg[0].numel() * 8,
            "pipeline": "two buffer sets in turn: upload of step i and readback of step i-1 overlap evaluation i",
            "readback_matches_device": ok}


def run_batch_system(args, warmup=None, steps=None):
    """Many independent geometries (H-chain frames of uneven length, Gaussian displacements sigma
    = 0.05 bohr, 3 s + 10 aux s per H) evaluated concurrently: every context on its own stream,
    the whole batch captured as one CUDA graph and replayed; L2 flushed before each replay.
    Returns a dict."""
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs
    warmup = args.warmup if warmup is None else warmup
    orb, aux = inputs.basis_3s_10aux()
    sizes = [int(x) for x in inputs.batch_sizes(args.batch_count, seed=3, lo=8, hi=args.batch_max)]
    t0 = time.perf_counter()
    ctxs, Cs, gs, Es, Gs, GGs = [], [], [], [], [], []
    for i, N in enumerate(sizes):
        ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, stream=torch.cuda.Stream())
        ctx.build_B(inputs.displaced_chain(N, seed=4 * 1000003 + i), orb, aux)
        s = ctx.sizes
        Q = torch.tensor(inputs.random_orthogonal(s["nbf"], 5000 + i), dtype=torch.float64, device="cuda")
        Cs.append(ctx.lowdin(Q))
        gs.append(torch.tensor(inputs.random_gamma(s["ngamma"], 6000 + i), dtype=torch.float64, device="cuda"))
        Es.append(torch.empty(1, dtype=torch.float64, device="cuda"))
        Gs.append(torch.empty(s["nbf"], s["nbf"], dtype=torch.float64, device="cuda"))
        GGs.append(torch.empty(s["ngamma"], dtype=torch.float64, device="cuda"))
        ctxs.append(ctx)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    master = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        nof.energy_grad_batch(ctxs, Cs, gs, Es, Gs, GGs, stream=master)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l0 = nof.kernel_launches()
    with torch.cuda.graph(graph, stream=master):
        nof.energy_grad_batch(ctxs, Cs, gs, Es, Gs, GGs, stream=master)
    per_batch = nof.kernel_launches() - l0
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    reps = steps if steps is not None else max(3, args.steps // max(1, len(ctxs)))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with ClockSampler(0) as clk:
        for i in range(reps):
            with torch.cuda.stream(master):
                flush.fill_(float(i))
                evs[i][0].record(master)
                graph.replay()
                evs[i][1].record(master)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    # algorithmic work of the batch (sum over frames) and its whole-batch roofline
    peaks, src = _peaks()
    fl, by = 0.0, 0.0
    for c in ctxs:
        f1, b1 = eval_work(c.sizes["naux"], c.sizes["nbf"], c.sizes["nact"])
        fl += f1
        by += b1
    nd = ctxs[0].split_digits()
    t_roof = max(fl / (peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) / (nd * (nd + 1) // 2) * 1e12),
                 by / (peaks["hbm_gbs"] * 1e9))
    out = {"workload": f"batch of {len(ctxs)} H-chain frames, lengths {min(sizes)}..{max(sizes)} (even, seed 3), "
                       f"sigma 0.05 bohr displacements, 3 s + 10 aux s per H",
           "value": len(ctxs) * reps / (ms / 1e3), "ms_per_step": ms / reps, "steps": reps, "warmup": warmup,
           "frames": len(ctxs), "setup_s": round(setup_s, 1), "digits": nd,
           "timing": "one CUDA-graph replay of the whole batch per step (CUDA events on the master stream), L2 "
                     "flushed (256 MiB write) before each step",
           "gpu_launches": per_batch * reps, "clocks": clk.summary(),
           "eval_roofline": {"algorithmic_flops": fl, "algorithmic_bytes": by, "t_roofline_ms": t_roof * 1e3,
                             "ms_per_batch": ms / reps, "frac": t_roof * 1e3 / (ms / reps), "peak_source": src}}
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()
    return out


def run_batch(args):
    o = run_batch_system(args)
    line = {"metric": METRIC, "value": o["value"], "unit": "evals/s", "n_gpus": 1, "steps": o["steps"],
            "warmup": o["warmup"], "ms_per_step": o["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"bf16-digit{o['digits']}", "data": "synthetic",
            "config": {"workload": o["workload"]}, "setup": {k: o[k] for k in ("timing", "setup_s", "frames")},
            "eval_roofline": o["eval_roofline"], "gpu_launches": o["gpu_launches"], "clocks": o["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def run_nlop(args):
    """The finite-field workload on H2 (R = 1.4 bohr, centred; 3 s + 10 aux s per H; N_g = 1;
    FP64 path): the paper's default ladder NPOINT = 9, STEP = 1e-4 along the bond, i.e. 21
    distinct fields, every field stepped from the field-free core guess until its step reports
    ||g|| < 1e-9 (checked every 25 steps), then the dipoles, differences and Romberg triangles.
    The rate is field-instance steps per second over the whole run (set-up excluded)."""
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs, nlop
    orb, aux = inputs.basis_3s_10aux()
    xyz = inputs.chain(2, 1.4)
    xyz = xyz - xyz.mean(axis=0)
    kw = dict(axis=2, step=1e-4, npoint=9, nsteps=2000, gtol=1e-9, check=25)
    res = None
    times = []
    runs = max(1, min(args.steps, 5))  # a run is a whole workload (about half a second)
    for rep in range(args.warmup + runs):  # every run builds its own contexts (set-up untimed)
        r = {}
        res = nlop.finite_field(xyz, orb, aux, **kw, timing=r)
        if rep >= args.warmup:
            times.append((r["ms"], int(res["steps"].sum()), r["step_launches"]))
    ms = sum(t[0] for t in times)
    total_steps = sum(t[1] for t in times)
    line = {"metric": "field-instance alternating steps/s (finite-field NLOP workload)",
            "value": total_steps / (ms / 1e3), "unit": "steps/s", "n_gpus": 1, "steps": runs,
            "warmup": args.warmup, "ms_per_step": ms / runs, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "H2 R=1.4 bohr, 3 s + 10 aux s per H, N_g=1, field along the bond, "
                                   "NPOINT=9, STEP=1e-4 (21 fields), stop at ||g|| < 1e-9 (checked every 25 "
                                   "steps), at most 2000 steps",
                       "runs": "one bench step is one whole run of the workload (at most 5 runs)",
                       "timing": "wall time, device synchronised on both sides, of the stepping (one "
                                 "CUDA-graph replay of the batched step per step; host convergence checks "
                                 "every 25 steps included), dipoles, differences and triangles of one run; "
                                 "context set-up excluded",
                       "steps_per_field": [int(x) for x in res["steps"]]},
            "result": {k: {"value": res[k][1][0], "delta": res[k][1][1], "k": res[k][1][2], "j": res[k][1][3]}
                       for k in ("alpha", "beta", "gamma")},
            "gpu_launches": int(sum(t[2] for t in times))}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = nlop_cpu_baseline(xyz, orb, aux)
    print(json.dumps(line), flush=True)
    return 0


def nlop_cpu_baseline(xyz, orb, aux, nfield=3):
    """The oracle's stepping for the first `nfield` fields of the same workload (same stopping
    rule), in field-instance steps per second."""
    import numpy as np
    from oracle import integrals, nlop as onlop, pnof, reference, ri, step as ostep
    S, T, V = integrals.one_electron(orb, xyz)
    H = T + V
    B = ri.fitted_B(orb, aux, xyz)
    vnn = integrals.nuclear_repulsion(xyz)
    pm = pnof.PairMap(2, 1, S.shape[0])
    D = onlop.dipole_integrals(orb, xyz)
    C0 = reference.core_guess(S, H)
    done = 0
    t0 = time.perf_counter()
    for f in onlop.field_points(1e-4, 9)[:nfield]:
        Hf, vf = onlop.field_hamiltonian(H, D, [0.0, 0.0, f], xyz, vnn)
        st = ostep.State(C0, np.full(pm.ngamma, 0.3))
        for it in range(2000):
            _, gn, _ = ostep.step(B, Hf, vf, st, pm)
            done += 1
            if (it + 1) % 25 == 0 and gn < 1e-9:
                break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "steps/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{done} oracle steps over the first {nfield} of the 21 fields in {dt:.1f} s"}


def run_gradient(args):
    """Nuclear gradients per second for the H50 chain of the h50 workload (FP64 path, the state of
    the h50 workload: Loewdin orbitals of a seeded rotation, seeded gamma), L2 flushed before each
    gradient, CUDA events on the context's stream."""
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs
    xyz, orb, aux = workload(2, "h50")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = nof.Context(precision=nof.PREC_FP64, stream=stream)
    ctx.build_B(xyz, orb, aux)
    s = ctx.sizes
    C = ctx.lowdin(torch.tensor(inputs.random_orthogonal(s["nbf"], 0), dtype=torch.float64, device="cuda"))
    gam = torch.tensor(inputs.random_gamma(s["ngamma"], 1), dtype=torch.float64, device="cuda")
    grad = torch.empty(xyz.shape[0], 3, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    steps = max(1, min(args.steps, 20))
    for _ in range(max(3, args.warmup)):
        ctx.nuclear_gradient(C, gam, grad)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = nof.kernel_launches()
    with ClockSampler(0) as clk:
        torch.cuda.nvtx.range_push("grads")  # the range a launch list can select (ncu --nvtx-include grads/)
        for i in range(steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            ctx.nuclear_gradient(C, gam, grad)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = nof.kernel_launches() - l0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    g = grad.cpu().numpy()
    line = {"metric": "nuclear gradients/s (RI-PNOF7, FP64 path)", "value": steps / (ms / 1e3), "unit": "gradients/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (FP64 path)", "l2": "flushed (256 MiB write) before every gradient",
                       "timing": "CUDA events on the context's stream around one gradient (J/K, Lagrangian, "
                                 "fitting coefficients, Gamma, Z, integral-derivative contractions)"},
            "result": {"max_abs_component": float(np.abs(g).max()), "net_force": float(np.abs(g.sum(axis=0)).max())},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_dynamics(args):
    """Born-Oppenheimer velocity Verlet of H2 (3 s + 10 aux s per H, FP64 path): every step
    converges the state at the new geometry (graph-replayed steps until ||g|| < 1e-8) and takes the
    analytic gradient. The rate is MD steps per second (wall time, device synchronised)."""
    import numpy as np
    import torch
    from paper_2512_13550_gb300 import geometry, inputs
    orb, aux = inputs.basis_3s_10aux()
    m_h = 1837.15
    x0 = np.array([[0.0, 0.0, -0.775], [0.0, 0.0, 0.775]])
    nsteps = max(2, min(args.steps, 20))
    geometry.verlet(x0, np.zeros((2, 3)), [m_h, m_h], 10.0, 1, orb, aux)  # warm-up (module loads, first contexts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xs, vs, Es = geometry.verlet(x0, np.zeros((2, 3)), [m_h, m_h], 10.0, nsteps, orb, aux)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    kin = 0.5 * m_h * np.sum(vs ** 2, axis=(1, 2))
    tot = Es + kin
    line = {"metric": "Born-Oppenheimer MD steps/s (converged RI-PNOF7 states, analytic forces)",
            "value": nsteps / dt, "unit": "steps/s", "n_gpus": 1, "steps": nsteps, "warmup": 1,
            "ms_per_step": 1e3 * dt / nsteps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "H2 from R = 1.55 bohr at rest, 3 s + 10 aux s per H, N_g = 1, dt = 10 au, "
                                   "every geometry converged to ||g|| < 1e-8 from the core guess",
                       "timing": "wall time, device synchronised on both sides, of the whole trajectory (one "
                                 "more converged point than steps)"},
            "result": {"R_final": float(np.linalg.norm(xs[-1, 1] - xs[-1, 0])),
                       "energy_drift": float(np.max(np.abs(tot - tot[0])))}}
    print(json.dumps(line), flush=True)
    return 0


def run_optimize(args):
    """The converged ON / NO loop (nof_optimize) on one system from its core-Hamiltonian guess and
    gamma = 0.3, split precision: outer iterations, evaluations and wall time (device synchronised
    on both sides; every evaluation ends with a three-number read-back that the loop's decisions
    need) to ||g||_F < gtol and |dE| < etol; set-up and core guess timed separately."""
    import torch
    import paper_2512_13550_gb300 as nof
    name = args.opt_system
    xyz, orb, aux = workload(2, name)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, stream=stream)
    ctx.build_B(xyz, orb, aux)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    C, _ = ctx.core_guess()
    gam = torch.full((ctx.sizes["ngamma"],), 0.3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    l0 = nof.kernel_launches()
    with ClockSampler(0) as clk:
        r = ctx.optimize(C, gam, gtol=args.opt_gtol, etol=args.opt_etol, maxit=args.opt_maxit,
                         eps_rel=args.opt_eps_rel, lr_grow=args.opt_lr_grow, maxloop=args.opt_maxloop,
                         orbopt=args.opt_orbopt)
        torch.cuda.synchronize()
    t3 = time.perf_counter()
    launches = nof.kernel_launches() - l0
    hist = r.pop("history")
    E_fin = r["E"]
    # first outer iteration whose energy is within 1e-6 Ha of the final one, and the evaluations
    # spent until then (each outer iteration after the first costs 1 + maxloop evaluations)
    k6 = next((k for k in range(len(hist)) if abs(hist[k, 0] - E_fin) < 1e-6), len(hist) - 1)
    ev6 = int(round(r["evaluations"] * (k6 + 1) / max(1, len(hist))))  # pro rata over the iterations
    sec = t3 - t2
    line = {"metric": "converged ON/NO optimisation (split precision): wall time to ||g|| < gtol",
            "value": sec, "unit": "s", "n_gpus": 1, "steps": r["iterations"], "warmup": 0,
            "ms_per_step": 1e3 * sec / max(1, r["iterations"]), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": f"bf16-digit{ctx.split_digits()}", "data": "synthetic",
            "config": {"workload": WORKLOADS[name] + ", from the core-Hamiltonian guess, gamma = 0.3",
                       "gtol": args.opt_gtol, "etol": args.opt_etol, "maxloop": args.opt_maxloop, "lr0": 0.02,
                       "eps_rel": args.opt_eps_rel, "lr_grow": args.opt_lr_grow, "orbopt": args.opt_orbopt},
            "result": r | {"evaluations_per_s": r["evaluations"] / sec,
                           "iterations_to_1e-6_Ha": int(k6) + 1, "evaluations_to_1e-6_Ha": int(ev6),
                           "seconds_to_1e-6_Ha_est": sec * ev6 / max(1, r["evaluations"]),
                           "E_history": [[int(k), float(hist[k, 0]), float(hist[k, 1])]
                                         for k in sorted(set(list(range(0, len(hist), max(1, len(hist) // 12)))
                                                             + [len(hist) - 1]))]},
            "setup_s": round(t1 - t0, 2), "core_guess_s": round(t2 - t1, 2),
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "nlop":
        return run_nlop(args)
    if args.workload == "gradient":
        return run_gradient(args)
    if args.workload == "dynamics":
        return run_dynamics(args)
    if args.workload == "optimize":
        return run_optimize(args)
    import torch
    import paper_2512_13550_gb300 as nof

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = HEADLINE if args.workload == "default" else args.workload
    prec = nof.PREC_SPLIT_BF16 if args.precision == "split" else nof.PREC_FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    if args.profile_evals:
        xyz, orb, aux = workload(2, name)
        ctx = nof.Context(precision=prec, stream=stream)
        ctx.build_B(xyz, orb, aux)
        s = ctx.sizes
        from paper_2512_13550_gb300 import inputs
        C = ctx.lowdin(torch.tensor(inputs.random_orthogonal(s["nbf"], 0), dtype=torch.float64, device="cuda"))
        gam = torch.tensor(inputs.random_gamma(s["ngamma"], 1), dtype=torch.float64, device="cuda")
        for _ in range(max(1, args.warmup)):
            E, _, _ = ctx.energy_grad(C, gam)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("evals")
        for _ in range(args.profile_evals):
            E, _, _ = ctx.energy_grad(C, gam)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_evals": args.profile_evals, "workload": name, "precision": prec,
                          "E": float(E.item())}), flush=True)
        return 0

    head = run_system(name, args, stream, prec, rank=rank, world=world, dist=dist, clocks=True, local=local,
                      fp64_steps=1 if name == "h1000" else 3)
    extras = {}
    if args.workload == "default" and not args.no_extras and world == 1:
        # the other workloads, each with its own rate, end-to-end rate, rooflines and FP64 comparison
        extras["h200"] = run_system("h200", args, stream, prec, steps=max(args.steps, 20), fp64_steps=3)
        extras["h50"] = run_system("h50", args, stream, prec, steps=max(10 * args.steps, 200), fp64_steps=10)
        if prec == nof.PREC_SPLIT_BF16:
            extras["batch"] = run_batch_system(args, warmup=3, steps=3)
    if dist is not None:
        dist.barrier()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    nd = head["digits"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": (f"bf16-digit{nd} (exact BF16 digit-plane products of ~{8 * nd}-bit operands, FP32 exact level "
                  f"sums, double-float/FP64 between the contractions)") if nd else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[name]},
        "setup": {k: head[k] for k in ("sizes", "setup_s", "tiles", "l2", "timing")} |
                 {"parallelism": f"replicas x{world}"},
        "accuracy": head.get("accuracy"),
        "fp64_plain_evals_per_s": head.get("fp64_plain_evals_per_s"),
        "speedup_vs_fp64_plain": head.get("speedup_vs_fp64_plain"),
        "roofline": head["roofline"],
        "eval_roofline": head["eval_roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head.get("clocks"),
    }
    if extras:
        line["configs"] = extras
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, 2 if name == "h1000" else (8 if name == "h200" else 500))
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def aggregate(ms_local: float, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput of `world` replicas: each rank evaluated `steps` of its own geometries
    in ms_local; the job takes as long as the slowest rank. Returns (value per second, t_max ms)."""
    t_max = ms_local
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return world * steps / (t_max / 1e3), t_max


if __name__ == "__main__":
    sys.exit(main())
