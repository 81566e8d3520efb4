#!/usr/bin/env python3
"""Benchmark of the density-fitted PNOF7 energy+gradient evaluation on one GB300.

Workload: H50 linear chain (spacing 1.8 bohr + U(-0.1, 0.1) seeded jitter per bond), 3
even-tempered s functions per H (alpha = 0.2 * 4^k) and 10 aux s per H (alpha = 0.1 * 3^k):
nbf = 150, naux = 500, 50 active orbitals, PNOF7 with 25 pairs and N_g = 1. One step is one
energy+gradient evaluation (transforms, J, K, energy, Lagrangian, orbital and occupation
gradients) at fixed (C, gamma), with C = S^{-1/2} Q for a seeded random orthogonal Q and
gamma ~ U(0.1, 1.2). The K timed steps are one region bracketed by CUDA events on the library's
stream. Every step's inputs exceed L2: when one context's B is smaller than twice L2 (H50: 90 MB
of digits), two contexts of the workload with separate copies of B take the steps in turn, so
each evaluation reads a B last touched two steps earlier.

Under torchrun (N > 1) every rank evaluates its own independent geometry (seed 2 + rank):
the path has no exchange step, so the ranks are replicas and `value` sums their work.

`--impl reference` times the CPU FP64 oracle (test infrastructure) on the same workload.
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
WORKLOAD = ("H50 chain, spacing 1.8+U(-0.1,0.1) bohr, 3 s/H (0.2*4^k) + 10 aux s/H (0.1*3^k): "
            "nbf=150, naux=500, nact=50, PNOF7, 25 pairs, N_g=1")
ACC_GATE = 1e-6
L2_BYTES = 129 * 1000 * 1000  # GB300 L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=["auto", "split", "fp64"], default="auto")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["h50", "h200", "batch", "nlop", "gradient", "dynamics"],
                    default="h50",
                    help="h50: the single-geometry benchmark; h200: the 10 x 20 lattice (nbf 600, "
                         "naux 2000, nact 200); batch: many uneven H-chain frames evaluated "
                         "concurrently as one CUDA-graph launch; nlop: the finite-field polarizability "
                         "and hyperpolarizabilities of H2 (21 field instances stepped together); gradient: "
                         "the nuclear gradient of the H50 chain on the FP64 path; dynamics: velocity-Verlet "
                         "steps of H2 on converged states")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-max", type=int, default=64, help="largest chain length in the batch")
    ap.add_argument("--no-graph", action="store_true",
                    help="time plain API calls instead of CUDA-graph replays of one evaluation")
    ap.add_argument("--profile-evals", type=int, default=0,
                    help="profiling mode: build, warm up, run this many evaluations inside the NVTX "
                         "range 'evals' (for ncu --nvtx --nvtx-include evals/) and exit")
    return ap.parse_args()


WORKLOAD_H200 = ("H200 10x20 square lattice, spacing 2.0 bohr, 3 s/H (0.2*4^k) + 10 aux s/H (0.1*3^k): "
                 "nbf=600, naux=2000, nact=200, PNOF7, 100 pairs, N_g=1")


def workload(seed=2, name="h50"):
    from paper_2512_13550_gb300 import inputs
    orb, aux = inputs.basis_3s_10aux()
    if name == "h200":
        return inputs.lattice(10, 20, 2.0), orb, aux
    xyz = inputs.jittered_chain(50, seed)
    return xyz, orb, aux


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


# ---------------------------------------------------------------------------------------
def oracle_setup(seed=2):
    """The oracle's one-time set-up for the H50 workload (integrals, RI fit, orbitals)."""
    from oracle import integrals, pnof, reference, ri
    from paper_2512_13550_gb300 import inputs
    xyz, orb, aux = workload(seed)
    S, T, V = integrals.one_electron(orb, xyz)
    B = ri.fitted_B(orb, aux, xyz)
    vnn = integrals.nuclear_repulsion(xyz)
    n = S.shape[0]
    pm = pnof.PairMap(50, 1, n)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 0))
    gam = inputs.random_gamma(pm.ngamma, 1)
    return (B, T + V, C, gam, pm, vnn)


def oracle_eval(system):
    from oracle import pnof
    return pnof.energy_and_gradients(*system)


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def oracle_rate(budget_s: float):
    """(evaluations, seconds) of the FP64 oracle (as it stands) on a bounded sample of H50
    evaluations, set-up excluded."""
    system = oracle_setup()
    oracle_eval(system)
    t0 = time.perf_counter()
    count = 0
    while True:
        oracle_eval(system)
        count += 1
        el = time.perf_counter() - t0
        if el >= budget_s or count >= 1000:
            break
    return count, el


def cpu_baseline(budget_s: float):
    """The oracle with its BLAS on every core, and (in a child process whose BLAS and OpenMP
    thread counts are set to 1) on one core."""
    count, el = oracle_rate(budget_s)
    line = {"value": count / el, "unit": "evals/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{count} H50 energy+gradient evaluations of the numpy FP64 oracle in "
                      f"{el:.1f} s (set-up excluded; BLAS threads as configured)"}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.oracle_rate({budget_s / 2!r})))")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=10 * budget_s + 120)
        c1, e1 = json.loads(out.stdout.strip().splitlines()[-1])
        line["single_thread"] = {"value": c1 / e1, "unit": "evals/s", "cores": 1,
                                 "sample": f"{c1} evaluations in {e1:.1f} s"}
        line["parallel_speedup"] = line["value"] / (c1 / e1)  # BLAS on all cores over one core
    except (subprocess.SubprocessError, ValueError, IndexError) as exc:
        line["single_thread"] = {"value": None, "error": str(exc)[:200]}
    return line


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    system = oracle_setup()
    for _ in range(args.warmup):
        oracle_eval(system)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_eval(system)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"{args.steps} timed H50 energy+gradient evaluations of the "
                                       f"numpy FP64 oracle (set-up excluded)"},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
def run_batch(args):
    """Throughput of many independent geometries (H-chain frames of uneven length, Gaussian
    displacements sigma = 0.05 bohr, 3 s + 10 aux s per H) evaluated concurrently: every context on
    its own stream, the whole batch captured as one CUDA graph and replayed."""
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs
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
    for _ in range(args.warmup):
        nof.energy_grad_batch(ctxs, Cs, gs, Es, Gs, GGs, stream=master)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l0 = nof.kernel_launches()
    with torch.cuda.graph(graph, stream=master):
        nof.energy_grad_batch(ctxs, Cs, gs, Es, Gs, GGs, stream=master)
    per_batch = nof.kernel_launches() - l0
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    reps = max(3, args.steps // max(1, len(ctxs)))
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
    line = {"metric": METRIC, "value": len(ctxs) * reps / (ms / 1e3), "unit": "evals/s", "n_gpus": 1,
            "steps": reps, "warmup": args.warmup, "ms_per_step": ms / reps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"batch of {len(ctxs)} H-chain frames, lengths {min(sizes)}..{max(sizes)} "
                                   f"(even, seed 3), sigma 0.05 bohr displacements, 3 s + 10 aux s per H",
                       "timing": "one CUDA-graph replay of the whole batch per step, L2 flushed between steps",
                       "setup_s": round(setup_s, 1)},
            "gpu_launches": per_batch * reps, "clocks": clk.summary()}
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
    import torch
    import paper_2512_13550_gb300 as nof
    from paper_2512_13550_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec = {"auto": nof.PREC_SPLIT_BF16, "split": nof.PREC_SPLIT_BF16, "fp64": nof.PREC_FP64}[args.precision]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    xyz, orb, aux = workload(2 + rank, args.workload)
    wl_name = WORKLOAD_H200 if args.workload == "h200" else WORKLOAD

    def make_ctx(p):
        ctx = nof.Context(precision=p, stream=stream)
        ctx.build_B(xyz, orb, aux)
        return ctx

    try:
        ctx = make_ctx(prec)
    except nof.NofError as e:
        if args.precision != "auto":
            raise
        print(f"# split path unavailable ({e}); timing the FP64 path", file=sys.stderr)
        prec = nof.PREC_FP64
        ctx = make_ctx(prec)
    s = ctx.sizes
    n = s["nbf"]
    tiles = None
    if prec == nof.PREC_SPLIT_BF16:
        t = ctx.tuned_tiles()
        tiles = {"gemm1_bn": t[0], "gemm2_bn": t[1], "gemm3_bn": t[2], "gemm3_chunk_atoms": t[3],
                 "picked_by": "autotuner (CUDA-event timing of candidate launch shapes at set-up; GEMM1 with L2 flushed)"}
    Q = torch.tensor(inputs.random_orthogonal(n, 0), dtype=torch.float64, device="cuda")
    C = ctx.lowdin(Q)
    gam = torch.tensor(inputs.random_gamma(s["ngamma"], 1), dtype=torch.float64, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(n, n, dtype=torch.float64, device="cuda")
    gg = torch.empty(s["ngamma"], dtype=torch.float64, device="cuda")

    if args.profile_evals:
        for _ in range(max(1, args.warmup)):
            ctx.energy_grad(C, gam, E, g, gg)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("evals")
        for _ in range(args.profile_evals):
            ctx.energy_grad(C, gam, E, g, gg)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_evals": args.profile_evals, "precision": prec,
                          "E": float(E.item())}), flush=True)
        return 0

    def contexts(c, p):
        """The contexts that take the timed steps in turn: `c` alone when its B (digits, or FP64)
        is larger than twice L2, else `c` and a second context of the same workload with its own
        copy of B, so that every evaluation reads a B last touched two steps earlier (inputs
        larger than L2 instead of a flush between steps)."""
        b_bytes = (2 * c.split_digits() if p == nof.PREC_SPLIT_BF16 else 8) * s["naux"] * n * n
        return [c] if b_bytes > L2_BYTES * 2 else [c, make_ctx(p)]

    def timed_loop(cs, steps, warmup, profile=False, graph=False, flush=None):
        """Time `steps` evaluations as one region bracketed by CUDA events, the contexts `cs`
        taking them in turn; returns (ms, kernel launches, profile). With graph=True one evaluation
        per context is captured in a CUDA graph and replayed (the library makes no host
        synchronisation or allocation inside an evaluation, so the capture holds all of it).
        With a `flush` buffer (larger than L2) it is written before every step instead, and each
        step is timed alone."""
        for c in cs:
            for _ in range(warmup):
                c.energy_grad(C, gam, E, g, gg)
        torch.cuda.synchronize()
        runs = [(lambda c=c: c.energy_grad(C, gam, E, g, gg)) for c in cs]
        per_eval = None
        if graph:
            cgs = []
            l0 = nof.kernel_launches()
            for c in cs:
                cg = torch.cuda.CUDAGraph()
                with torch.cuda.graph(cg, stream=stream):
                    c.energy_grad(C, gam, E, g, gg)
                cgs.append(cg)
            per_eval = (nof.kernel_launches() - l0) // len(cs)
            torch.cuda.synchronize()
            for _ in range(warmup):
                for cg in cgs:
                    cg.replay()
            torch.cuda.synchronize()
            runs = [cg.replay for cg in cgs]
        l0 = nof.kernel_launches()
        if flush is not None:
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
            for i in range(steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                runs[i % len(cs)]()
                evs[i][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs)
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(steps):
                runs[i % len(cs)]()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        launches = nof.kernel_launches() - l0 if per_eval is None else per_eval * steps
        prof = None
        if profile:  # the dominant kernel of cs[0], timed with CUDA events inside the library
            cs[0].profile(True)
            for i in range(steps):
                cs[i % len(cs)].energy_grad(C, gam, E, g, gg)
            prof = cs[0].profile_read()
            cs[0].profile(False)
        return ms, launches, prof

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ctxs = contexts(ctx, prec)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, launches, prof = timed_loop(ctxs, args.steps, args.warmup, profile=True, graph=not args.no_graph)
    torch.cuda.synchronize()
    value, t_max = aggregate(ms, args.steps, world, dist, device="cuda")
    # the same steps on one context with a 256 MiB write before each (timed per step), reported
    # beside the value for comparison
    flushbuf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms_fl, _, _ = timed_loop([ctx], args.steps, args.warmup, graph=not args.no_graph, flush=flushbuf)
    del flushbuf
    if dist is not None:
        dist.barrier()
    E_fast = float(E.item())
    g_fast = g.clone()

    # accuracy and throughput of the plain FP64 path on the same inputs
    if prec == nof.PREC_FP64:
        ctx64, E64, dE, dg = ctx, E_fast, 0.0, 0.0
        ms64, steps64 = ms, args.steps
    else:
        ctx64 = make_ctx(nof.PREC_FP64)
        ms64, _, _ = timed_loop(contexts(ctx64, nof.PREC_FP64), args.fp64_steps, 3, graph=not args.no_graph)
        steps64 = args.fp64_steps
        E64 = float(E.item())
        dE = abs(E_fast - E64)
        dg = float((g_fast - g).abs().max().item())

    # end-to-end through the public API from pinned host buffers, pipelined the way a serving
    # loop would run it: every step uploads its own inputs and the host reads back every step's
    # E and g. Two contexts of the workload (each with its own copy of B's digits, 180 MB in all:
    # more than L2) and two buffer sets take the steps in turn on the same stream, so the
    # evaluations stay serialised and each reads a B last touched two steps earlier. Step i's
    # upload (on a copy stream) and step i-1's readback (on a second copy stream) overlap
    # evaluation i; each context replays its recorded graph.
    hC = C.cpu().pin_memory()
    hgam = gam.cpu().pin_memory()
    hE = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    hg = [torch.empty(n, n, dtype=torch.float64).pin_memory() for _ in range(2)]
    bC, bgam = [torch.empty_like(C) for _ in range(2)], [torch.empty_like(gam) for _ in range(2)]
    bE, bg, bgg = [torch.empty_like(E) for _ in range(2)], [torch.empty_like(g) for _ in range(2)], \
        [torch.empty_like(gg) for _ in range(2)]
    ectx = ctxs * 2 if len(ctxs) == 1 else ctxs  # the context of each buffer set
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("up", "done", "down")}
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps + 1):
        if i < e2e_steps:
            k = i % 2
            with torch.cuda.stream(up):  # set k's inputs are free once evaluation i-2 is done
                up.wait_event(ev["done"][k])
                bC[k].copy_(hC, non_blocking=True)
                bgam[k].copy_(hgam, non_blocking=True)
                ev["up"][k].record(up)
            with torch.cuda.stream(stream):
                stream.wait_event(ev["up"][k])
                stream.wait_event(ev["down"][k])  # and its outputs once step i-2's readback is done
                ectx[k].energy_grad(bC[k], bgam[k], bE[k], bg[k], bgg[k])
                ev["done"][k].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev["done"][k])
                hE[k].copy_(bE[k], non_blocking=True)
                hg[k].copy_(bg[k], non_blocking=True)
                ev["down"][k].record(down)
        if i >= 1:
            ev["down"][(i - 1) % 2].synchronize()  # the host has step i-1's E and g
    e2e_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    e2e_ok = bool(torch.equal(hg[(e2e_steps - 1) % 2], g_fast.cpu()))  # g_fast: the timed loop's result
    h2d = hC.numel() * 8 + hgam.numel() * 8
    d2h = hE[0].numel() * 8 + hg[0].numel() * 8

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    dom_ms, dom_launches, dom_name = prof
    roof = roofline(prec, s, dom_ms / max(dom_launches, 1), dom_name, traffic=(
        TRAFFIC_GEMM1_BYTES if args.workload == "h50" else None),
        nd=ctx.split_digits() if prec == nof.PREC_SPLIT_BF16 else 4)
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if prec == nof.PREC_SPLIT_BF16 else "f64",
        "data": "synthetic",
        "config": {"workload": wl_name, "path": "split-bf16 tcgen05" if prec else "plain fp64",
                   "tiles": tiles,
                   "l2": ("inputs larger than L2: two contexts with separate copies of B's digits take "
                          "the steps in turn" if len(ctxs) == 2 else "inputs larger than L2 (B's digits)"),
                   "l2_flushed_evals_per_s": args.steps / (ms_fl / 1e3),
                   "timing": "CUDA-graph replay of one evaluation per step" if not args.no_graph
                             else "one API call per step",
                   "parallelism": f"replicas x{world}"},
        "accuracy": {"max_abs_dE_vs_fp64_gpu": dE, "max_abs_dg_vs_fp64_gpu": dg,
                     "gate": ACC_GATE, "pass": bool(dE <= ACC_GATE and dg <= ACC_GATE)},
        "fp64_plain_evals_per_s": steps64 / (ms64 / 1e3),
        "speedup_vs_fp64_plain": value / world / (steps64 / (ms64 / 1e3)),
        "roofline": roof,
        "e2e": {"value": world * e2e_steps / e2e_s, "unit": "evals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "two buffer sets in turn: upload of step i and readback of step i-1 overlap evaluation i",
                "l2": ("two contexts in turn, each with its own copy of B's digits (more than L2 in all)"
                       if ectx[0] is not ectx[1] else "inputs larger than L2 (B's digits)"),
                "readback_matches_device": e2e_ok},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and args.workload == "h50":
        line["cpu_baseline"] = cpu_baseline(args.cpu_budget)
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


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 roofline of the plain path: 2 FP64 FMA per clock per SM (the rate an FMA-throughput probe
# measured on GB300: 1.19 TFLOP/s), x 152 SMs x 2.07 GHz x 2 FLOP = 1.26 TFLOP/s.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12

# DRAM bytes (read + write) of one GEMM1 launch on the H50 workload from an ncu capture of the
# current kernel (profiles/), or None when the kernel has changed since the counters were taken.
TRAFFIC_GEMM1_BYTES = 96589824 + 4070656  # profiles/digit_gemm_h50_ncu.md (paired-MMA kernel)


def roofline(prec, s, ms_per_launch, name, traffic=None, nd=4):
    n, X, a = s["nbf"], s["naux"], s["nact"]
    peaks, src = _peaks()
    if prec == 0:
        flops = 2.0 * X * n * n * a  # half transform T = B C_a
        achieved = flops / (ms_per_launch / 1e3) / 1e12
        peak = FP64_PEAK_TFLOPS
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if peak else None, "traffic": None,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz (probe-measured rate)"}
    # half transform GEMM1: reads the nd BF16 digit planes of B (2 nd bytes per element of B) and
    # writes T as double-floats (8 bytes per element of T); on the tensor cores it is
    # nd (nd + 1) / 2 BF16 digit-plane products of (X n) x n x a. It is timed inside evaluation
    # steps that run back to back, so a tensor bound takes the sustained BF16 peak.
    nbytes = 2.0 * nd * X * n * n + 8.0 * X * n * a
    flops = nd * (nd + 1) // 2 * 2.0 * X * n * n * a
    tc_peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    t_tc = flops / (tc_peak * 1e12)
    sec = ms_per_launch / 1e3
    if t_tc > t_hbm:
        achieved = flops / sec / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": achieved / tc_peak, "traffic": traffic, "algorithmic_flops": flops,
                "algorithmic_bytes": nbytes, "ms_per_launch": ms_per_launch, "digits": nd,
                "peak_source": f"{src} BF16 dense GEMM, sustained (MEASURED_PEAKS.json bf16_tflops_sustained)"}
    achieved = nbytes / sec / 1e9
    peak = peaks["hbm_gbs"]
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes": nbytes, "ms_per_launch": ms_per_launch, "digits": nd,
            "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


if __name__ == "__main__":
    sys.exit(main())
