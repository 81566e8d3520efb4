"""Finite-field polarizability and hyperpolarizabilities on the GPU (NLOPs subsection of
DoNOF 2.0, arXiv 2512.13550).

The differences use the dipole at -2h, -h, 0, h, 2h for every step h_k = STEP 2^{k-1},
k = 1 .. NPOINT. Since 2 h_k = h_{k+1}, these 5 NPOINT points hold 2 NPOINT + 3 distinct
fields: 0 and +-h_1 .. +-h_{NPOINT+1}. Every distinct field gets a context (same geometry and
basis, field set by nof_set_field) and its own state. The states take alternating steps
together (nof_step_batch: one stream per field, forked from and joined to a master stream), at
most `nsteps`. With graph=True (the default) the batched step uses the device-side step
counters and is recorded once as a CUDA graph that every later step replays (re-recorded when
the set of unconverged fields changes), so a step costs one graph launch instead of some 170
kernel launches per field. With `gtol`, every `check` steps the fields whose last step reported
||g|| < gtol stop (the paper converges every field to thresholds; continued ADAM steps would
eventually leave a converged minimum). The dipole along `axis` at each final state
(nof_dipole) then gives the centred differences (nof_field_differences) and the three
Romberg-Richardson triangles with their selected values (nof_romberg). All arithmetic is in the library; this module only allocates
device memory and orders the calls.
"""
from __future__ import annotations

import numpy as np

from . import PREC_FP64, Context, field_differences, polarizability_invariants, romberg, step_batch


def field_points(step: float, npoint: int) -> np.ndarray:
    """The distinct fields in the order nof_field_differences expects: 0, +h_1 .. +h_{n+1},
    -h_1 .. -h_{n+1}."""
    h = step * 2.0 ** np.arange(npoint + 1)
    return np.concatenate([[0.0], h, -h])


def finite_field(xyz, orb, aux, axis: int = 2, step: float = 1e-3, npoint: int = 9, nsteps: int = 100,
                 precision: int = PREC_FP64, C0=None, gamma0=None, gtol=None, check: int = 25, timing=None,
                 graph: bool = True, **opts):
    """alpha, beta, gamma along `axis` from alternating steps at every field.

    C0, gamma0: the common starting point (default: the field-free core guess and gamma = 0.3).
    Returns a dict: fields, mu (dipole along the axis at each field), steps (per field),
    D = (alpha(h), beta(h), gamma(h)), alpha / beta / gamma = (R, (value, Delta, k, j)), and the
    contexts. With a dict `timing`, its "ms" receives the wall time of the stepping, dipoles,
    differences and triangles (device synchronised on both sides; context set-up excluded),
    "setup_launches" the kernel launches of the set-up and "step_launches" those of the
    stepping (graph replays included)."""
    import time
    import torch
    from . import kernel_launches
    l0 = kernel_launches()
    fields = field_points(step, npoint)
    ctxs = []
    for f in fields:
        c = Context(precision=precision, stream=torch.cuda.Stream(), **opts)
        c.build_B(xyz, orb, aux)
        F = np.zeros(3)
        F[axis] = f
        c.set_field(F)
        ctxs.append(c)
    s = ctxs[0].sizes
    n, ng = s["nbf"], s["ngamma"]
    dev = dict(dtype=torch.float64, device="cuda")
    if C0 is None:
        C0, _ = ctxs[0].core_guess()  # fields[0] = 0
    C0 = torch.as_tensor(np.asarray(C0.cpu() if hasattr(C0, "cpu") else C0), **dev)
    g0 = torch.full((ng,), 0.3, **dev) if gamma0 is None else torch.as_tensor(np.asarray(gamma0), **dev)
    torch.cuda.synchronize()
    Cs = [C0.clone() for _ in ctxs]
    gs = [g0.clone() for _ in ctxs]
    ms = [torch.zeros(n, n, **dev) for _ in ctxs]
    vs = [torch.zeros(n, n, **dev) for _ in ctxs]
    outs = [torch.empty(3, **dev) for _ in ctxs]
    torch.cuda.synchronize()
    setup_launches = kernel_launches() - l0
    t0 = time.perf_counter()
    master = torch.cuda.Stream()
    active = list(range(len(ctxs)))
    steps = [0] * len(ctxs)

    def batched_step(idx):
        step_batch([ctxs[i] for i in idx], [Cs[i] for i in idx], [gs[i] for i in idx], [ms[i] for i in idx],
                   [vs[i] for i in idx], [outs[i] for i in idx], stream=master, device_counter=graph)

    launches = 0  # kernels run by the stepping (a replay runs the kernels its recording counted)

    def record(idx):
        g = torch.cuda.CUDAGraph()
        l1 = kernel_launches()
        with torch.cuda.graph(g, stream=master):
            batched_step(idx)
        return g, kernel_launches() - l1

    recorded, per_replay = record(active) if graph else (None, 0)
    for it in range(nsteps):
        if graph:
            with torch.cuda.stream(master):  # a replay runs on the current stream
                recorded.replay()
            launches += per_replay
        else:
            l1 = kernel_launches()
            batched_step(active)
            launches += kernel_launches() - l1
        for i in active:
            steps[i] = it + 1
        if gtol is not None and (it + 1) % check == 0:
            master.synchronize()
            gn = torch.stack([outs[i][1] for i in active]).cpu().numpy()
            still = [i for i, g in zip(active, gn) if not g < gtol]
            if not still:
                break
            if still != active and graph:
                recorded, per_replay = record(still)
            active = still
    master.synchronize()
    mus = [c.dipole(C, g) for c, C, g in zip(ctxs, Cs, gs)]
    torch.cuda.synchronize()
    mu = np.array([m[axis].item() for m in mus])
    al, be, ga = field_differences(mu, npoint, step)
    out = dict(alpha=romberg(al), beta=romberg(be), gamma=romberg(ga))
    if timing is not None:
        timing["ms"] = 1e3 * (time.perf_counter() - t0)
        timing["setup_launches"] = setup_launches
        timing["step_launches"] = launches
    return dict(fields=fields, mu=mu, steps=np.array(steps), D=(al, be, ga), **out,
                steps_out=[o.cpu().numpy() for o in outs], contexts=ctxs)


def isotropic_alpha(xyz, orb, aux, **kw):
    """ISOALPHA: alpha_xx, alpha_yy, alpha_zz (the selected Romberg values of finite_field with the
    field along x, y and z), the isotropic mean and the anisotropy (Raman convention)."""
    diag = []
    for axis in range(3):
        r = finite_field(xyz, orb, aux, axis=axis, **kw)
        diag.append(r["alpha"][1][0])
    iso, aniso = polarizability_invariants(*diag)
    return dict(alpha_diag=tuple(diag), alpha_iso=iso, alpha_aniso=aniso)

