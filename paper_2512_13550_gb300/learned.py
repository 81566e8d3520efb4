"""Learned starting guess for the occupations and orbitals (a machine-learning add-on; the paper has none).

A perceptron (x -> relu 256 -> relu 256 -> y) maps per-pair features to y = sin^2 gamma_g (twice the
weak occupation of subspace g; unlike gamma itself it is unique, since the trigonometric mapping is
even and pi-periodic in gamma) of the occupation optimum at the core-Hamiltonian orbitals, so a new
geometry can start from predicted occupations instead of a constant. Training pairs come from the
method itself: nof_core_guess, then one nof_step with the orbital rate set to zero and a long
occupation loop (the ON optimisation of the paper with J, K fixed). Every network operation runs
in the library's FP32 kernels (nof_mlp_forward / nof_mlp_loss_grad / nof_mlp_adam); the features
are host-side statistics of the geometry and of the core-guess orbital energies.

Features of subspace g (strong orbital g, weak orbital N - 1 - g for N_g = 1): the core energies of
both orbitals and their gap, the distance of the pair from the Fermi level (g' = N/2 - 1 - g) as
g'/(N/2) and 1/(g' + 1), 8/N, and the mean and spread of the bond lengths (bohr).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, inputs, load_library

NFEAT = 8


def pair_features(xyz: np.ndarray, eps: np.ndarray, nelec: int) -> np.ndarray:
    npair = nelec // 2
    d = np.linalg.norm(np.diff(xyz, axis=0), axis=1) if xyz.shape[0] > 1 else np.zeros(1)
    out = np.zeros((npair, NFEAT))
    for g in range(npair):
        p = 2 * npair - 1 - g
        gp = npair - 1 - g
        out[g] = [eps[g], eps[p], eps[p] - eps[g], gp / npair, 1.0 / (gp + 1), 8.0 / nelec,
                  d.mean(), d.std()]
    return out


def _he_init(F, H, O, seed):
    """He-style normal weights and zero biases from the shared seeded generator (host, once)."""
    parts, k = [], 0
    for shape in [(H, F), (H,), (H, H), (H,), (O, H), (O,)]:
        m = int(np.prod(shape))
        parts.append(inputs.normal(seed * 7919 + k, m) * np.sqrt(2.0 / shape[1]) if len(shape) == 2 else np.zeros(m))
        k += 1
    return np.concatenate(parts)


class MLP:
    """FP32 perceptron on the device, trained with Adam; parameters and moments are torch tensors."""

    def __init__(self, F: int = NFEAT, H: int = 256, O: int = 1, seed: int = 0):
        import torch
        lib = load_library()
        self.F, self.H, self.O = F, H, O
        self.P = int(lib.nof_mlp_param_count(F, H, O))
        self.theta = torch.tensor(_he_init(F, H, O, seed), dtype=torch.float32, device="cuda")
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.t = 0
        self.mu = np.zeros(F)
        self.sd = np.ones(F)


def _fptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def mlp_loss_grad(net: MLP, X, T, work=None):
    """Loss and gradient (into net.grad) for device FP32 batches X [B][F], T [B][O]."""
    import torch
    B = X.shape[0]
    work = torch.empty(int(load_library().nof_mlp_work_size(B, net.H, net.O)), dtype=torch.float32,
                       device="cuda") if work is None else work
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(load_library().nof_mlp_loss_grad(B, net.F, net.H, net.O, _fptr(net.theta), _fptr(X), _fptr(T),
                                            _fptr(loss), _fptr(net.grad), _fptr(work), _stream()))
    return loss


def mlp_forward(net: MLP, X):
    import torch
    B = X.shape[0]
    work = torch.empty(int(load_library().nof_mlp_work_size(B, net.H, net.O)), dtype=torch.float32, device="cuda")
    Y = torch.empty(B, net.O, dtype=torch.float32, device="cuda")
    _check(load_library().nof_mlp_forward(B, net.F, net.H, net.O, _fptr(net.theta), _fptr(X), _fptr(Y),
                                          _fptr(work), _stream()))
    return Y


def mlp_adam(net: MLP, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    net.t += 1
    _check(load_library().nof_mlp_adam(net.P, _fptr(net.theta), _fptr(net.grad), _fptr(net.m), _fptr(net.v),
                                       net.t, lr, b1, b2, eps, wd, _stream()))


def train(net: MLP, feats: np.ndarray, targets: np.ndarray, iters: int = 800, lr: float = 1e-3, wd: float = 0.3):
    """Full-batch Adam on standardised features; returns the loss history (host floats)."""
    import torch
    net.mu = feats.mean(0)
    net.sd = feats.std(0) + 1e-8
    X = torch.tensor((feats - net.mu) / net.sd, dtype=torch.float32, device="cuda")
    T = torch.tensor(targets.reshape(-1, net.O), dtype=torch.float32, device="cuda")
    work = torch.empty(int(load_library().nof_mlp_work_size(X.shape[0], net.H, net.O)), dtype=torch.float32,
                       device="cuda")
    hist = []
    for it in range(iters):
        loss = mlp_loss_grad(net, X, T, work)
        mlp_adam(net, lr, wd=wd)
        if it % 20 == 0 or it == iters - 1:
            hist.append(float(loss.item()))
    return hist


def predict(net: MLP, feats: np.ndarray) -> np.ndarray:
    """Network output y (= predicted sin^2 gamma) per pair."""
    import torch
    X = torch.tensor((feats - net.mu) / net.sd, dtype=torch.float32, device="cuda")
    return mlp_forward(net, X).cpu().numpy().reshape(-1).astype(np.float64)


def angles(y: np.ndarray) -> np.ndarray:
    """Occupation angles in [0, pi/2] from predicted sin^2 gamma."""
    return np.arcsin(np.sqrt(np.clip(y, 0.0, 1.0)))


# ----------------------------------------------------------------------------------------------
# Data from the method itself
# ----------------------------------------------------------------------------------------------

def optimise(ctx, gamma0: np.ndarray, steps: int, C0=None):
    """Run `steps` alternating ON/NO steps from the core guess (or C0); returns the per-step energies,
    the final gamma (host) and the core orbital energies."""
    import torch
    n = ctx.sizes["nbf"]
    if C0 is None:
        C, eps = ctx.core_guess()
    else:
        C, eps = C0.clone(), None
    gam = torch.tensor(gamma0, dtype=torch.float64, device="cuda")
    m = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(m)
    ctx.t = ctypes.c_int(0)
    Es = []
    for _ in range(steps):
        out = ctx.step(C, gam, m, v)
        Es.append(out)
    Es = torch.stack(Es).cpu().numpy()
    return Es, gam.cpu().numpy(), (eps.cpu().numpy() if eps is not None else None)


def generate(sizes, orb, aux, seed=11, precision=1, on_iters=300, gamma0=0.3):
    """(features, sin^2 gamma*) pairs for displaced H chains of the given lengths, gamma* being the
    occupation optimum at the core-Hamiltonian orbitals."""
    from . import Context
    feats, targs = [], []
    for i, N in enumerate(sizes):
        xyz = inputs.displaced_chain(int(N), seed=seed * 100003 + i)
        ctx = Context(precision=precision, lr=0.0, on_iters=on_iters)
        ctx.build_B(xyz, orb, aux)
        _, gam, eps = optimise(ctx, np.full(ctx.sizes["ngamma"], gamma0), 1)
        feats.append(pair_features(xyz, eps, int(N)))
        targs.append(np.sin(gam[: int(N) // 2]) ** 2)
        ctx.close()
    return np.concatenate(feats), np.concatenate(targs)


def evaluate(net: MLP, sizes, orb, aux, steps=60, seed=13, precision=1, gamma0=0.3, straight=False):
    """Energies along the optimisation from the core guess with learned vs constant starting
    angles, for held-out geometries (displaced chains, or straight 1.8-bohr chains): list of
    (N, E_learned[steps], E_constant[steps], seconds: set-up, core guess, per step)."""
    import time

    import torch

    from . import Context
    out = []
    for i, N in enumerate(sizes):
        xyz = inputs.chain(int(N), 1.8) if straight else inputs.displaced_chain(int(N), seed=seed * 100003 + i)
        t0 = time.perf_counter()
        ctx = Context(precision=precision)
        ctx.build_B(xyz, orb, aux)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        C0, eps = ctx.core_guess()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ng = ctx.sizes["ngamma"]
        g_learn = np.full(ng, gamma0)
        g_learn[: int(N) // 2] = angles(predict(net, pair_features(xyz, eps.cpu().numpy(), int(N))))
        E1, _, _ = optimise(ctx, g_learn, steps, C0=C0)
        t3 = time.perf_counter()
        E2, _, _ = optimise(ctx, np.full(ng, gamma0), steps, C0=C0)
        out.append((int(N), E1[:, 0], E2[:, 0], (t1 - t0, t2 - t1, (t3 - t2) / steps)))
        ctx.close()
    return out


def main(argv=None):
    """Generate training data with the method, train, and compare learned against constant starts
    on held-out chains; prints one JSON line."""
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-chains", type=int, default=600)
    ap.add_argument("--max-len", type=int, default=32)
    ap.add_argument("--eval-sizes", type=int, nargs="*", default=[40, 48, 64])
    ap.add_argument("--eval-steps", type=int, default=40)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--min-len", type=int, default=6)
    ap.add_argument("--basis", choices=["3s10aux", "h1000"], default="3s10aux",
                    help="3s10aux: 3 s + 10 aux s per H; h1000: 1 contracted s + 3 aux s per H")
    ap.add_argument("--straight-eval", action="store_true", help="evaluate on straight 1.8-bohr chains")
    ap.add_argument("--converged", action="store_true",
                    help="train on converged solutions (occupations and pair rotation angles, nof_optimize) "
                         "and compare learned and core-guess starts to convergence on held-out chains")
    ap.add_argument("--gtol", type=float, default=1e-4)
    args = ap.parse_args(argv)
    if args.converged:
        return study(args)
    orb, aux = inputs.basis_h1000() if args.basis == "h1000" else inputs.basis_3s_10aux()
    t0 = time.perf_counter()
    X, y = generate(inputs.batch_sizes(args.train_chains, seed=21, lo=args.min_len, hi=args.max_len), orb, aux,
                    seed=11)
    Xv, yv = generate(inputs.batch_sizes(max(8, args.train_chains // 8), seed=22, lo=args.min_len, hi=args.max_len),
                      orb, aux, seed=12)
    t_data = time.perf_counter() - t0
    net = MLP(NFEAT, 256, 1, seed=0)
    t0 = time.perf_counter()
    hist = train(net, X, y, iters=args.iters, lr=1e-3, wd=0.3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pv = predict(net, Xv)
    res = evaluate(net, args.eval_sizes, orb, aux, steps=args.eval_steps, straight=args.straight_eval)
    rows = []
    for N, El, Ec, secs in res:
        Emin = min(El.min(), Ec.min())
        def first(E, tol):
            idx = np.nonzero(E - Emin <= tol)[0]
            return int(idx[0]) + 1 if idx.size else None
        rows.append({"N": N, "E_first_learned": float(El[0]), "E_first_constant": float(Ec[0]),
                     "E_end_learned": float(El[-1]), "E_end_constant": float(Ec[-1]),
                     "steps_to_1e-3_learned": first(El, 1e-3), "steps_to_1e-3_constant": first(Ec, 1e-3),
                     "setup_s": round(secs[0], 2), "core_guess_s": round(secs[1], 2), "step_s": round(secs[2], 4),
                     "E_learned_every_5": [float(x) for x in El[4::5]],
                     "E_constant_every_5": [float(x) for x in Ec[4::5]]})
    print(json.dumps({"basis": args.basis, "train_pairs": int(X.shape[0]), "data_s": round(t_data, 1), "train_s": round(t_train, 2),
                      "loss_first": hist[0], "loss_last": hist[-1],
                      "val_rmse": float(np.sqrt(np.mean((pv - yv) ** 2))),
                      "val_rmse_mean_predictor": float(np.sqrt(np.mean((y.mean() - yv) ** 2))),
                      "eval": rows}))


# ----------------------------------------------------------------------------------------------
# Occupations and orbital rotations from converged solutions (the loop of nof_optimize)
# ----------------------------------------------------------------------------------------------
NOUT = 2  # per pair: sin^2 gamma_g and the rotation angle between orbitals g and p(g)


def pair_partner(npair: int, g: int) -> int:
    """Weak orbital p(g) of subspace g for N_g = 1 (Fig. 1 pairing: HOMO-LUMO, HOMO-1 - LUMO+1, ...)."""
    return 2 * npair - 1 - g


def rotation_targets(C0: np.ndarray, C: np.ndarray, S: np.ndarray, npair: int) -> np.ndarray:
    """theta_g: the plane rotation of the core-guess orbitals g and p(g) closest to the converged
    ones. With U = C0^T S C (C = C0 U), the 2 x 2 block of U on (g, p(g)) is matched by the rotation
    [[cos, sin], [-sin, cos]] that maximises the trace of its product with the block (orthogonal
    Procrustes): theta = atan2(U_pg - U_gp, U_gg + U_pp). The energy does not change when a
    converged orbital changes sign, so both sign choices of column p(g) are tried and the one whose
    block a rotation fits best (the larger Procrustes trace, the norm of the atan2 arguments) is
    kept; changing both signs is a rotation by pi, so the angle is reduced to (-pi/2, pi/2]."""
    U = C0.T @ S @ C
    out = np.zeros(npair)
    for g in range(npair):
        p = pair_partner(npair, g)
        fits = []
        for sp in (1.0, -1.0):
            y, x = U[p, g] - sp * U[g, p], U[g, g] + sp * U[p, p]
            fits.append((np.hypot(x, y), np.arctan2(y, x)))
        th = max(fits)[1]
        out[g] = (th + 0.5 * np.pi) % np.pi - 0.5 * np.pi
    return out


class BF16Net:
    """The trained network's parameters converted once to BF16 for inference on the tensor cores
    (nof_mlp_forward_bf16); the standardisation of the features is the training one."""

    def __init__(self, net: MLP):
        import torch
        self.net = net
        self.wb = torch.empty(net.P, dtype=torch.int16, device="cuda")
        _check(load_library().nof_mlp_to_bf16(net.P, _fptr(net.theta), ctypes.c_void_p(self.wb.data_ptr()),
                                              _stream()))

    def __call__(self, feats: np.ndarray) -> np.ndarray:
        import torch
        net = self.net
        X = torch.tensor((feats - net.mu) / net.sd, dtype=torch.float32, device="cuda")
        B = X.shape[0]
        Y = torch.empty(B, net.O, dtype=torch.float32, device="cuda")
        work = torch.empty(2 * B * net.H, dtype=torch.float32, device="cuda")
        _check(load_library().nof_mlp_forward_bf16(B, net.F, net.H, net.O, ctypes.c_void_p(self.wb.data_ptr()),
                                                   _fptr(net.theta), _fptr(X), _fptr(Y), _fptr(work), _stream()))
        return Y.cpu().numpy().astype(np.float64)


def converged_solutions(sizes, orb, aux, seed=31, gtol=1e-4, etol=1e-7, maxit=3000, precision=1):
    """Per-pair features and targets (sin^2 gamma*, theta*) from converged solutions of displaced
    H chains: nof_optimize from the core guess and gamma = 0.3 to ||g|| < gtol. Returns (X, T,
    records) with one record per chain (N, iterations, evaluations, converged, seconds)."""
    import time

    import torch

    from . import Context
    feats, targs, recs = [], [], []
    for i, N in enumerate(sizes):
        N = int(N)
        xyz = inputs.displaced_chain(N, seed=seed * 100003 + i)
        ctx = Context(precision=precision)
        ctx.build_B(xyz, orb, aux)
        S, _ = ctx.get_SH()
        C0, eps = ctx.core_guess()
        C = C0.clone()
        gam = torch.full((ctx.sizes["ngamma"],), 0.3, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        r = ctx.optimize(C, gam, gtol=gtol, etol=etol, maxit=maxit)
        dt = time.perf_counter() - t0
        npair = N // 2
        g = gam.cpu().numpy()[:npair]
        th = rotation_targets(C0.cpu().numpy(), C.cpu().numpy(), S.cpu().numpy(), npair)
        feats.append(pair_features(xyz, eps.cpu().numpy(), N))
        targs.append(np.stack([np.sin(g) ** 2, th], axis=1))
        recs.append((N, r["iterations"], r["evaluations"], r["converged"], round(dt, 3), r["E"]))
        ctx.close()
    return np.concatenate(feats), np.concatenate(targs), recs


def learned_start(bnet: BF16Net, xyz, eps: np.ndarray, C0, ngamma: int, gamma0: float = 0.3,
                  rotate: bool = True):
    """The learned starting point: gamma_g from the predicted sin^2 gamma, and C0 exp(Y) with
    Y_{g, p(g)} = -Y_{p(g), g} the predicted pair angles (BF16 inference; C0 itself when rotate is
    False). Returns (C, gamma) as device tensors."""
    import torch
    from scipy.linalg import expm
    N = xyz.shape[0]
    npair = N // 2
    y = bnet(pair_features(xyz, eps, N))
    gam = np.full(ngamma, gamma0)
    gam[:npair] = angles(y[:, 0])
    n = C0.shape[0]
    Y = np.zeros((n, n))
    for g in range(npair if rotate else 0):  # exp(Y) rotates the plane (g, p(g)) by theta_g: C_g -> cos C_g + sin C_p
        p = pair_partner(npair, g)
        Y[p, g] = y[g, 1]
        Y[g, p] = -y[g, 1]
    C = torch.tensor(C0.cpu().numpy() @ expm(Y), dtype=torch.float64, device="cuda")
    return C, torch.tensor(gam, dtype=torch.float64, device="cuda")


def optimize_with_fallback(ctx, learned, core, **params):
    """nof_optimize from the learned start; when that does not converge, again from the core guess
    (the automatic fallback). The learned start's first energy is no criterion: on held-out chains
    it lies above the core guess's while the loop from it converges in fewer evaluations. Returns
    the result of the run that is kept, with "fallback" set and the evaluations of both runs."""
    r = ctx.optimize(learned[0].clone(), learned[1].clone(), **params)
    if r["converged"]:
        r["fallback"] = False
        return r, learned
    spent = r["evaluations"]
    r = ctx.optimize(core[0].clone(), core[1].clone(), **params)
    r["fallback"] = True
    r["evaluations"] += spent
    return r, core


def compare_starts(bnet: BF16Net, sizes, orb, aux, seed=41, gtol=1e-4, etol=1e-7, maxit=3000, precision=1):
    """Held-out displaced chains, optimised to convergence from the core guess (gamma = 0.3), from the
    learned start (occupations and pair rotations), from the learned occupations alone and through
    the fallback: per chain (N, E_start and evaluations, seconds, E_final for each start)."""
    import time

    import torch

    from . import Context
    out = []
    for i, N in enumerate(sizes):
        N = int(N)
        xyz = inputs.displaced_chain(N, seed=seed * 100003 + i)
        ctx = Context(precision=precision)
        ctx.build_B(xyz, orb, aux)
        C0, eps = ctx.core_guess()
        row = {"N": N}
        e = eps.cpu().numpy()
        starts = {"core": (C0.clone(), torch.full((ctx.sizes["ngamma"],), 0.3, dtype=torch.float64, device="cuda")),
                  "learned": learned_start(bnet, xyz, e, C0, ctx.sizes["ngamma"]),
                  "learned_occupations": learned_start(bnet, xyz, e, C0, ctx.sizes["ngamma"], rotate=False)}
        for name in ("core", "learned", "learned_occupations", "learned_or_core"):
            t0 = time.perf_counter()
            if name == "learned_or_core":
                r, _ = optimize_with_fallback(ctx, starts["learned"], starts["core"], gtol=gtol, etol=etol, maxit=maxit)
            else:
                C, gam = starts[name]
                r = ctx.optimize(C.clone(), gam.clone(), gtol=gtol, etol=etol, maxit=maxit)
            dt = time.perf_counter() - t0
            row[name] = {"E_start": float(r["history"][0, 0]), "E_final": r["E"], "iterations": r["iterations"],
                         "evaluations": r["evaluations"], "converged": r["converged"], "seconds": round(dt, 3)}
            if name == "learned_or_core":
                row[name]["fallback"] = r["fallback"]
        out.append(row)
        ctx.close()
    return out

def study(args):
    """Converged training data, training, BF16 inference and the comparison of starts; one JSON line."""
    import json
    import time

    import torch
    orb, aux = inputs.basis_h1000() if args.basis == "h1000" else inputs.basis_3s_10aux()
    t0 = time.perf_counter()
    X, T, recs = converged_solutions(inputs.batch_sizes(args.train_chains, seed=21, lo=args.min_len, hi=args.max_len),
                                     orb, aux, seed=31, gtol=args.gtol)
    Xv, Tv, _ = converged_solutions(inputs.batch_sizes(max(8, args.train_chains // 8), seed=22, lo=args.min_len,
                                                       hi=args.max_len), orb, aux, seed=32, gtol=args.gtol)
    t_data = time.perf_counter() - t0
    net = MLP(NFEAT, 256, NOUT, seed=0)
    t0 = time.perf_counter()
    hist = train(net, X, T, iters=args.iters, lr=1e-3, wd=0.3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    bnet = BF16Net(net)
    pv = bnet(Xv)
    rmse = np.sqrt(np.mean((pv - Tv) ** 2, axis=0))
    base = np.sqrt(np.mean((T.mean(0) - Tv) ** 2, axis=0))
    rows = compare_starts(bnet, args.eval_sizes, orb, aux, gtol=args.gtol)
    print(json.dumps({"basis": args.basis, "train_chains": len(recs), "train_pairs": int(X.shape[0]),
                      "converged_fraction": float(np.mean([r[3] for r in recs])),
                      "mean_evaluations_per_training_chain": float(np.mean([r[2] for r in recs])),
                      "data_s": round(t_data, 1), "train_s": round(t_train, 2), "loss_first": hist[0],
                      "loss_last": hist[-1], "val_rmse_bf16": rmse.tolist(), "val_rmse_mean_predictor": base.tolist(),
                      "eval": rows}))
    return 0


if __name__ == "__main__":
    main()
