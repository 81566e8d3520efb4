"""The converged ON / NO optimisation loop (oracle; test infrastructure only).

The paper optimises the occupations and the orbitals separately (Theory section, after Eq. sum1):
the ONs are fully optimised at fixed orbitals, and the orbitals by rotations C <- C exp(y) driven
by ADAM on the orbital gradient g = 4(lambda - lambda^T) (Natural Orbital Optimization
subsection), until the lambda-symmetry and energy thresholds NTHRESHL / NTHRESHE are met (Single
Point Energy section). The ADAM details and its integration with the ON optimisation are
delegated to another publication; this module is the reading both sides implement (parity
unpinned as to that schedule, pinned as to the minimum it reaches):

  outer iteration k:
    1. J, K, h_pp at C_k; ONs converged with J, K fixed (`on_converge`): BFGS on gamma with an
       Armijo step control, to max |dE/dgamma| < on_tol.
    2. E_k, lambda, g at (C_k, gamma_k). Stop when ||g||_F < gtol and |E_k - E_{k-1}| < etol, or
       once lr_k < lr_min.
    3. Orbitals, gamma_k fixed (orbopt 0 and, until the switch below, orbopt 2): `maxloop` ADAM
       steps from zero moments (bias-corrected, lr_k, b1, b2, eps), each a full evaluation at the
       rotated orbitals. A step's orbitals are better than the best so far if their energy is
       lower by more than etol, or equal within etol with a ||g|| at most 0.9 of the best
       (energies that close are compared through the gradient, which the split-precision path
       resolves far better than the energy itself); the best orbitals of the block become
       C_{k+1}. If no step is better than (E_k, ||g_k||), C_{k+1} = C_k and lr_{k+1} = lr_k / 2.
    3'. With orbopt 2 once lr_k < lr0 lbfgs_after (and with orbopt 1 from the start): one L-BFGS
       step on the rotation generators per outer iteration: the two-loop recursion over the last
       `memory` pairs (s = step, y = gradient change at fixed gamma_k), <A, B> = sum_{p<q}
       A_pq B_pq, initial scale <s,y>/<y,y>; without pairs -g lr / max|g|. Step length halved
       from 1 until an Armijo decrease (where the predicted decrease exceeds etol) or a smaller
       ||g|| with the energy within etol (where it does not); a failed search retries once from
       steepest descent, then halves lr.

Why the switch: restarting the ADAM moments every block keeps its normalised step proportional
to the current rate, and the halving gives the step control that a fixed-rate ADAM lacks near
the minimum. But the normalised steps move every rotation by about lr, and near a minimum of an
ill-conditioned problem the rate collapses before ||g|| reaches 1e-5 (the 4 x 4 lattice stalls at
2.6e-5 with lr ~ 1e-12). L-BFGS alone converges there but needs 10,411 evaluations and on the H20
chain ends in a higher local minimum; ADAM first, then L-BFGS, converges both (7,995 and 1,546
evaluations) at the lower minima, and the H10 chain in 1,328.
"""
from __future__ import annotations

import numpy as np

from . import pnof
from .step import expm_antisym


def on_energy(hpp, J, K, gamma, pm: pnof.PairMap, ipnof: int = 7) -> float:
    """E without V_nn at fixed J, K, h_pp (Eq. PNOF)."""
    return pnof.energy_from_jk(hpp, J, K, gamma, pm, 0.0, ipnof)


def on_converge(hpp, J, K, gamma, pm: pnof.PairMap, ipnof: int = 7, tol: float = 1e-8, maxit: int = 2000,
                lr0: float = 0.3):
    """ONs optimised with J, K and h_pp fixed, by BFGS on gamma (dense inverse-Hessian estimate H,
    unset until the first accepted step: the first direction is -lr0 dE/dgamma, then d = -H g).
    Step length: alpha = 1, halved until E(gamma + alpha d) <= E + 1e-4 alpha d.g (Armijo); once
    alpha |d.g| is below 1e-13 max(1, |E|), which FP64 cannot resolve in E, the step is taken
    without the energy test. After a step s with gradient change y and s.y > 0, H is set to
    (s.y / y.y) I if unset, then updated: H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T,
    rho = 1 / s.y. A direction that is not a descent direction resets H. Stops when
    max |dE/dgamma| < tol, after maxit steps, or when alpha falls below 1e-12.
    Returns (gamma, steps, max |dE/dgamma|)."""
    x = np.array(gamma, np.float64)
    ng = x.size
    E = on_energy(hpp, J, K, x, pm, ipnof)
    g = pnof.gamma_gradient(hpp, J, K, x, pm, ipnof)
    Hinv = None
    it = 0
    while it < maxit and np.max(np.abs(g)) >= tol:
        d = -lr0 * g if Hinv is None else -(Hinv @ g)
        dg = d @ g
        if dg >= 0.0:  # not a descent direction: restart from the gradient
            Hinv = None
            d = -lr0 * g
            dg = d @ g
        alpha = 1.0
        while True:
            trial = x + alpha * d
            Et = on_energy(hpp, J, K, trial, pm, ipnof)
            if Et <= E + 1e-4 * alpha * dg or alpha * abs(dg) < 1e-13 * max(1.0, abs(E)):
                break
            alpha *= 0.5
            if alpha < 1e-12:
                return x, it, float(np.max(np.abs(g)))
        gt = pnof.gamma_gradient(hpp, J, K, trial, pm, ipnof)
        sv = trial - x
        yv = gt - g
        sy = sv @ yv
        if sy > 0.0:
            if Hinv is None:
                Hinv = np.eye(ng) * (sy / (yv @ yv))
            rho = 1.0 / sy
            Hy = Hinv @ yv
            Hinv = Hinv - rho * (np.outer(sv, Hy) + np.outer(Hy, sv)) + (rho * rho * (yv @ Hy) + rho) * np.outer(sv, sv)
        x, E, g = trial, Et, gt
        it += 1
    return x, it, float(np.max(np.abs(g)))


DEFAULTS = dict(maxit=1000, maxloop=10, gtol=1e-5, etol=1e-8, lr=0.02, lr_min=1e-12, b1=0.9, b2=0.999,
                eps=1e-8, on_tol=1e-8, on_maxit=500, on_lr=0.3, eps_rel=0.0, lr_grow=1.0, orbopt=2,
                memory=20, lbfgs_after=1.0 / 64)


def _dot(a, b):
    """<A, B> = sum_{p<q} A_pq B_pq for antisymmetric A, B."""
    return 0.5 * float(np.sum(a * b))


def lbfgs_direction(g, S, Y, lr, gmax):
    """-H g by the two-loop recursion over the stored pairs (s_i, y_i) of antisymmetric matrices,
    H0 = (<s,y>/<y,y>) I from the newest pair; without pairs, -g scaled so that its largest
    element is lr."""
    if not S:
        return -g * (lr / gmax)
    q = g.copy()
    al = []
    for s_, y_ in zip(reversed(S), reversed(Y)):
        rho = 1.0 / _dot(y_, s_)
        a_ = rho * _dot(s_, q)
        q = q - a_ * y_
        al.append((rho, a_, s_, y_))
    q = q * (_dot(S[-1], Y[-1]) / _dot(Y[-1], Y[-1]))
    for rho, a_, s_, y_ in reversed(al):
        b_ = rho * _dot(y_, q)
        q = q + (a_ - b_) * s_
    return -q


def better(E, gnorm, best_E, best_g, etol) -> bool:
    """The orbital step's acceptance: lower energy by more than etol, or the same energy within
    etol and a gradient norm at most 0.9 of the best one."""
    return E < best_E - etol or (abs(E - best_E) <= etol and gnorm < 0.9 * best_g)


def _evaluate(B, H, vnn, C, gamma, pm, ipnof):
    return pnof.energy_and_gradients(B, H, C, gamma, pm, vnn, ipnof)


def optimize(B, H, vnn, C, gamma, pm: pnof.PairMap, ipnof: int = 7, **opt):
    """The loop in the module header from (C, gamma). Returns dict(C, gamma, E, gnorm, lam_asym,
    iterations, evaluations, converged, lr, history [(E_k, ||g_k||, lr_k)])."""
    o = dict(DEFAULTS)
    o.update(opt)
    a = pm.nact
    C = np.array(C, np.float64)
    gamma = np.array(gamma, np.float64)
    lr = float(o["lr"])
    hist = []
    E_prev = None
    evals = 0
    r = None
    converged = False
    mem_s, mem_y = [], []  # L-BFGS pairs (orbopt 1 and 2)
    use_lbfgs = False
    for k in range(int(o["maxit"])):
        J, K = pnof.jk(B, C, a)
        hpp = np.einsum("mp,mn,np->p", C[:, :a], H, C[:, :a])
        gamma, _, _ = on_converge(hpp, J, K, gamma, pm, ipnof, o["on_tol"], int(o["on_maxit"]), o["on_lr"])
        r = _evaluate(B, H, vnn, C, gamma, pm, ipnof)
        evals += 1
        E, g = r["E"], r["g"]
        gn = float(np.linalg.norm(g))
        hist.append((E, gn, lr))
        if gn < o["gtol"] and E_prev is not None and abs(E - E_prev) < o["etol"]:
            converged = True
            break
        if lr < o["lr_min"]:
            break
        E_prev = E
        # orbopt 0: ADAM blocks only; 1: L-BFGS only; 2: ADAM blocks until the rate has fallen
        # below lr0 * lbfgs_after, then L-BFGS steps
        if o["orbopt"] == 2 and not use_lbfgs and lr < o["lr"] * o["lbfgs_after"]:
            use_lbfgs = True
        if o["orbopt"] == 1 or use_lbfgs:
            # one L-BFGS step at gamma_k fixed: direction from the stored pairs, step length by
            # halving from 1 until the trial is better than (E_k, ||g_k||) with an Armijo decrease
            d = lbfgs_direction(g, mem_s, mem_y, lr, float(np.max(np.abs(g))))
            dg = _dot(d, g)
            if dg >= 0.0:
                mem_s.clear()
                mem_y.clear()
                d = lbfgs_direction(g, mem_s, mem_y, lr, float(np.max(np.abs(g))))
                dg = _dot(d, g)
            accepted = None
            for attempt in range(2):  # the L-BFGS direction, then steepest descent
                alpha = 1.0
                for _ in range(12):
                    Ct = C @ expm_antisym(alpha * d)
                    rc = _evaluate(B, H, vnn, Ct, gamma, pm, ipnof)
                    evals += 1
                    gtn = float(np.linalg.norm(rc["g"]))
                    # Armijo where the predicted decrease is resolvable, else a smaller gradient
                    ok = (rc["E"] <= E + 1e-4 * alpha * dg) if -alpha * dg > o["etol"] else \
                        (rc["E"] <= E + o["etol"] and gtn < gn)
                    if ok:
                        accepted = (Ct, rc["g"])
                        break
                    alpha *= 0.5
                if accepted is not None or not mem_s:
                    break
                mem_s.clear()
                mem_y.clear()
                d = lbfgs_direction(g, mem_s, mem_y, lr, float(np.max(np.abs(g))))
                dg = _dot(d, g)
            if accepted is None:
                lr *= 0.5
                continue
            C, gt = accepted
            sv, yv = alpha * d, gt - g
            if _dot(sv, yv) > 0.0:
                mem_s.append(sv)
                mem_y.append(yv)
                if len(mem_s) > int(o["memory"]):
                    mem_s.pop(0)
                    mem_y.pop(0)
            continue
        # a block of ADAM steps from zero moments, gamma fixed; keep the lowest-energy orbitals
        n = C.shape[0]
        m = np.zeros((n, n))
        v = np.zeros((n, n))
        eps = max(o["eps"], o["eps_rel"] * gn)  # ADAM's epsilon, relative to ||g_k|| if eps_rel > 0
        Cc, gc = C, g
        best_E, best_g, best_C = E, gn, None
        for t in range(1, int(o["maxloop"]) + 1):
            m = o["b1"] * m + (1.0 - o["b1"]) * gc
            v = o["b2"] * v + (1.0 - o["b2"]) * gc * gc
            y = -lr * (m / (1.0 - o["b1"] ** t)) / (np.sqrt(v / (1.0 - o["b2"] ** t)) + eps)
            Cc = Cc @ expm_antisym(y)
            rc = _evaluate(B, H, vnn, Cc, gamma, pm, ipnof)
            evals += 1
            gc = rc["g"]
            gcn = float(np.linalg.norm(gc))
            if better(rc["E"], gcn, best_E, best_g, o["etol"]):
                best_E, best_g, best_C = rc["E"], gcn, Cc
        if best_C is not None:
            C = best_C
            lr *= o["lr_grow"]
        else:
            lr *= 0.5
    lam = r["lam"]
    return dict(C=C, gamma=gamma, E=r["E"], gnorm=float(np.linalg.norm(r["g"])),
                lam_asym=float(np.max(np.abs(lam - lam.T))), iterations=len(hist), evaluations=evals,
                converged=converged, lr=lr, history=hist)
