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
    2. E_k, lambda, g at (C_k, gamma_k). Stop when ||g||_F < gtol and |E_k - E_{k-1}| < etol.
    3. `maxloop` ADAM steps on the orbitals from zero moments with gamma_k fixed (bias-corrected,
       lr_k, b1, b2, eps), each a full evaluation at the rotated orbitals; the lowest-energy
       orbitals of the block become C_{k+1}. If none of them lowers E_k, C_{k+1} = C_k and the
       rate halves: lr_{k+1} = lr_k / 2. The loop also stops once lr_k < lr_min: the energy can
       then no longer be lowered at FP64 resolution (near ||g|| ~ 1e-7 on small chains the best
       possible decrease along -g is below the energy's rounding).

Restarting the moments every block keeps ADAM's normalised step proportional to the current
rate instead of to the gradients of earlier blocks, and the halving gives the step control that
a fixed-rate ADAM lacks near the minimum (a single ADAM run with halving stalls at ||g|| ~ 1e-3
on the H10 chain; this loop reaches 1e-5 in 86 outer iterations).
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
                eps=1e-8, on_tol=1e-8, on_maxit=500, on_lr=0.3)


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
        # a block of ADAM steps from zero moments, gamma fixed; keep the lowest-energy orbitals
        n = C.shape[0]
        m = np.zeros((n, n))
        v = np.zeros((n, n))
        Cc, gc = C, g
        best_E, best_C = E, None
        for t in range(1, int(o["maxloop"]) + 1):
            m = o["b1"] * m + (1.0 - o["b1"]) * gc
            v = o["b2"] * v + (1.0 - o["b2"]) * gc * gc
            y = -lr * (m / (1.0 - o["b1"] ** t)) / (np.sqrt(v / (1.0 - o["b2"] ** t)) + o["eps"])
            Cc = Cc @ expm_antisym(y)
            rc = _evaluate(B, H, vnn, Cc, gamma, pm, ipnof)
            evals += 1
            gc = rc["g"]
            if rc["E"] < best_E:
                best_E, best_C = rc["E"], Cc
        if best_C is not None:
            C = best_C
        else:
            lr *= 0.5
    lam = r["lam"]
    return dict(C=C, gamma=gamma, E=r["E"], gnorm=float(np.linalg.norm(r["g"])),
                lam_asym=float(np.max(np.abs(lam - lam.T))), iterations=len(hist), evaluations=evals,
                converged=converged, lr=lr, history=hist)
