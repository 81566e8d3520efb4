"""Geometry optimisation and Born-Oppenheimer dynamics on converged RI-PNOF states (oracle; test
infrastructure only).

The paper lists geometry optimisation (OPTGEO) and an interface for ab initio molecular dynamics
among DoNOF's capabilities without printing their algorithms. Readings:
  * every geometry gets the converged state of the library's alternating steps from the core
    guess and gamma = 0.3, stopped at the first check (every `check` steps) where the step
    reports ||g|| < gtol (as in nlop.run; gtol = 1e-8 by default: a tighter threshold meets the
    rounding floor of the steps, and further ADAM steps drift off the minimum); the energy and
    the analytic gradient (gradient.py) are taken at that state;
  * optimisation: BFGS on the Cartesian coordinates with the inverse Hessian started at
    I / hess0, each step scaled down to at most `max_step` bohr, stopping when the largest force
    component is below ftol;
  * dynamics: velocity Verlet, x' = x + v dt + a dt^2 / 2, v' = v + (a + a') dt / 2, a = -grad/m.
Parity: the optimised geometry has a vanishing force and the lowest converged energy of a scan
around it, and the trajectory conserves the total energy (tests/test_oracle_dynamics.py).
"""
from __future__ import annotations

import numpy as np

from . import gradient, integrals, pnof, reference, ri, step


def converged_point(orb, aux, xyz, ncwo=1, ipnof=7, gtol=1e-8, check=25, max_steps=4000, Z=None):
    """(E, dE/dR [natom][3], steps) at the converged state of geometry xyz."""
    S, T, V = integrals.one_electron(orb, xyz, Z)
    H = T + V
    B = ri.fitted_B(orb, aux, xyz)
    vnn = integrals.nuclear_repulsion(xyz, Z)
    pm = pnof.PairMap(int(round(np.sum(np.ones(xyz.shape[0]) if Z is None else Z))), ncwo, S.shape[0])
    st = step.State(reference.core_guess(S, H), np.full(pm.ngamma, 0.3))
    done = 0
    for it in range(max_steps):
        _, gn, _ = step.step(B, H, vnn, st, pm, ipnof)
        done = it + 1
        if done % check == 0 and gn < gtol:
            break
    E = pnof.energy(B, H, st.C, st.gamma, pm, vnn, ipnof)
    g = gradient.nuclear_gradient(orb, aux, xyz, st.C, st.gamma, pm, Z, ipnof)
    return E, g, done


def optimize(orb, aux, xyz, ftol=1e-6, max_iter=60, max_step=0.2, hess0=0.5, **kw):
    """BFGS to a stationary point; returns (xyz, E, grad, iterations)."""
    x = np.array(xyz, np.float64).ravel()
    E, g, _ = converged_point(orb, aux, x.reshape(-1, 3), **kw)
    g = g.ravel()
    Hinv = np.eye(x.size) / hess0
    it = 0
    for it in range(1, max_iter + 1):
        if np.max(np.abs(g)) < ftol:
            break
        dx = -Hinv @ g
        nrm = np.linalg.norm(dx)
        if nrm > max_step:
            dx *= max_step / nrm
        x1 = x + dx
        E1, g1, _ = converged_point(orb, aux, x1.reshape(-1, 3), **kw)
        g1 = g1.ravel()
        s, y = x1 - x, g1 - g
        sy = s @ y
        if sy > 1e-12:
            rho = 1.0 / sy
            I = np.eye(x.size)
            Hinv = (I - rho * np.outer(s, y)) @ Hinv @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
        x, E, g = x1, E1, g1
    return x.reshape(-1, 3), E, g.reshape(-1, 3), it


def verlet(orb, aux, xyz, vel, masses, dt, nsteps, **kw):
    """Velocity Verlet; returns positions [nsteps+1][natom][3], velocities, potential energies."""
    x = np.array(xyz, np.float64)
    v = np.array(vel, np.float64)
    m = np.asarray(masses, np.float64)[:, None]
    E, g, _ = converged_point(orb, aux, x, **kw)
    a = -g / m
    xs, vs, Es = [x.copy()], [v.copy()], [E]
    for _ in range(nsteps):
        x = x + v * dt + 0.5 * a * dt * dt
        E, g, _ = converged_point(orb, aux, x, **kw)
        a1 = -g / m
        v = v + 0.5 * (a + a1) * dt
        a = a1
        xs.append(x.copy()); vs.append(v.copy()); Es.append(E)
    return np.array(xs), np.array(vs), np.array(Es)
