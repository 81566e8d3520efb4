"""Geometry optimisation and Born-Oppenheimer dynamics on converged RI-PNOF states (FP64 path).

The paper lists geometry optimisation (OPTGEO) and an ab initio molecular-dynamics interface
among DoNOF's capabilities. At every geometry a context is built, the state is stepped from the
core guess and gamma = 0.3 until a step reports ||g|| < gtol (checked every `check` steps; one
alternating step per CUDA-graph replay, device-side step counter), and the energy and the
analytic nuclear gradient (nof_nuclear_gradient) are taken at that state.
  * optimize: BFGS on the Cartesian coordinates (inverse Hessian started at I / hess0, steps
    scaled down to at most max_step bohr) until the largest force component is below ftol;
  * verlet: velocity Verlet, x' = x + v dt + a dt^2 / 2, v' = v + (a + a') dt / 2, a = -grad / m.
The geometry updates are a few host-side numbers per step; all the electronic-structure work runs
in the library.
"""
from __future__ import annotations

import numpy as np

from . import PREC_FP64, Context


def converged_point(xyz, orb, aux, ncwo: int = 1, ipnof: int = 7, gtol: float = 1e-8, check: int = 25,
                    max_steps: int = 4000):
    """(E, dE/dR [natom][3] as numpy, steps) at the converged state of geometry xyz."""
    import torch
    st = torch.cuda.Stream()
    ctx = Context(precision=PREC_FP64, stream=st, ncwo=ncwo, ipnof=ipnof)
    ctx.build_B(np.asarray(xyz, np.float64), orb, aux)
    n, ng = ctx.sizes["nbf"], ctx.sizes["ngamma"]
    dev = dict(dtype=torch.float64, device="cuda")
    with torch.cuda.stream(st):
        C, _ = ctx.core_guess()
        gam = torch.full((ng,), 0.3, **dev)
        m, v = torch.zeros(n, n, **dev), torch.zeros(n, n, **dev)
        out = torch.empty(3, **dev)
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        ctx.step(C, gam, m, v, out, device_counter=True)
    done = 0
    for it in range(max_steps):
        with torch.cuda.stream(st):
            graph.replay()
        done = it + 1
        if done % check == 0:
            st.synchronize()
            if out[1].item() < gtol:
                break
    with torch.cuda.stream(st):
        E = ctx.energy_grad(C, gam, grad=False)[0]
        g = ctx.nuclear_gradient(C, gam)
    st.synchronize()
    ctx.sync()
    return float(E.item()), g.cpu().numpy(), done


def optimize(xyz, orb, aux, ftol: float = 1e-6, max_iter: int = 60, max_step: float = 0.2, hess0: float = 0.5,
             **kw):
    """BFGS to a stationary point; returns (xyz, E, grad, iterations)."""
    x = np.array(xyz, np.float64).ravel()
    E, g, _ = converged_point(x.reshape(-1, 3), orb, aux, **kw)
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
        E1, g1, _ = converged_point(x1.reshape(-1, 3), orb, aux, **kw)
        g1 = g1.ravel()
        s, y = x1 - x, g1 - g
        sy = float(s @ y)
        if sy > 1e-12:
            rho = 1.0 / sy
            eye = np.eye(x.size)
            Hinv = (eye - rho * np.outer(s, y)) @ Hinv @ (eye - rho * np.outer(y, s)) + rho * np.outer(s, s)
        x, E, g = x1, E1, g1
    return x.reshape(-1, 3), E, g.reshape(-1, 3), it


def verlet(xyz, vel, masses, dt: float, nsteps: int, orb, aux, **kw):
    """Velocity Verlet; returns positions [nsteps+1][natom][3], velocities, potential energies."""
    x = np.array(xyz, np.float64)
    v = np.array(vel, np.float64)
    mass = np.asarray(masses, np.float64)[:, None]
    E, g, _ = converged_point(x, orb, aux, **kw)
    a = -g / mass
    xs, vs, Es = [x.copy()], [v.copy()], [E]
    for _ in range(nsteps):
        x = x + v * dt + 0.5 * a * dt * dt
        E, g, _ = converged_point(x, orb, aux, **kw)
        a1 = -g / mass
        v = v + 0.5 * (a + a1) * dt
        a = a1
        xs.append(x.copy()); vs.append(v.copy()); Es.append(E)
    return np.array(xs), np.array(vs), np.array(Es)
