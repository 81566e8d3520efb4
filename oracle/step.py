"""Alternating ON / NO optimisation step (oracle; test infrastructure only).

The paper optimises the occupations and the orbitals separately (Theory section, after
Eq. sum1): the ONs through the unconstrained angles gamma of the trigonometric mapping, the
NOs by orbital rotation C^(i+1) = U C^(i), U = exp(y), y antisymmetric, driven by ADAM on the
orbital gradient g = 4(lambda - lambda^T) (Natural Orbital Optimization subsection). The ADAM
details are delegated to another publication, so this step is a reading (parity unpinned
as to its hyper-parameters; both the oracle and the GPU path implement exactly this):

  1. J, K, h_pp at the current C.
  2. ON update with J, K, h_pp fixed: `on_iters` steepest-descent steps
     gamma <- gamma - on_lr * dE/dgamma.
  3. E, lambda and g at (C, gamma_new) (same transformed tensors as step 1).
  4. ADAM (Kingma & Ba 2015, bias-corrected) on the antisymmetric g:
     m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g*g,
     y = -lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
  5. U = exp(y) by scaling and squaring (Taylor degree 12 on y / 2^s with ||y/2^s||_F <= 1/2),
     and C <- C U, the column-major (phi_p = sum_mu C_mu,p chi_mu) form of the paper's
     C^(i+1) = U C^(i).

Returned: the energy at (C, gamma_new), ||g||_F and max |lambda - lambda^T|.
"""
from __future__ import annotations

import numpy as np

from . import pnof


def expm_antisym(y: np.ndarray, degree: int = 12) -> np.ndarray:
    nrm = np.linalg.norm(y)
    s = 0
    while nrm / (2.0 ** s) > 0.5:
        s += 1
    z = y / (2.0 ** s)
    n = y.shape[0]
    U = np.eye(n)
    term = np.eye(n)
    for k in range(1, degree + 1):
        term = term @ z / k
        U = U + term
    for _ in range(s):
        U = U @ U
    return U


class State:
    def __init__(self, C, gamma):
        n = C.shape[0]
        self.C = np.array(C, np.float64)
        self.gamma = np.array(gamma, np.float64)
        self.m = np.zeros((n, n))
        self.v = np.zeros((n, n))
        self.t = 0


DEFAULTS = dict(lr=0.02, b1=0.9, b2=0.999, eps=1e-8, on_iters=20, on_lr=0.3)


def step(B, H, vnn, st: State, pm: pnof.PairMap, ipnof=7, **opt):
    o = dict(DEFAULTS); o.update(opt)
    a = pm.nact
    C = st.C
    J, K = pnof.jk(B, C, a)
    hpp = np.einsum("mp,mn,np->p", C[:, :a], H, C[:, :a])
    for _ in range(int(o["on_iters"])):
        st.gamma = st.gamma - o["on_lr"] * pnof.gamma_gradient(hpp, J, K, st.gamma, pm, ipnof)
    E = pnof.energy_from_jk(hpp, J, K, st.gamma, pm, vnn, ipnof)
    lam = pnof.lagrangian(B, H, C, st.gamma, pm, ipnof)
    g = pnof.orbital_gradient(lam)
    st.t += 1
    st.m = o["b1"] * st.m + (1.0 - o["b1"]) * g
    st.v = o["b2"] * st.v + (1.0 - o["b2"]) * g * g
    mh = st.m / (1.0 - o["b1"] ** st.t)
    vh = st.v / (1.0 - o["b2"] ** st.t)
    y = -o["lr"] * mh / (np.sqrt(vh) + o["eps"])
    st.C = C @ expm_antisym(y)
    return E, float(np.linalg.norm(g)), float(np.max(np.abs(lam - lam.T)))
