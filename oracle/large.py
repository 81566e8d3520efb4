"""PNOF energy, J, K and gradients for systems too large for the [X][n][n] route of pnof.py
(oracle; test infrastructure only).

The definitions are those of pnof.py: the JKL-only energy of Eq. (PNOF) with the PNOF7 pair
coefficients, the Lagrangian of the Natural Orbital Optimization subsection, and the
Coulomb-metric density fitting of the RI option (ERITYP='RI' in the Single Point Energy section).
Only the order of work differs, so that memory stays O(X n a) instead of O(X n^2):

* the three-centre integrals (P|mu nu) are generated a slice of aux functions at a time and
  transformed at once to the orbital basis, (P|q p) = sum_{mu nu} C_{mu q} (P|mu nu) C_{nu p},
  for every orbital q and every active orbital p;
* the fitted tensor in the orbital basis follows as b^P_{qp} = sum_Q (V^{-1/2})_{PQ} (Q|q p);
* lambda = C^T Lambda needs no atomic-orbital quantity once b is known for every q:
  lambda_{qp} = n_p h_{qp} + sum_P b^P_{qp} D^P_p - sum_{P, r} b^P_{qr} B_{pr} b^P_{rp},
  with h_{qp} = (C^T H C)_{qp}, d^P_p = b^P_{pp}, D^P = A d^P.

Parity: pinned against pnof.energy_and_gradients (itself pinned to closed forms, brute force and
finite differences) on small systems in tests/test_oracle_large.py.
"""
from __future__ import annotations

import numpy as np

from . import integrals, pnof, ri


def mo_three_center(orb, aux, xyz, C, nact, P_slice=None):
    """(P|q p) for the aux functions in P_slice, every orbital q and the active orbitals p:
    array [Ps][n][nact]."""
    M = integrals.three_center(orb, aux, xyz, P_slice)
    return np.matmul(C.T[None, :, :], np.matmul(M, C[:, :nact]))


def fitted_mo(Q3, V):
    """b^P_{qp} = sum_Q (V^{-1/2})_{PQ} (Q|q p) from the stacked (Q|q p) [X][n][nact]."""
    X, n, a = Q3.shape
    return (ri.inverse_sqrt_metric(V) @ Q3.reshape(X, n * a)).reshape(X, n, a)


def energy_and_gradients_mo(bfull, H, C, gamma, pm: pnof.PairMap, vnn: float, ipnof: int = 7):
    """Same outputs as pnof.energy_and_gradients from b^P_{qp} for all q (bfull [X][n][nact])."""
    a = pm.nact
    n_bf = C.shape[0]
    b = bfull[:, :a, :]
    d = np.einsum("Ppp->Pp", b)
    J = d.T @ d
    K = np.einsum("Ppq,Ppq->pq", b, b)
    hmo = C.T @ H @ C[:, :a]                        # h_{qp}, q all, p active
    hpp = np.diag(hmo[:a, :]).copy()
    E = pnof.energy_from_jk(hpp, J, K, gamma, pm, vnn, ipnof)
    A, Bc = pnof.coefficients(gamma, pm, ipnof)
    nocc = pnof.occupation_numbers(gamma, pm)
    D = d @ A.T                                     # D^P_p = sum_r A_pr d^P_r
    lam = np.zeros((n_bf, n_bf))
    lam[:, :a] = hmo * nocc[None, :]
    lam[:, :a] += np.einsum("Pqp,Pp->qp", bfull, D)
    # sum_{P, r} b^P_{qr} (B_{pr} b^P_{rp}): one (n x a)(a x a) product per P
    Wt = Bc.T[None, :, :] * b                       # [P][r][p] = B_pr b^P_rp
    lam[:, :a] -= np.matmul(bfull, Wt).sum(axis=0)
    return dict(E=E, J=J, K=K, hpp=hpp, lam=lam, g=pnof.orbital_gradient(lam),
                g_gamma=pnof.gamma_gradient(hpp, J, K, gamma, pm, ipnof))
