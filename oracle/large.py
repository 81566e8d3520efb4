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

The *_blocked / *_inplace variants compute the same quantities with the aux index taken a block at a
time, so that the only array of size X n a is b itself (the H1000 chain: 24 GB in FP64).

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


def fit_inplace(Q3, V, cols: int = 1 << 18):
    """b^P_{qp} = sum_Q (V^{-1/2})_{PQ} (Q|q p) written over the stacked (Q|q p) [X][n][nact],
    a block of `cols` (q, p) columns at a time."""
    X = Q3.shape[0]
    flat = Q3.reshape(X, -1)
    W = ri.inverse_sqrt_metric(V)
    for c0 in range(0, flat.shape[1], cols):
        flat[:, c0:c0 + cols] = W @ flat[:, c0:c0 + cols]
    return Q3


def energy_and_gradients_mo_blocked(bfull, H, C, gamma, pm: pnof.PairMap, vnn: float, ipnof: int = 7,
                                    block: int = 32):
    """energy_and_gradients_mo with every sum over the aux index P taken `block` aux functions at a
    time (same definitions; only the order of the P sum differs)."""
    a = pm.nact
    n_bf = C.shape[0]
    X = bfull.shape[0]
    d = np.stack([np.diagonal(bfull[P, :a, :]) for P in range(X)])  # d^P_p = b^P_pp  [X][a]
    J = d.T @ d
    K = np.zeros((a, a))
    for P0 in range(0, X, block):
        b = bfull[P0:P0 + block, :a, :]
        K += np.einsum("Ppq,Ppq->pq", b, b)
    hmo = C.T @ H @ C[:, :a]
    hpp = np.diag(hmo[:a, :]).copy()
    E = pnof.energy_from_jk(hpp, J, K, gamma, pm, vnn, ipnof)
    A, Bc = pnof.coefficients(gamma, pm, ipnof)
    nocc = pnof.occupation_numbers(gamma, pm)
    D = d @ A.T
    lam = np.zeros((n_bf, n_bf))
    lam[:, :a] = hmo * nocc[None, :]
    for P0 in range(0, X, block):
        bf = bfull[P0:P0 + block]
        lam[:, :a] += np.einsum("Pqp,Pp->qp", bf, D[P0:P0 + block])
        Wt = Bc.T[None, :, :] * bf[:, :a, :]       # [P][r][p] = B_pr b^P_rp
        lam[:, :a] -= np.matmul(bf, Wt).sum(axis=0)
    return dict(E=E, J=J, K=K, hpp=hpp, lam=lam, g=pnof.orbital_gradient(lam),
                g_gamma=pnof.gamma_gradient(hpp, J, K, gamma, pm, ipnof))
