"""Density-fitted (RI) three-index tensor (oracle; test infrastructure only).

The paper's default ERITYP='RI' replaces the four-index integrals by a resolution of the
identity, which lowers the orbital transformation to fourth order (Single Point Energy
section). The paper does not name the metric; this oracle reads it as Coulomb-metric fitting,

    (mu nu|lam sig) ~= sum_P B^P_{mu nu} B^P_{lam sig},   B^P = sum_Q (V^{-1/2})_{PQ} (Q|mu nu),

with V_PQ = (P|Q) and V^{-1/2} from a symmetric eigendecomposition (a library routine used
as one step). Any other square root of V^{-1} (e.g. a Cholesky factor) gives the same fitted
four-index tensor, so parity is checked on that tensor and everything downstream, never on B.
If the metric's smallest eigenvalue is below 1e-12 of its largest the fit is refused rather
than truncated.

Parity: pinned by the exactness of the fit when the aux set spans all orbital products, by
the variational property (pq|pq)_RI <= (pq|pq), and by J/K invariance under orthogonal
mixing of the aux index.
"""
from __future__ import annotations

import numpy as np

from . import integrals


class IllConditioned(ValueError):
    pass


def inverse_sqrt_metric(V: np.ndarray, rcond: float = 1e-12) -> np.ndarray:
    w, U = np.linalg.eigh(V)
    if w[0] < rcond * w[-1]:
        raise IllConditioned(f"metric eigenvalue ratio {w[0] / w[-1]:.3e} below {rcond}")
    return (U / np.sqrt(w)) @ U.T


def fitted_B(orb, aux, xyz) -> np.ndarray:
    """B [X][n][n] for the given geometry and basis pair."""
    V = integrals.two_center(aux, xyz)
    M = integrals.three_center(orb, aux, xyz)
    X, n, _ = M.shape
    return (inverse_sqrt_metric(V) @ M.reshape(X, n * n)).reshape(X, n, n)


def fitted_eri(B: np.ndarray) -> np.ndarray:
    """sum_P B^P_{mu nu} B^P_{lam sig} as an n^4 array (tiny systems)."""
    return np.einsum("Pij,Pkl->ijkl", B, B)
