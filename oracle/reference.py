"""Brute-force validators for tiny systems (oracle; test infrastructure only).

These give the oracle something other than itself to be checked against:
  * rhf_energy_ao: the closed-shell Hartree-Fock energy written in the AO basis with the
    density D = C_occ C_occ^T. When every strong orbital has n = 1 and every weak one n = 0
    the cumulant of the paper's 2RDM expansion vanishes and Eq. PNOF must reduce to it.
  * fci_two_electron: exact ground-state energy of two electrons in n orbitals by full
    diagonalisation over ordered orbital pairs (the ground state is the spatially symmetric
    singlet). The paper notes that all PNOFs coincide for two-electron systems.
  * doci_two_orbital: the 2 x 2 pair-excitation problem for one pair in two orbitals.
  * lowdin: S^{-1/2} by symmetric eigendecomposition, for orthonormal starting orbitals.
"""
from __future__ import annotations

import numpy as np


def lowdin(S: np.ndarray) -> np.ndarray:
    w, U = np.linalg.eigh(S)
    return (U / np.sqrt(w)) @ U.T


def orthonormal_orbitals(S: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """C = S^{-1/2} Q: S-orthonormal for any orthogonal Q."""
    return lowdin(S) @ Q


def core_guess(S: np.ndarray, H: np.ndarray) -> np.ndarray:
    X = lowdin(S)
    w, U = np.linalg.eigh(X.T @ H @ X)
    return X @ U


def rhf_energy_ao(B, H, C, nocc: int, vnn: float) -> float:
    """E = 2 tr(D H) + 2 sum_P (tr D B^P)^2 - sum_P tr(D B^P D B^P) + V_nn."""
    Co = C[:, :nocc]
    D = Co @ Co.T
    e1 = 2.0 * np.sum(D * H)
    tP = np.einsum("mn,Pmn->P", D, B)
    coul = 2.0 * np.sum(tP * tP)
    DB = np.einsum("ml,Pln->Pmn", D, B)
    exch = np.einsum("Pmn,Pnm->", DB, DB)
    return e1 + coul - exch + vnn


def mo_integrals(eri_ao: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(ij|kl) in the orbital basis from (mu nu|lam sig) in the AO basis."""
    return np.einsum("abcd,ai,bj,ck,dl->ijkl", eri_ao, C, C, C, C, optimize=True)


def fci_two_electron(h_mo: np.ndarray, eri_mo: np.ndarray) -> float:
    """Lowest eigenvalue of h(1) + h(2) + 1/r12 over ordered pairs (i, j)."""
    n = h_mo.shape[0]
    I = np.eye(n)
    Hm = np.einsum("ik,jl->ijkl", h_mo, I) + np.einsum("ik,jl->ijkl", I, h_mo) \
        + np.einsum("ikjl->ijkl", eri_mo)
    w = np.linalg.eigvalsh(Hm.reshape(n * n, n * n))
    return float(w[0])


def doci_two_orbital(h11, h22, J11, J22, K12) -> float:
    M = np.array([[2.0 * h11 + J11, K12], [K12, 2.0 * h22 + J22]])
    return float(np.linalg.eigvalsh(M)[0])
