"""The reconstructed two-particle density matrix of the PNOF functionals, element by element
(oracle; test infrastructure only).

This is a second route to the energy of Eq. (PNOF), independent of the A/B coefficient
bookkeeping in pnof.py. It assembles the 2RDM over spin orbitals and contracts it with the
two-electron integrals as in Eq. (Energy) of the Theory section,

    E = sum_ik Gamma_ik h_ki + sum_ijkl D_ijkl <kl|ij>,

in Loewdin's normalisation (the trace of D is the number of electron pairs N(N-1)/2). The 2RDM
is the cumulant expansion printed in the Theory section,

    D_ijkl = (n_i n_j / 2) (delta_ik delta_jl - delta_il delta_jk) + lambda_ijkl,

with the spin-restricted cumulant of the (2,2)-positivity reconstruction written in terms of two
auxiliary matrices Delta and Pi (same section, spatial orbitals p, q, r, t):

    lambda^{ss}_{pq,rt} = -(Delta_pq / 2) (delta_pr delta_qt - delta_pt delta_qr),  s = alpha, beta
    lambda^{ab}_{pq,rt} = -(Delta_pq / 2) delta_pr delta_qt + (Pi_pr / 2) delta_pq delta_rt.

The other spin orderings follow from the antisymmetry D_ijkl = -D_ijlk = -D_jikl. The paper
defers Delta and Pi to the publications of each functional. Reading (the electron-pairing
functionals over the subspaces Omega_g of Eq. OmegaG):

    Delta_pp = n_p^2;  Delta_pq = n_p n_q for p != q in one subspace;  0 across subspaces;
    Pi_pp = n_p;  Pi_pq = c_p c_q for p != q in one subspace (c_p = +sqrt(n_p) for the strong
    orbital, -sqrt(n_p) for a weak one);  across subspaces Pi_pq = -Phi_p Phi_q for PNOF7
    (Phi_p = sqrt(n_p (1 - n_p))) and 0 for PNOF5.

Parity: pinned by brute force. For two electrons in one subspace the reconstruction is the
exact 2RDM of the pair wavefunction sum_p c_p |p alpha p beta>, which `pair_state_2rdm` computes
from fermion operators acting on determinants. The Loewdin trace and the contraction
sum_j D_ij,kj = (N - 1)/2 Gamma_ik hold for any occupations. The value of the inter-subspace
term -Phi_p Phi_q itself is the PNOF7 reading above (parity unpinned as to that value).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import pnof


def delta_pi(gamma, pm: pnof.PairMap, ipnof: int = 7):
    """Occupations n and the auxiliary matrices Delta and Pi (nact x nact) of the reading above."""
    n = pnof.occupation_numbers(gamma, pm)
    a = pm.nact
    c = np.where(pm.strong, np.sqrt(n), -np.sqrt(n))
    phi = np.sqrt(n * (1.0 - n))
    Delta = np.zeros((a, a))
    Pi = np.zeros((a, a))
    for p in range(a):
        for q in range(a):
            if p == q:
                Delta[p, q] = n[p] * n[p]
                Pi[p, q] = n[p]
            elif pm.pair[p] == pm.pair[q]:
                Delta[p, q] = n[p] * n[q]
                Pi[p, q] = c[p] * c[q]
            elif ipnof == 7:
                Pi[p, q] = -phi[p] * phi[q]
            elif ipnof != 5:
                raise ValueError("only PNOF5 and PNOF7 are defined here")
    return n, Delta, Pi


def spin_orbital_2rdm(n, Delta, Pi):
    """D[i, j, k, l] over spin orbitals i = 2 p + s (s = 0 alpha, 1 beta) from the cumulant
    expansion, every element written out from the formulas in the module header."""
    a = len(n)
    m = 2 * a
    D = np.zeros((m, m, m, m))

    def dl(x, y):
        return 1.0 if x == y else 0.0

    for i, j, k, l in itertools.product(range(m), repeat=4):
        p, si = divmod(i, 2)
        q, sj = divmod(j, 2)
        r, sk = divmod(k, 2)
        t, sl = divmod(l, 2)
        # Hartree-Fock part over spin orbitals (occupation n_p for both spins)
        hf = 0.5 * n[p] * n[q] * (dl(i, k) * dl(j, l) - dl(i, l) * dl(j, k))
        cum = 0.0
        if si == sj == sk == sl:  # same-spin block
            cum = -0.5 * Delta[p, q] * (dl(p, r) * dl(q, t) - dl(p, t) * dl(q, r))
        elif si == sk and sj == sl and si != sj:  # (p s, q s' | r s, t s'): the printed block
            cum = -0.5 * Delta[p, q] * dl(p, r) * dl(q, t) + 0.5 * Pi[p, r] * dl(p, q) * dl(r, t)
        elif si == sl and sj == sk and si != sj:  # exchanged order: minus the block at (l, k)
            cum = -(-0.5 * Delta[p, q] * dl(p, t) * dl(q, r) + 0.5 * Pi[p, t] * dl(p, q) * dl(t, r))
        D[i, j, k, l] = hf + cum
    return D


def spin_orbital_eri(eri_mo):
    """<kl|ij> over spin orbitals as G[k, l, i, j] = (k i | l j) delta_{s_k s_i} delta_{s_l s_j},
    from the chemists' spatial integrals (p q | r s) (real orbitals)."""
    a = eri_mo.shape[0]
    m = 2 * a
    G = np.zeros((m, m, m, m))
    for k, l, i, j in itertools.product(range(m), repeat=4):
        pk, sk = divmod(k, 2)
        pl, sl = divmod(l, 2)
        pi, si = divmod(i, 2)
        pj, sj = divmod(j, 2)
        if sk == si and sl == sj:
            G[k, l, i, j] = eri_mo[pk, pi, pl, pj]
    return G


def energy_from_2rdm(h_mo, eri_mo, n, D, vnn: float) -> float:
    """Eq. (Energy) with the 1RDM diagonal in the natural orbitals (Gamma_ii = n_i for each spin):
    sum_i n_i h_ii + sum_ijkl D_ijkl <kl|ij> + V_nn."""
    G = spin_orbital_eri(eri_mo)
    one = 2.0 * float(np.dot(n, np.diag(h_mo)[: len(n)]))
    two = float(np.einsum("ijkl,klij->", D, G))
    return one + two + vnn


def loewdin_trace(D) -> float:
    """sum_ij D_ij,ij (the number of electron pairs in Loewdin's normalisation)."""
    m = D.shape[0]
    return float(sum(D[i, j, i, j] for i in range(m) for j in range(m)))


def partial_trace(D):
    """sum_j D_ij,kj over spin orbitals (equals (N - 1)/2 Gamma_ik for an N-electron 2RDM)."""
    return np.einsum("ijkj->ik", D)


# ---- brute force: the 2RDM of an explicit two-electron state ----------------------------------
def _apply_annihilate(det: int, i: int):
    """a_i |det>: (sign, new det) or None; orbitals ordered by index, sign from the occupied
    orbitals before i."""
    if not (det >> i) & 1:
        return None
    sign = -1.0 if bin(det & ((1 << i) - 1)).count("1") % 2 else 1.0
    return sign, det & ~(1 << i)


def _apply_create(det: int, i: int):
    if (det >> i) & 1:
        return None
    sign = -1.0 if bin(det & ((1 << i) - 1)).count("1") % 2 else 1.0
    return sign, det | (1 << i)


def pair_state_2rdm(coef, nspatial: int):
    """D_ijkl = (1/2) <Psi| a+_i a+_j a_l a_k |Psi> for Psi = sum_p coef[p] a+_{p alpha} a+_{p beta}
    |0> (spin orbital i = 2 p + s), by applying the operators to every determinant."""
    m = 2 * nspatial
    psi = {}
    for p, cp in enumerate(coef):
        if cp == 0.0:
            continue
        # a+_{p alpha} a+_{p beta} |0>: create beta first, then alpha
        s1, d1 = _apply_create(0, 2 * p + 1)
        s2, d2 = _apply_create(d1, 2 * p)
        psi[d2] = psi.get(d2, 0.0) + cp * s1 * s2
    D = np.zeros((m, m, m, m))
    for i, j, k, l in itertools.product(range(m), repeat=4):
        acc = 0.0
        for det, cv in psi.items():
            r = _apply_annihilate(det, k)
            if r is None:
                continue
            s, d = r
            r = _apply_annihilate(d, l)
            if r is None:
                continue
            s *= r[0]
            d = r[1]
            r = _apply_create(d, j)
            if r is None:
                continue
            s *= r[0]
            d = r[1]
            r = _apply_create(d, i)
            if r is None:
                continue
            s *= r[0]
            d = r[1]
            acc += psi.get(d, 0.0) * s * cv
        D[i, j, k, l] = 0.5 * acc
    return D
