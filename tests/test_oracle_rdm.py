"""Pins of the PNOF energy bookkeeping through the reconstructed 2RDM (no GPU).

The energy of Eq. (PNOF) as pnof.py assembles it from its A and B coefficients must equal the
contraction of the spin-orbital 2RDM of the Theory section's cumulant expansion (oracle/rdm.py,
every element written out from the printed Delta/Pi structure) with the two-electron integrals,
Eq. (Energy). The 2RDM itself is pinned by brute force (two electrons: the exact 2RDM of the pair
wavefunction from fermion operators) and by Loewdin's normalisation and partial-trace relation.
"""
import numpy as np
import pytest

from oracle import integrals, pnof, rdm, reference, ri
from paper_2512_13550_gb300 import inputs


@pytest.mark.parametrize("ncwo", [1, 2, 3])
def test_one_pair_reconstruction_is_the_pair_wavefunction_2rdm(ncwo):
    """Two electrons in one subspace: the cumulant reconstruction equals the exact 2RDM of
    Psi = sum_p c_p |p alpha p beta> with c_p = +-sqrt(n_p) (strong +, weak -), built by applying
    a+ a+ a a to determinants, for PNOF5 and PNOF7 alike (no second subspace)."""
    a = ncwo + 1
    pm = pnof.PairMap(2, ncwo, a)
    for seed in range(3):
        gam = inputs.uniform(300 + seed, pm.ngamma, 0.05, 1.5)
        for ipnof in (5, 7):
            n, Delta, Pi = rdm.delta_pi(gam, pm, ipnof)
            D = rdm.spin_orbital_2rdm(n, Delta, Pi)
            coef = np.where(pm.strong, np.sqrt(n), -np.sqrt(n))
            Dbf = rdm.pair_state_2rdm(coef, a)
            np.testing.assert_allclose(D, Dbf, rtol=0, atol=1e-15)


@pytest.mark.parametrize("npair,ncwo", [(2, 1), (3, 1), (2, 2)])
@pytest.mark.parametrize("ipnof", [5, 7])
def test_loewdin_normalisation_and_partial_trace(npair, ncwo, ipnof):
    """Tr D = N(N - 1)/2 and sum_j D_ij,kj = (N - 1)/2 Gamma_ik for random occupations."""
    N = 2 * npair
    pm = pnof.PairMap(N, ncwo, npair * (ncwo + 1))
    gam = inputs.uniform(400 + N + ncwo, pm.ngamma, -2.0, 2.0)
    n, Delta, Pi = rdm.delta_pi(gam, pm, ipnof)
    D = rdm.spin_orbital_2rdm(n, Delta, Pi)
    assert abs(rdm.loewdin_trace(D) - N * (N - 1) / 2) < 1e-13
    Gamma = np.diag(np.repeat(n, 2))  # spin orbital 2p + s has occupation n_p
    np.testing.assert_allclose(rdm.partial_trace(D), (N - 1) / 2 * Gamma, rtol=0, atol=1e-14)
    # antisymmetry and hermiticity of the assembled object
    np.testing.assert_allclose(D, -D.transpose(1, 0, 2, 3), atol=1e-15)
    np.testing.assert_allclose(D, -D.transpose(0, 1, 3, 2), atol=1e-15)
    np.testing.assert_allclose(D, D.transpose(2, 3, 0, 1), atol=1e-15)


def _mo(basis, natom, seed, fitted):
    orb, aux = basis
    xyz = inputs.chain(natom, 1.8)
    S, T, V = integrals.one_electron(orb, xyz)
    n = S.shape[0]
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, seed))
    eri_ao = ri.fitted_eri(ri.fitted_B(orb, aux, xyz)) if fitted else integrals.four_center(orb, xyz)
    return C.T @ (T + V) @ C, reference.mo_integrals(eri_ao, C), integrals.nuclear_repulsion(xyz), n


@pytest.mark.parametrize("case", [
    ("H4 STO-3G-like, exact ERIs", inputs.basis_h4, 4, 1, False),
    ("H4 STO-3G-like, RI", inputs.basis_h4, 4, 1, True),
    ("H6 3s, RI, N_g = 2", inputs.basis_3s_10aux, 6, 2, True),
    ("H8 STO-3G-like, exact ERIs", inputs.basis_h4, 8, 1, False),
])
@pytest.mark.parametrize("ipnof", [5, 7])
def test_energy_from_2rdm_equals_pnof_energy(case, ipnof):
    """Eq. (Energy) with the reconstructed 2RDM equals Eq. (PNOF) with pnof.py's A and B, on the
    same integrals (J_pq = (pp|qq), K_pq = (pq|pq)), for random orbitals and occupations."""
    _, basis, natom, ncwo, fitted = case
    h_mo, eri_mo, vnn, nbf = _mo(basis(), natom, 11, fitted)
    pm = pnof.PairMap(natom, ncwo, nbf)
    a = pm.nact
    J = np.einsum("ppqq->pq", eri_mo[:a, :a, :a, :a])
    K = np.einsum("pqpq->pq", eri_mo[:a, :a, :a, :a])
    for seed in (1, 2):
        gam = inputs.random_gamma(pm.ngamma, seed)
        n, Delta, Pi = rdm.delta_pi(gam, pm, ipnof)
        D = rdm.spin_orbital_2rdm(n, Delta, Pi)
        E2 = rdm.energy_from_2rdm(h_mo[:a, :a], eri_mo[:a, :a, :a, :a], n, D, vnn)
        Ejk = pnof.energy_from_jk(np.diag(h_mo)[:a], J, K, gam, pm, vnn, ipnof)
        assert abs(E2 - Ejk) < 1e-12 * max(1.0, abs(Ejk))


def test_inter_pair_term_is_seen_by_the_2rdm_route():
    """The PNOF7 and PNOF5 energies differ by exactly the inter-subspace Pi term,
    -sum_{p, q in different subspaces} Phi_p Phi_q K_pq, on both routes (so a dropped or
    sign-flipped Phi term in the A/B bookkeeping would fail the equality test above)."""
    h_mo, eri_mo, vnn, nbf = _mo(inputs.basis_h4(), 4, 3, True)
    pm = pnof.PairMap(4, 1, nbf)
    a = pm.nact
    K = np.einsum("pqpq->pq", eri_mo[:a, :a, :a, :a])
    J = np.einsum("ppqq->pq", eri_mo[:a, :a, :a, :a])
    gam = inputs.random_gamma(pm.ngamma, 5)
    n = pnof.occupation_numbers(gam, pm)
    phi = np.sqrt(n * (1 - n))
    diff = ~pm.same
    term = -np.sum(np.where(diff, np.outer(phi, phi) * K, 0.0))
    assert abs(term) > 1e-4
    e7 = pnof.energy_from_jk(np.diag(h_mo)[:a], J, K, gam, pm, vnn, 7)
    e5 = pnof.energy_from_jk(np.diag(h_mo)[:a], J, K, gam, pm, vnn, 5)
    assert abs((e7 - e5) - term) < 1e-13
    D7 = rdm.spin_orbital_2rdm(*rdm.delta_pi(gam, pm, 7))
    D5 = rdm.spin_orbital_2rdm(*rdm.delta_pi(gam, pm, 5))
    d2 = rdm.energy_from_2rdm(h_mo[:a, :a], eri_mo[:a, :a, :a, :a], n, D7, 0.0) - \
        rdm.energy_from_2rdm(h_mo[:a, :a], eri_mo[:a, :a, :a, :a], n, D5, 0.0)
    assert abs(d2 - term) < 1e-13
