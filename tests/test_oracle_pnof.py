"""Pins of the oracle's pairing, occupations, energy and gradients (no GPU)."""
import numpy as np
import pytest

from oracle import integrals, pnof, reference, ri, step
from paper_2512_13550_gb300 import inputs


def _system(natom=4, spacing=1.8, basis=None):
    orb, aux = basis if basis is not None else inputs.basis_h4()
    xyz = inputs.chain(natom, spacing)
    S, T, V = integrals.one_electron(orb, xyz)
    B = ri.fitted_B(orb, aux, xyz)
    return S, T + V, B, integrals.nuclear_repulsion(xyz)


def test_pair_map_fig1_example():
    # Fig. 1: six paired electrons (three subspaces), N_g = 2, in 9 orbitals
    pm = pnof.PairMap(6, 2, 9)
    assert pm.nact == 9 and pm.ngamma == 6
    # strong orbitals 0,1,2; subspace 0 takes the top orbital of each weak block
    assert [pm.weak_orbital(0, i) for i in (1, 2)] == [5, 8]
    assert [pm.weak_orbital(2, i) for i in (1, 2)] == [3, 6]
    assert sorted(np.concatenate([np.flatnonzero(pm.pair == g) for g in range(3)])) == list(range(9))


def test_pair_map_ng1_is_homo_lumo_pairing():
    pm = pnof.PairMap(8, 1, 10)
    assert [pm.weak_orbital(g, 1) for g in range(4)] == [7, 6, 5, 4]
    with pytest.raises(ValueError):
        pnof.PairMap(8, 2, 10)


@pytest.mark.parametrize("ncwo", [1, 2, 3])
def test_sum_rule_trace_bounds(ncwo):
    npair = 3
    pm = pnof.PairMap(2 * npair, ncwo, npair * (ncwo + 1) + 2)
    for seed in range(5):
        gam = inputs.uniform(100 + seed, pm.ngamma, -3.0, 3.0)
        n = pnof.occupation_numbers(gam, pm)
        assert np.all(n >= 0) and np.all(n <= 1)
        for g in range(npair):
            assert abs(np.sum(n[pm.pair == g]) - 1.0) < 1e-15
        assert abs(2 * np.sum(n) - 2 * npair) < 1e-13
        assert np.all(n[:npair] >= 0.5)   # trig mapping keeps n_g >= 1/2


def test_jk_invariants():
    S, H, B, vnn = _system()
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(4, 0))
    J, K = pnof.jk(B, C, 4)
    np.testing.assert_allclose(np.diag(J), np.diag(K), rtol=0, atol=1e-14)
    np.testing.assert_allclose(J, J.T, atol=1e-14)
    np.testing.assert_allclose(K, K.T, atol=1e-14)
    assert np.all(K >= 0)
    assert np.linalg.eigvalsh(J)[0] > -1e-12
    assert np.all(K <= np.sqrt(np.outer(np.diag(J), np.diag(J))) + 1e-14)
    # brute force: contract the fitted 4-index tensor with C
    eri = reference.mo_integrals(ri.fitted_eri(B), C)
    np.testing.assert_allclose(J, np.einsum("ppqq->pq", eri), atol=1e-13)
    np.testing.assert_allclose(K, np.einsum("pqpq->pq", eri), atol=1e-13)


def test_jk_invariant_under_aux_mixing():
    S, H, B, vnn = _system()
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(4, 0))
    O = inputs.random_orthogonal(B.shape[0], 9)
    B2 = np.einsum("PQ,Qmn->Pmn", O, B)
    for x, y in zip(pnof.jk(B, C, 4), pnof.jk(B2, C, 4)):
        np.testing.assert_allclose(x, y, atol=1e-13)


def test_rhf_limit():
    S, H, B, vnn = _system()
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(4, 0))
    pm = pnof.PairMap(4, 1, 4)
    e = pnof.energy(B, H, C, np.zeros(pm.ngamma), pm, vnn)
    assert abs(e - reference.rhf_energy_ao(B, H, C, 2, vnn)) < 1e-12


def test_brillouin_at_rhf_limit():
    """At n in {0,1}, g_ov = -4 F_vo with F = H + 2J[D] - K[D] built in AO form."""
    S, H, B, vnn = _system()
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(4, 3))
    pm = pnof.PairMap(4, 1, 4)
    lam = pnof.lagrangian(B, H, C, np.zeros(pm.ngamma), pm)
    g = pnof.orbital_gradient(lam)
    D = C[:, :2] @ C[:, :2].T
    F = H + 2 * np.einsum("P,Pmn->mn", np.einsum("ls,Pls->P", D, B), B) \
        - np.einsum("Pml,ls,Psn->mn", B, D, B)
    Fmo = C.T @ F @ C
    np.testing.assert_allclose(g[:2, 2:], -4 * Fmo[2:, :2].T, atol=1e-12)


def test_two_electron_doci_and_fci():
    """H2/STO-3G: min over gamma of PNOF7 at the symmetry orbitals = 2x2 DOCI = full CI."""
    orb = inputs.Basis([inputs.sto3g_like_shell(1.24)])
    xyz = inputs.chain(2, 1.4)
    S, T, V = integrals.one_electron(orb, xyz)
    H = T + V
    eri = integrals.four_center(orb, xyz)
    # exact 4-index ERIs written as a rank-revealing B (eigendecomposition of the supermatrix)
    w, U = np.linalg.eigh(eri.reshape(4, 4))
    B = (U[:, w > 1e-12] * np.sqrt(w[w > 1e-12])).T.reshape(-1, 2, 2)
    vnn = integrals.nuclear_repulsion(xyz)
    C = reference.core_guess(S, H)
    pm = pnof.PairMap(2, 1, 2)
    from scipy.optimize import minimize_scalar
    res = minimize_scalar(lambda g: pnof.energy(B, H, C, np.array([g]), pm, vnn),
                          bounds=(0.0, 1.5), method="bounded", options={"xatol": 1e-12})
    hmo = C.T @ H @ C
    J, K = pnof.jk(B, C, 2)
    doci = reference.doci_two_orbital(hmo[0, 0], hmo[1, 1], J[0, 0], J[1, 1], K[0, 1]) + vnn
    fci = reference.fci_two_electron(hmo, reference.mo_integrals(eri, C)) + vnn
    assert abs(res.fun - doci) < 1e-10
    assert abs(doci - fci) < 1e-12
    assert abs(fci - (-1.1373)) < 1e-4          # textbook minimal-basis H2 full CI
    # one pair: PNOF7 and PNOF5 coincide
    g = np.array([res.x])
    assert abs(pnof.energy(B, H, C, g, pm, vnn, 7) - pnof.energy(B, H, C, g, pm, vnn, 5)) < 1e-15


@pytest.mark.slow
def test_two_electron_full_loop_reaches_fci():
    """The paper notes that all PNOFs coincide for two electrons: with N_g = n - 1 the full
    ON/NO loop must reach the two-electron full-CI energy of the same RI integrals."""
    orb = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, 2))
    aux = inputs.Basis(inputs.even_tempered_shells(0.1, 3.0, 8))
    xyz = inputs.chain(2, 1.4)
    S, T, V = integrals.one_electron(orb, xyz)
    H = T + V
    vnn = integrals.nuclear_repulsion(xyz)
    B = ri.fitted_B(orb, aux, xyz)
    C0 = reference.core_guess(S, H)
    fci = reference.fci_two_electron(C0.T @ H @ C0, reference.mo_integrals(ri.fitted_eri(B), C0)) + vnn
    pm = pnof.PairMap(2, 3, 4)
    st = step.State(C0, np.full(pm.ngamma, 0.3))
    for _ in range(600):
        E, gn, _ = step.step(B, H, vnn, st, pm, lr=0.01)
    assert abs(E - fci) < 1e-8 and gn < 1e-6


@pytest.mark.parametrize("ipnof,ncwo", [(7, 1), (5, 1), (7, 2)])
def test_gradients_match_finite_differences(ipnof, ncwo):
    natom = 4
    nb = 2 if ncwo == 2 else 1
    orb = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, nb)) if nb == 2 else None
    basis = (orb, inputs.basis_h4()[1]) if orb is not None else None
    S, H, B, vnn = _system(natom, basis=basis)
    n = S.shape[0]
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 0))
    pm = pnof.PairMap(natom, ncwo, n)
    gam = inputs.random_gamma(pm.ngamma, 1)
    r = pnof.energy_and_gradients(B, H, C, gam, pm, vnn, ipnof)
    np.testing.assert_allclose(r["g"], -r["g"].T, atol=1e-14)
    eps = 1e-4
    for p in range(n):
        for q in range(p + 1, n):
            y = np.zeros((n, n)); y[p, q] = eps; y[q, p] = -eps
            ep = pnof.energy(B, H, C @ step.expm_antisym(y), gam, pm, vnn, ipnof)
            em = pnof.energy(B, H, C @ step.expm_antisym(-y), gam, pm, vnn, ipnof)
            assert abs((ep - em) / (2 * eps) - r["g"][p, q]) < 1e-7 * max(1.0, abs(r["g"][p, q]))
    for k in range(pm.ngamma):
        e = np.zeros(pm.ngamma); e[k] = 1e-5
        fd = (pnof.energy(B, H, C, gam + e, pm, vnn, ipnof) - pnof.energy(B, H, C, gam - e, pm, vnn, ipnof)) / 2e-5
        assert abs(fd - r["g_gamma"][k]) < 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------------------
# softmax ON mapping (isoftmax = 1)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("ncwo", [1, 2, 3])
def test_softmax_sum_rule_and_trace(ncwo):
    npair = 3
    pm = pnof.PairMap(2 * npair, ncwo, npair * (ncwo + 1) + 2, isoftmax=1)
    for seed in range(5):
        gam = inputs.uniform(200 + seed, pm.ngamma, -4.0, 4.0)
        n = pnof.occupation_numbers(gam, pm)
        assert np.all(n > 0) and np.all(n < 1)
        for g in range(npair):
            assert abs(np.sum(n[pm.pair == g]) - 1.0) < 1e-15
        assert abs(2 * np.sum(n) - 2 * npair) < 1e-13
        s, t, _, _ = pnof.occupations(gam, pm)
        np.testing.assert_allclose(s * s + t * t, 1.0, atol=1e-15)


def test_softmax_one_weak_orbital_is_the_logistic_function():
    """N_g = 1: n_p = exp(x) / (1 + exp(x)) is the logistic function (scipy's expit), n_g its
    complement; a positive variable puts more than half the pair's electrons in the weak orbital
    (the mapping does not keep n_g >= 1/2)."""
    from scipy.special import expit
    pm = pnof.PairMap(6, 1, 6, isoftmax=1)
    gam = np.array([-2.5, 0.0, 1.75])
    n = pnof.occupation_numbers(gam, pm)
    for g in range(3):
        p = pm.weak_orbital(g, 1)
        assert abs(n[p] - expit(gam[g])) < 1e-15
        assert abs(n[g] - expit(-gam[g])) < 1e-15
    assert n[2] < 0.5


@pytest.mark.parametrize("ncwo", [1, 2])
def test_softmax_and_trigonometric_agree_at_equal_occupations(ncwo):
    """Both mappings reach the same occupations (x_i = ln(n_{p_i} / n_g)); the energy and the
    orbital gradient then agree, and dE/dx follows from dE/dgamma_trig through the Jacobians:
    dE/dn restricted to the sum-rule surface is the same whichever variables describe it."""
    natom = 4
    nb = 2 if ncwo == 2 else 1
    orb = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, nb)) if nb == 2 else None
    basis = (orb, inputs.basis_h4()[1]) if orb is not None else None
    S, H, B, vnn = _system(natom, basis=basis)
    n_bf = S.shape[0]
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n_bf, 5))
    pm_t = pnof.PairMap(natom, ncwo, n_bf)
    pm_s = pnof.PairMap(natom, ncwo, n_bf, isoftmax=1)
    gam_t = inputs.random_gamma(pm_t.ngamma, 6)
    n = pnof.occupation_numbers(gam_t, pm_t)
    x = np.zeros(pm_s.ngamma)
    for g in range(pm_s.npair):
        for i in range(1, ncwo + 1):
            x[(i - 1) * pm_s.npair + g] = np.log(n[pm_s.weak_orbital(g, i)] / n[g])
    np.testing.assert_allclose(pnof.occupation_numbers(x, pm_s), n, atol=1e-15)
    rt = pnof.energy_and_gradients(B, H, C, gam_t, pm_t, vnn)
    rs = pnof.energy_and_gradients(B, H, C, x, pm_s, vnn)
    assert abs(rt["E"] - rs["E"]) < 1e-12
    np.testing.assert_allclose(rs["g"], rt["g"], atol=1e-12)
    # chain rule check: with dn/dgamma (trig) and dn/dx (softmax) both spanning the sum-rule
    # tangent space, dE/dx = (dn/dx)^T G and dE/dgamma = (dn/dgamma)^T G for one G
    def dn(gam, pm):
        s, _, ds, _ = pnof.occupations(gam, pm)
        return 2.0 * s[:, None] * ds
    Jt, Js = dn(gam_t, pm_t), dn(x, pm_s)
    G, *_ = np.linalg.lstsq(Jt.T, rt["g_gamma"], rcond=None)
    np.testing.assert_allclose(Js.T @ G, rs["g_gamma"], atol=1e-10)


@pytest.mark.parametrize("ipnof,ncwo", [(7, 1), (5, 1), (7, 2)])
def test_softmax_gradients_match_finite_differences(ipnof, ncwo):
    natom = 4
    nb = 2 if ncwo == 2 else 1
    orb = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, nb)) if nb == 2 else None
    basis = (orb, inputs.basis_h4()[1]) if orb is not None else None
    S, H, B, vnn = _system(natom, basis=basis)
    n = S.shape[0]
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 0))
    pm = pnof.PairMap(natom, ncwo, n, isoftmax=1)
    gam = inputs.uniform(7, pm.ngamma, -2.0, 1.0)
    r = pnof.energy_and_gradients(B, H, C, gam, pm, vnn, ipnof)
    for k in range(pm.ngamma):
        e = np.zeros(pm.ngamma); e[k] = 1e-5
        fd = (pnof.energy(B, H, C, gam + e, pm, vnn, ipnof) - pnof.energy(B, H, C, gam - e, pm, vnn, ipnof)) / 2e-5
        assert abs(fd - r["g_gamma"][k]) < 1e-7 * max(1.0, abs(fd))
