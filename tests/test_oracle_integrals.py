"""Pins of the oracle's integrals and RI fit against sources other than the oracle itself."""
import json
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import integrals, reference, ri
from paper_2512_13550_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g_r1.4.json")


@pytest.fixture(scope="module")
def h2():
    g = json.load(open(GOLD))
    orb = inputs.Basis([inputs.sto3g_like_shell(1.24)])
    xyz = inputs.chain(2, g["R_bohr"])
    S, T, V = integrals.one_electron(orb, xyz)
    eri = integrals.four_center(orb, xyz)
    return g, orb, xyz, S, T, V, eri


def test_h2_sto3g_textbook_integrals(h2):
    g, orb, xyz, S, T, V, eri = h2
    tol = g["tol"]
    assert abs(S[0, 1] - g["S12"]) < tol
    assert abs(T[0, 0] - g["T11"]) < tol and abs(T[0, 1] - g["T12"]) < tol
    assert abs(V[0, 0] - g["V11_total"]) < tol and abs(V[0, 1] - g["V12_total"]) < tol
    assert abs(eri[0, 0, 0, 0] - g["eri_1111"]) < tol
    assert abs(eri[0, 0, 1, 1] - g["eri_1122"]) < tol
    assert abs(eri[1, 0, 0, 0] - g["eri_2111"]) < tol
    assert abs(eri[1, 0, 1, 0] - g["eri_2121"]) < tol


def test_h2_sto3g_textbook_energies(h2):
    g, orb, xyz, S, T, V, eri = h2
    H = T + V
    vnn = integrals.nuclear_repulsion(xyz)
    C = reference.core_guess(S, H)
    D = C[:, :1] @ C[:, :1].T
    J = np.einsum("ls,mnls->mn", D, eri)
    K = np.einsum("ls,mlns->mn", D, eri)
    e_rhf = np.sum(D * (2 * H + 2 * J - K)) + vnn
    assert abs(e_rhf - g["E_RHF_total"]) < g["tol"]
    e_fci = reference.fci_two_electron(C.T @ H @ C, reference.mo_integrals(eri, C)) + vnn
    assert abs(e_fci - g["E_FCI_total"]) < g["tol"]


def test_boys_limits():
    assert integrals.boys_f0(np.array([0.0]))[0] == 1.0
    t = np.array([50.0, 200.0])
    np.testing.assert_allclose(integrals.boys_f0(t), 0.5 * np.sqrt(np.pi / t), rtol=1e-12)
    # continuity across the series / closed-form switch, and F0 = int_0^1 exp(-t u^2) du
    for tv in [1e-9, 1.1e-8, 1e-3, 0.7, 3.0]:
        q, _ = integrate.quad(lambda u: np.exp(-tv * u * u), 0.0, 1.0, epsabs=1e-15)
        assert abs(integrals.boys_f0(np.array([tv]))[0] - q) < 1e-13


def _gaussian_cloud_potential(a, r):
    """Potential of a unit-charge Gaussian cloud of exponent a by Gauss's law quadrature."""
    rho = lambda s: (a / np.pi) ** 1.5 * np.exp(-a * s * s)
    inner, _ = integrate.quad(lambda s: rho(s) * 4 * np.pi * s * s, 0, r, epsabs=1e-14)
    outer, _ = integrate.quad(lambda s: rho(s) * 4 * np.pi * s, r, np.inf, epsabs=1e-14)
    return inner / r + outer


def _cloud_interaction(a, b, R):
    """Interaction of unit Gaussian clouds (exponents a, b) at separation R by radial quadrature."""
    def avg(r):  # spherical average of cloud b (centred at distance R) over a sphere of radius r
        x = 2 * b * r * R
        return (b / np.pi) ** 1.5 * np.exp(-b * (r - R) ** 2) * (-np.expm1(-2 * x)) / (2 * x)
    val, _ = integrate.quad(lambda r: _gaussian_cloud_potential(a, r) * 4 * np.pi * r * r * avg(r),
                            1e-9, R + 12.0 / np.sqrt(min(a, b)), limit=200, epsabs=1e-12)
    return val


@pytest.mark.parametrize("a,b,R", [(0.3, 0.3, 1.8), (0.1, 2.7, 1.1), (1.5, 0.45, 3.6)])
def test_two_center_matches_electrostatics_of_gaussian_clouds(a, b, R):
    aux = inputs.Basis([((a,), (1.0,)), ((b,), (1.0,))])
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    V = integrals.two_center(aux, xyz)
    na, nb = (2 * a / np.pi) ** 0.75, (2 * b / np.pi) ** 0.75
    qa, qb = na * (np.pi / a) ** 1.5, nb * (np.pi / b) ** 1.5
    expect = qa * qb * _cloud_interaction(a, b, R)
    # (a on atom 0) with (b on atom 1) is aux index 0 and 3
    assert abs(V[0, 3] - expect) < 1e-9 * max(1.0, abs(expect))


def test_nuclear_attraction_matches_cloud_potential():
    a, R = 0.7, 1.3
    orb = inputs.Basis([((a,), (1.0,))])
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    _, _, V = integrals.one_electron(orb, xyz)
    # |g|^2 is a unit cloud of exponent 2a; attraction to its own nucleus (r -> 0 limit) + other
    self_term = -_gaussian_cloud_potential(2 * a, 1e-7)
    other = -_gaussian_cloud_potential(2 * a, R)
    assert abs(V[0, 0] - (self_term + other)) < 1e-8


def test_metric_and_overlap_positive_definite():
    orb, aux = inputs.basis_3s_10aux()
    xyz = inputs.jittered_chain(6, seed=2)
    S, _, _ = integrals.one_electron(orb, xyz)
    V = integrals.two_center(aux, xyz)
    for M in (S, V):
        np.testing.assert_allclose(M, M.T, atol=1e-14)
        assert np.linalg.eigvalsh(M)[0] > 0


def test_ri_exact_when_aux_spans_products():
    # one centre, two primitives: the three products have exponents 1, 2, 3
    orb = inputs.Basis(inputs.even_tempered_shells(0.5, 3.0, 2))
    aux = inputs.Basis([((1.0,), (1,)), ((2.0,), (1,)), ((3.0,), (1,))])
    xyz = np.zeros((1, 3))
    B = ri.fitted_B(orb, aux, xyz)
    np.testing.assert_allclose(ri.fitted_eri(B), integrals.four_center(orb, xyz), atol=1e-13)


def test_ri_variational_and_converging():
    orb = inputs.Basis([inputs.sto3g_like_shell(1.24)])
    xyz = inputs.chain(4, 1.8)
    exact = integrals.four_center(orb, xyz)
    n = 4
    prev = None
    for count in (4, 6, 8):
        aux = inputs.Basis(inputs.even_tempered_shells(0.1, 3.0, count))
        fit = ri.fitted_eri(ri.fitted_B(orb, aux, xyz))
        diag_err = np.array([exact[p, q, p, q] - fit[p, q, p, q] for p in range(n) for q in range(n)])
        assert np.all(diag_err > -1e-12)          # (pq|pq)_RI <= (pq|pq)
        err = np.max(np.abs(fit - exact))
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 3e-3  # atom-centred s aux cannot represent bond-midpoint products exactly


def test_ri_ill_conditioned_metric_is_refused():
    aux = inputs.Basis([((1.0,), (1,)), ((1.0 + 1e-9,), (1,))])
    xyz = np.zeros((1, 3))
    with pytest.raises(ri.IllConditioned):
        ri.inverse_sqrt_metric(integrals.two_center(aux, xyz))


def test_overlap_alone_equals_one_electron_overlap():
    for orb, xyz in [(inputs.basis_h4()[0], inputs.chain(4, 1.8)), (inputs.basis_3s_10aux()[0], inputs.chain(6, 1.8))]:
        np.testing.assert_allclose(integrals.overlap(orb, xyz), integrals.one_electron(orb, xyz)[0], atol=1e-15)


def test_separate_one_electron_matrices_equal_one_electron():
    """overlap, kinetic and nuclear_attraction (summed over a partition of the nuclei) equal the
    matrices of one_electron, on a non-collinear geometry with a nuclear charge of 2."""
    from paper_2512_13550_gb300 import inputs
    orb, _ = inputs.basis_3s_10aux()
    xyz = np.array([[0.0, 0.0, 0.0], [1.4, 0.2, 0.0], [0.3, 1.7, 0.4], [2.1, 1.5, -0.6], [-1.2, 0.4, 0.9]])
    Z = np.array([1.0, 2.0, 1.0, 1.0, 1.0])
    S, T, V = integrals.one_electron(orb, xyz, Z)
    np.testing.assert_allclose(integrals.overlap(orb, xyz), S, atol=1e-14, rtol=0)
    np.testing.assert_allclose(integrals.kinetic(orb, xyz), T, atol=1e-13, rtol=0)
    parts = [integrals.nuclear_attraction(orb, xyz, Z, c) for c in ([0, 1], [2], [3, 4])]
    np.testing.assert_allclose(sum(parts), V, atol=1e-12, rtol=0)
    np.testing.assert_allclose(integrals.nuclear_attraction(orb, xyz, Z), V, atol=1e-13, rtol=0)
