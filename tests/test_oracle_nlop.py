"""Pins of the oracle's finite-field workload (no GPU): dipole integrals, field term, dipole,
finite differences, Romberg triangle and its selection rule."""
import numpy as np

from oracle import integrals, nlop, pnof, reference, ri
from paper_2512_13550_gb300 import inputs


def _h4_centred():
    orb, aux = inputs.basis_h4()
    xyz = inputs.chain(4, 1.8)
    xyz = xyz - xyz.mean(axis=0)
    return orb, aux, xyz


def test_dipole_integrals_match_quadrature():
    """<u|r_k|v> of two contracted s functions on different centres: the Gaussians factorise
    over x, y, z, so each component is one 1-D quadrature times two closed-form overlaps."""
    orb = inputs.Basis([inputs.sto3g_like_shell(1.24)])
    xyz = np.array([[0.3, -0.2, 0.1], [-0.4, 0.5, 1.6]])
    D = nlop.dipole_integrals(orb, xyz)
    funcs = integrals._functions(orb, xyz)
    grid = np.linspace(-12.0, 12.0, 48001)
    dx = grid[1] - grid[0]

    fa, fb = funcs
    for k in range(3):
        # the 3-D function is a sum of products, so integrate primitive pairs separately
        total = 0.0
        for ai, ci in zip(fa[1], fa[2]):
            for bj, cj in zip(fb[1], fb[2]):
                part = ci * cj
                for ax in range(3):
                    ga = np.exp(-ai * (grid - fa[0][ax]) ** 2)
                    gb = np.exp(-bj * (grid - fb[0][ax]) ** 2)
                    w = grid if ax == k else 1.0
                    part *= np.sum(w * ga * gb) * dx
                total += part
        assert abs(D[k, 0, 1] - total) < 1e-10
        assert abs(D[k, 1, 0] - D[k, 0, 1]) < 1e-15
    S = integrals.overlap(orb, xyz)
    for k in range(3):  # a function with itself: the centre times the norm
        np.testing.assert_allclose(np.diag(D[k]), xyz[:, k] * np.diag(S), atol=1e-14)


def test_dipole_integrals_origin_dependence():
    orb, _, xyz = _h4_centred()
    d = np.array([0.7, -1.1, 2.3])
    D0 = nlop.dipole_integrals(orb, xyz)
    D1 = nlop.dipole_integrals(orb, xyz + d)
    S = integrals.overlap(orb, xyz)
    for k in range(3):
        np.testing.assert_allclose(D1[k], D0[k] + d[k] * S, atol=1e-13)


def test_field_energy_is_linear_with_slope_minus_dipole():
    orb, aux, xyz = _h4_centred()
    S, T, V = integrals.one_electron(orb, xyz)
    H = T + V
    B = ri.fitted_B(orb, aux, xyz)
    vnn = integrals.nuclear_repulsion(xyz)
    n = S.shape[0]
    pm = pnof.PairMap(4, 1, n)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 4))
    gam = inputs.random_gamma(pm.ngamma, 5)
    D = nlop.dipole_integrals(orb, xyz)
    E0 = pnof.energy(B, H, C, gam, pm, vnn)
    mu = nlop.dipole(C, gam, pm, D, xyz)
    for F in ([0.01, 0.0, 0.0], [0.0, -0.02, 0.0], [0.003, 0.004, -0.05]):
        Hf, vf = nlop.field_hamiltonian(H, D, F, xyz, vnn)
        assert abs(pnof.energy(B, Hf, C, gam, pm, vf) - (E0 - np.dot(F, mu))) < 1e-12
    # the electronic part counts 2 n_p electrons per orbital: a uniform shift of the molecule
    # by d changes mu by (sum_A Z_A - N) d = 0 for the neutral molecule
    D1 = nlop.dipole_integrals(orb, xyz + 1.5)
    np.testing.assert_allclose(nlop.dipole(C, gam, pm, D1, xyz + 1.5), mu, atol=1e-12)


def test_differences_and_romberg_reproduce_polynomial_derivatives():
    """mu(F) = a F + b F^2 + c F^3 + e F^5: alpha(h) = a + c h^2 + e h^4 (Romberg column 3
    is exact), beta(h) = 2b exactly, gamma(h) = 6c + 30 e h^2 (column 2 is exact)."""
    a, b, c, e = 4.5, -0.75, 120.0, 3.0e4
    step_size, npoint = 1e-3, 5
    mu = {f: a * f + b * f * f + c * f ** 3 + e * f ** 5 for f in nlop.field_points(step_size, npoint)}
    al, be, ga = nlop.differences(mu, step_size, npoint)
    h = step_size * 2.0 ** np.arange(npoint)
    np.testing.assert_allclose(al, a + c * h ** 2 + e * h ** 4, rtol=1e-9)
    np.testing.assert_allclose(be, 2 * b, rtol=1e-6)
    np.testing.assert_allclose(ga, 6 * c + 30 * e * h ** 2, rtol=1e-9)  # e (32 - 2 - 2 + 32) / 2 = 30 e
    Ra, _ = nlop.romberg(al)
    assert abs(Ra[0, 2] - a) < 1e-9 * abs(a)
    Rg, _ = nlop.romberg(ga)
    assert abs(Rg[0, 1] - 6 * c) < 1e-6 * abs(6 * c)


def test_romberg_triangle_entries_and_selection_rule():
    # D(h_k) = c0 + c1 h^2 + c2 h^4 + c3 h^6 with h_k = 2^{k-1}: column j removes h^{2(j-1)}
    h = 2.0 ** np.arange(6)
    Dv = 7.0 + 0.5 * h ** 2 - 0.01 * h ** 4 + 1e-4 * h ** 6
    R, (val, delta, k, j) = nlop.romberg(Dv)
    assert np.isnan(R[5, 1]) and np.isnan(R[1, 5]) and not np.isnan(R[0, 5])
    np.testing.assert_allclose(R[:3, 3], 7.0, rtol=1e-13)
    # the first pair of column 4 (and beyond) already agrees to rounding: Delta = 0 there
    assert delta < 1e-12 and abs(val - 7.0) < 1e-12 and j >= 4
    # hand-made table: column 1 = [1, 2, 4, 4.5]; R(k, 2) = R(k,1) + (R(k,1) - R(k+1,1)) / 3
    R, (val, delta, k, j) = nlop.romberg([1.0, 2.0, 4.0, 4.5])
    np.testing.assert_allclose(R[:3, 1], [1 - 1 / 3, 2 - 2 / 3, 4 - 0.5 / 3])
    assert (k, j) == (3, 1) and delta == 0.5 and val == R[2, 1]
    # ties in Delta go to the candidate of smallest magnitude: pairs (1,2) and (2,3) of
    # column 1 both have Delta = 1; R(1,2) = -2 - 1/3 ... R(2,2) = -1 - 1/3 ...
    R, (val, delta, k, j) = nlop.romberg([-2.0, -1.0, 0.0, 7.0])
    cands = [(abs(R[0, 0] - R[1, 0]), R[0, 1]), (abs(R[1, 0] - R[2, 0]), R[1, 1])]
    assert cands[0][0] == cands[1][0] == 1.0
    assert (k, j) == (2, 1) and val == R[1, 1] and abs(R[1, 1]) < abs(R[0, 1])


def test_centrosymmetric_chain_dipole_is_odd_in_the_field():
    """A centred H4 chain with inversion-symmetric starting orbitals: for F != 0 the trajectory
    under -F is the inversion image of the one under F, so mu(-F) = -mu(F) and beta(h) reduces
    to -2 mu(0) / h^2. (At F = 0 the symmetric state is a saddle for this chain: ADAM turns the
    1e-14 rounding in gradient elements that vanish by symmetry into full-size steps, so mu(0)
    itself is not zero after a few steps; the pin is on the nonzero fields.)"""
    orb, aux, xyz = _h4_centred()
    S, T, V = integrals.one_electron(orb, xyz)
    H = T + V
    B = ri.fitted_B(orb, aux, xyz)
    vnn = integrals.nuclear_repulsion(xyz)
    n = S.shape[0]
    pm = pnof.PairMap(4, 1, n)
    C0 = reference.core_guess(S, H)
    D = nlop.dipole_integrals(orb, xyz)
    r = nlop.run(B, H, D, xyz, vnn, pm, axis=2, step_size=2e-3, npoint=4, nsteps=3,
                 C0=C0, gamma0=np.full(pm.ngamma, 0.3))
    for f in r["mu"]:
        if f != 0.0:
            assert abs(r["mu"][f] + r["mu"][-f]) < 1e-11
    al, be, ga = r["D"]
    h = 2e-3 * 2.0 ** np.arange(4)
    np.testing.assert_allclose(be, -2.0 * r["mu"][0.0] / h ** 2, rtol=1e-6)


def test_polarizability_invariants():
    """Isotropic tensor: mean = the value, anisotropy 0; axially symmetric (a, a, c): anisotropy
    |c - a| (the Raman-convention formula reduces to it)."""
    assert nlop.polarizability_invariants(4.0, 4.0, 4.0) == (4.0, 0.0)
    iso, an = nlop.polarizability_invariants(2.0, 2.0, 5.0)
    assert abs(iso - 3.0) < 1e-15 and abs(an - 3.0) < 1e-15
