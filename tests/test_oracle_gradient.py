"""Pins of the oracle's nuclear gradient (no GPU): integral derivatives against finite
differences of the integral routines, the gradient against finite differences of the energy
along the orbital connection, and its translational and rotational invariance."""
import numpy as np
import pytest

from oracle import gradient, integrals, pnof, reference, ri
from paper_2512_13550_gb300 import inputs

H = 1e-5


def _geometry(natom=3, seed=5):
    """A non-collinear, non-planar-by-symmetry arrangement, so that every component matters."""
    xyz = inputs.chain(natom, 1.6)
    return xyz + inputs.uniform(seed, natom * 3, -0.35, 0.35).reshape(natom, 3)


def _fd(fun, xyz, A, k, h=H):
    xp = xyz.copy(); xp[A, k] += h
    xm = xyz.copy(); xm[A, k] -= h
    return (fun(xp) - fun(xm)) / (2 * h)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_one_electron_derivatives_match_finite_differences(which):
    orb, _ = inputs.basis_h4()
    xyz = _geometry()
    Z = np.array([1.0, 2.0, 1.0])
    d = gradient.one_electron_derivatives(orb, xyz, Z)[which]
    for A in range(3):
        for k in range(3):
            fd = _fd(lambda x: integrals.one_electron(orb, x, Z)[which], xyz, A, k)
            np.testing.assert_allclose(d[A, k], fd, rtol=0, atol=2e-8)


def test_three_and_two_center_derivatives_match_finite_differences():
    orb, aux = inputs.basis_h4()
    xyz = _geometry()
    d3 = gradient.three_center_derivatives(orb, aux, xyz)
    d2 = gradient.two_center_derivatives(aux, xyz)
    for A in range(3):
        for k in range(3):
            fd3 = _fd(lambda x: integrals.three_center(orb, aux, x), xyz, A, k)
            np.testing.assert_allclose(d3[A, k], fd3, rtol=0, atol=2e-8)
            fd2 = _fd(lambda x: integrals.two_center(aux, x), xyz, A, k)
            np.testing.assert_allclose(d2[A, k], fd2, rtol=0, atol=2e-8)
    # translation invariance of every integral: the derivatives over all centres sum to zero
    np.testing.assert_allclose(d3.sum(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(d2.sum(axis=0), 0.0, atol=1e-12)


def test_boys_f1():
    t = np.array([0.0, 1e-6, 0.3, 2.0, 30.0])
    u = np.linspace(0.0, 1.0, 200001)
    quad = [np.trapezoid(u * u * np.exp(-ti * u * u), u) for ti in t]
    np.testing.assert_allclose(gradient.boys_f1(t), quad, rtol=1e-9, atol=0)


def _energy_on_connection(orb, aux, x, C0, gam, pm, Z, ipnof):
    S, T, V = integrals.one_electron(orb, x, Z)
    B = ri.fitted_B(orb, aux, x)
    C = gradient.connected_orbitals(C0, S)
    return pnof.energy(B, T + V, C, gam, pm, integrals.nuclear_repulsion(x, Z), ipnof)


@pytest.mark.parametrize("ipnof,ncwo", [(7, 1), (5, 1), (7, 2)])
def test_gradient_matches_finite_differences_of_the_energy(ipnof, ncwo):
    orb = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, 2)) if ncwo == 2 else inputs.basis_h4()[0]
    aux = inputs.basis_h4()[1]
    natom = 4
    xyz = _geometry(natom, seed=9)
    Z = np.ones(natom)
    S, T, V = integrals.one_electron(orb, xyz, Z)
    n = S.shape[0]
    pm = pnof.PairMap(natom, ncwo, n)
    C0 = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 3))
    gam = inputs.random_gamma(pm.ngamma, 4)
    g = gradient.nuclear_gradient(orb, aux, xyz, C0, gam, pm, Z, ipnof)
    for A in range(natom):
        for k in range(3):
            fd = _fd(lambda x: _energy_on_connection(orb, aux, x, C0, gam, pm, Z, ipnof), xyz, A, k, 1e-4)
            assert abs(g[A, k] - fd) < 1e-7 * max(1.0, abs(fd)), (A, k, g[A, k], fd)
    # a rigid translation or rotation changes no integral of s functions: no net force or torque
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-10)
    np.testing.assert_allclose(np.cross(xyz, g).sum(axis=0), 0.0, atol=1e-10)
