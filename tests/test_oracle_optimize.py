"""Pins of the oracle's converged ON / NO loop (oracle/optimize.py; no GPU).

The loop's schedule is a reading (the paper delegates its ADAM details), but what it converges to
is fixed: a stationary point of E over (C, gamma) with a symmetric lambda. It is checked against
a library minimiser, against two-electron full CI (where every PNOF is exact), and by the local
curvature at the converged point."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import integrals, optimize, pnof, reference, ri, step
from paper_2512_13550_gb300 import inputs


def _chain(natom, basis, spacing=1.8):
    orb, aux = basis
    xyz = inputs.chain(natom, spacing)
    S, T, V = integrals.one_electron(orb, xyz)
    return S, T + V, ri.fitted_B(orb, aux, xyz), integrals.nuclear_repulsion(xyz), orb, aux, xyz


def test_on_converge_reaches_the_library_minimum():
    """ONs at fixed orbitals (the core guess, where the ON minimum is interior: at arbitrary
    orbitals it may lie on the trigonometric mapping's boundary n_g = 1/2, where the gradient has a
    kink): the Armijo descent stops below the tolerance at the energy that scipy's BFGS finds from
    the same start."""
    S, H, B, vnn, *_ = _chain(6, inputs.basis_3s_10aux())
    n = S.shape[0]
    pm = pnof.PairMap(6, 2, n)
    C = reference.core_guess(S, H)
    J, K = pnof.jk(B, C, pm.nact)
    hpp = np.einsum("mp,mn,np->p", C[:, :pm.nact], H, C[:, :pm.nact])
    g0 = inputs.random_gamma(pm.ngamma, 4)
    gam, its, gmax = optimize.on_converge(hpp, J, K, g0, pm, tol=1e-9)
    assert gmax < 1e-9 and its > 0
    f = lambda x: optimize.on_energy(hpp, J, K, x, pm)
    df = lambda x: pnof.gamma_gradient(hpp, J, K, x, pm)
    ref = minimize(f, g0, jac=df, method="BFGS", options={"gtol": 1e-11, "maxiter": 10000})
    assert abs(f(gam) - ref.fun) < 1e-12
    assert f(gam) < f(g0)


def test_two_electron_loop_reaches_full_ci():
    """H2 with every orbital in the one subspace (N_g = n - 1): PNOF7 is exact for two electrons,
    so the loop's converged energy is the two-electron full CI energy with the same fitted
    integrals."""
    S, H, B, vnn, *_ = _chain(2, inputs.basis_3s_10aux(), spacing=1.4)
    n = S.shape[0]
    pm = pnof.PairMap(2, n - 1, n)
    C0 = reference.core_guess(S, H)
    r = optimize.optimize(B, H, vnn, C0, np.full(pm.ngamma, 0.3), pm, gtol=1e-7, etol=1e-11, maxit=3000)
    assert r["converged"]
    eri = reference.mo_integrals(ri.fitted_eri(B), C0)
    e_fci = reference.fci_two_electron(C0.T @ H @ C0, eri) + vnn
    assert abs(r["E"] - e_fci) < 1e-8


def test_converged_point_is_a_symmetric_lambda_minimum():
    """H6 (3 s + 10 aux s per H): at convergence lambda is symmetric (the paper's NTHRESHL test),
    the occupation gradient vanishes, and small random rotations do not lower the energy."""
    S, H, B, vnn, *_ = _chain(6, inputs.basis_3s_10aux())
    n = S.shape[0]
    pm = pnof.PairMap(6, 1, n)
    r = optimize.optimize(B, H, vnn, reference.core_guess(S, H), np.full(pm.ngamma, 0.3), pm,
                          gtol=1e-6, etol=1e-10)
    assert r["converged"] and r["gnorm"] < 1e-6
    assert r["lam_asym"] < 1e-6
    C, gam = r["C"], r["gamma"]
    J, K = pnof.jk(B, C, pm.nact)
    hpp = np.einsum("mp,mn,np->p", C[:, :pm.nact], H, C[:, :pm.nact])
    assert np.max(np.abs(pnof.gamma_gradient(hpp, J, K, gam, pm))) < 1e-8
    E0 = pnof.energy(B, H, C, gam, pm, vnn)
    assert abs(E0 - r["E"]) < 1e-12
    for seed in range(4):
        Y = inputs.random_antisymmetric(n, 50 + seed) * 1e-3
        assert pnof.energy(B, H, C @ step.expm_antisym(Y), gam, pm, vnn) > E0 - 1e-13
    # outer energies never increase (a block keeps orbitals only if they lower E at fixed ONs, and
    # the ON optimisation at the new orbitals lowers it further) and end at the returned energy
    Es = [h[0] for h in r["history"]]
    assert Es[-1] == r["E"] and Es[-1] < Es[0] - 0.1
    assert all(e1 <= e0 + 1e-12 for e0, e1 in zip(Es, Es[1:]))


@pytest.mark.parametrize("natom,basis,spacing", [(4, inputs.basis_h4, 1.8), (6, inputs.basis_h4, 2.2)])
def test_loop_and_library_minimiser_agree(natom, basis, spacing):
    """Chains with one contracted s per H: the loop's converged energy equals that of scipy's
    L-BFGS over all independent variables (y_pq, p < q, and gamma) at once from the same start
    (finite-difference gradients of E(C0 exp(Y), gamma))."""
    S, H, B, vnn, *_ = _chain(natom, basis(), spacing)
    n = S.shape[0]
    pm = pnof.PairMap(natom, 1, n)
    # a generic start: the core guess of a symmetric chain is a symmetry-preserving stationary
    # point in the rotations that mix symmetry classes, where a gradient method can stay
    C0 = reference.core_guess(S, H) @ step.expm_antisym(inputs.random_antisymmetric(n, 9) * 0.05)
    g0 = np.full(pm.ngamma, 0.3)
    r = optimize.optimize(B, H, vnn, C0, g0, pm, gtol=1e-6, etol=1e-10)
    assert r["converged"]
    iu = np.triu_indices(n, 1)

    def f(x):
        Y = np.zeros((n, n))
        Y[iu] = x[:len(iu[0])]
        Y = Y - Y.T
        C = C0 @ step.expm_antisym(Y)
        gam = x[len(iu[0]):]
        e = pnof.energy_and_gradients(B, H, C, gam, pm, vnn)
        return e["E"]

    x0 = np.concatenate([np.zeros(len(iu[0])), g0])
    ref = minimize(f, x0, method="L-BFGS-B",
                   options={"maxiter": 20000, "maxfun": 200000, "ftol": 1e-15, "gtol": 1e-9})
    assert ref.fun > r["E"] - 1e-9  # the library finds nothing lower
    assert abs(r["E"] - ref.fun) < 1e-8
