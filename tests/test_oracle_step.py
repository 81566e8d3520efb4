"""Pins of the oracle's optimiser step (no GPU)."""
import numpy as np
import scipy.linalg

from oracle import integrals, pnof, reference, ri, step
from paper_2512_13550_gb300 import inputs


def test_expm_antisymmetric_is_orthogonal_and_matches_library():
    for scale in (1e-3, 0.3, 3.0):
        y = inputs.random_antisymmetric(7, 5, scale)
        U = step.expm_antisym(y)
        np.testing.assert_allclose(U @ U.T, np.eye(7), atol=1e-13)
        np.testing.assert_allclose(U, scipy.linalg.expm(y), atol=1e-12)


def _h4():
    orb, aux = inputs.basis_h4()
    xyz = inputs.chain(4, 1.8)
    S, T, V = integrals.one_electron(orb, xyz)
    return S, T + V, ri.fitted_B(orb, aux, xyz), integrals.nuclear_repulsion(xyz)


def test_step_preserves_orthonormality_and_descends():
    S, H, B, vnn = _h4()
    pm = pnof.PairMap(4, 1, 4)
    st = step.State(reference.orthonormal_orbitals(S, inputs.random_orthogonal(4, 0)),
                    inputs.random_gamma(pm.ngamma, 1))
    energies = []
    for _ in range(20):
        E, gn, _ = step.step(B, H, vnn, st, pm, lr=0.005)
        energies.append(E)
    np.testing.assert_allclose(st.C.T @ S @ st.C, np.eye(4), atol=1e-12)
    assert np.all(np.diff(energies) < 0)


def test_converged_lambda_is_symmetric():
    S, H, B, vnn = _h4()
    pm = pnof.PairMap(4, 1, 4)
    st = step.State(reference.core_guess(S, H), np.full(pm.ngamma, 0.3))
    for _ in range(300):
        E, gn, asym = step.step(B, H, vnn, st, pm)
    assert gn < 1e-4 and asym < 2e-5
