"""Geometry optimisation and Verlet dynamics of H2 on the GPU (FP64 path, converged states)
against the oracle's drivers."""
import numpy as np
import pytest

from oracle import dynamics as odyn
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M_H = 1837.15


def _h2(R):
    return np.array([[0.0, 0.0, -R / 2], [0.0, 0.0, R / 2]])


def test_h2_optimisation_and_dynamics_match_oracle():
    from paper_2512_13550_gb300 import geometry
    orb, aux = inputs.basis_3s_10aux()
    x_w, E_w, g_w, it_w = odyn.optimize(orb, aux, _h2(1.6), ftol=1e-6)
    x_g, E_g, g_g, it_g = geometry.optimize(_h2(1.6), orb, aux, ftol=1e-6)
    assert np.max(np.abs(g_g)) < 1e-6
    np.testing.assert_allclose(x_g, x_w, rtol=0, atol=1e-6)
    assert abs(E_g - E_w) < 1e-9
    xs_w, vs_w, Es_w = odyn.verlet(orb, aux, _h2(1.55), np.zeros((2, 3)), [M_H, M_H], dt=10.0, nsteps=4)
    xs_g, vs_g, Es_g = geometry.verlet(_h2(1.55), np.zeros((2, 3)), [M_H, M_H], 10.0, 4, orb, aux)
    np.testing.assert_allclose(xs_g, xs_w, rtol=0, atol=1e-8)
    np.testing.assert_allclose(Es_g, Es_w, rtol=0, atol=1e-9)
