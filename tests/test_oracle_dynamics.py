"""Pins of the oracle's geometry optimisation and dynamics on converged states (no GPU): H2 in the
3 s + 10 aux s basis."""
import numpy as np

from oracle import dynamics
from paper_2512_13550_gb300 import inputs

M_H = 1837.15  # proton mass plus one electron, in electron masses


def _h2(R):
    return np.array([[0.0, 0.0, -R / 2], [0.0, 0.0, R / 2]])


def test_optimised_h2_is_a_minimum_of_the_converged_energy():
    orb, aux = inputs.basis_3s_10aux()
    xyz, E, g, it = dynamics.optimize(orb, aux, _h2(1.6), ftol=1e-6)
    assert np.max(np.abs(g)) < 1e-6 and it < 30
    R = np.linalg.norm(xyz[1] - xyz[0])
    assert 1.2 < R < 1.6
    for d in (-0.01, 0.01):
        Ed, _, _ = dynamics.converged_point(orb, aux, _h2(R + d))
        assert Ed > E
    # a rigid motion of the optimised molecule changes nothing
    np.testing.assert_allclose(g.sum(axis=0), 0.0, atol=1e-10)


def test_verlet_energy_error_is_second_order_in_the_time_step():
    """Velocity Verlet on the converged surface: over the same 40 au from a stretched bond, halving
    the step cuts the total-energy error by about 4 (a force inconsistent with the energy would
    leave a drift that does not shrink with the step). The centre of mass stays put and the motion
    stays on the bond axis."""
    orb, aux = inputs.basis_3s_10aux()
    err = []
    for dt, n in ((10.0, 4), (5.0, 8)):
        xs, vs, Es = dynamics.verlet(orb, aux, _h2(1.55), np.zeros((2, 3)), [M_H, M_H], dt=dt, nsteps=n)
        kin = 0.5 * M_H * np.sum(vs ** 2, axis=(1, 2))
        tot = Es + kin
        err.append(np.max(np.abs(tot - tot[0])))
        assert kin[-1] > 1e-4  # the bond actually moves
        np.testing.assert_allclose(xs.mean(axis=1), 0.0, atol=1e-10)
        np.testing.assert_allclose(xs[:, :, :2], 0.0, atol=1e-10)
    assert 3.0 < err[0] / err[1] < 5.0, err
    assert err[1] < 5e-6
