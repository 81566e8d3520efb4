"""The slice-by-slice orbital-basis oracle route equals the plain [X][n][n] route."""
import numpy as np
import pytest

import systems
from oracle import integrals, large, pnof


@pytest.mark.parametrize("name,mk", [
    ("H10", lambda: systems.chain3s(10)),
    ("H8_ncwo2", lambda: systems.chain3s(8, ncwo=2)),
    ("H4", lambda: systems.h4()),
])
def test_mo_route_equals_plain_route(name, mk):
    sysm = mk()
    o = sysm.oracle
    C, gam = sysm.orbitals(4), sysm.gamma(5)
    a = o["pm"].nact
    X = integrals.naux(sysm.aux, sysm.xyz)
    # three uneven slices of aux functions, stacked
    cuts = [0, X // 3, X // 3 + 1, X]
    Q3 = np.concatenate([large.mo_three_center(sysm.orb, sysm.aux, sysm.xyz, C, a, slice(lo, hi))
                         for lo, hi in zip(cuts[:-1], cuts[1:])])
    bfull = large.fitted_mo(Q3, integrals.two_center(sysm.aux, sysm.xyz))
    got = large.energy_and_gradients_mo(bfull, o["H"], C, gam, o["pm"], o["vnn"])
    ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"])
    assert abs(got["E"] - ref["E"]) < 1e-11
    for key in ("J", "K", "lam", "g", "g_gamma"):
        np.testing.assert_allclose(got[key], ref[key], atol=1e-11, rtol=0)


def test_blocked_route_and_inplace_fit_equal_the_mo_route():
    """The P-blocked evaluation and the in-place fit (the H1000 memory plan) give the mo route's
    results on H10 with uneven blocks."""
    sysm = systems.chain3s(10)
    o = sysm.oracle
    C, gam = sysm.orbitals(4), sysm.gamma(5)
    a = o["pm"].nact
    Q3 = large.mo_three_center(sysm.orb, sysm.aux, sysm.xyz, C, a)
    V = integrals.two_center(sysm.aux, sysm.xyz)
    ref = large.energy_and_gradients_mo(large.fitted_mo(Q3, V), o["H"], C, gam, o["pm"], o["vnn"])
    b2 = large.fit_inplace(Q3.copy(), V, cols=37)
    got = large.energy_and_gradients_mo_blocked(b2, o["H"], C, gam, o["pm"], o["vnn"], block=7)
    assert abs(got["E"] - ref["E"]) < 1e-12
    for key in ("J", "K", "lam", "g", "g_gamma"):
        np.testing.assert_allclose(got[key], ref[key], atol=1e-12, rtol=0)
