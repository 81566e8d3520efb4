"""Softmax ON mapping (isoftmax = 1) on the GPU against the oracle: energy, orbital gradient and
dE/dgamma on both precision paths, and a step trajectory on the FP64 path."""
import numpy as np
import pytest

import systems
from oracle import pnof, step
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _n(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


def _pm(sysm):
    o = sysm.oracle
    return pnof.PairMap(sysm.xyz.shape[0], sysm.ncwo, o["n"], isoftmax=1)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
@pytest.mark.parametrize("make", [systems.h4, lambda: systems.chain3s(6, ncwo=2), lambda: systems.chain3s(14)])
def test_softmax_energy_and_gradients_match_oracle(make, precision, tol):
    import paper_2512_13550_gb300 as nof
    sysm = make()
    o = sysm.oracle
    pm = _pm(sysm)
    ctx = nof.Context(precision=precision, ncwo=sysm.ncwo, isoftmax=1)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    assert ctx.sizes["ngamma"] == pm.ngamma
    for seed in (3, 4):
        C = sysm.orbitals(seed)
        gam = inputs.uniform(50 + seed, pm.ngamma, -2.5, 1.5)
        want = pnof.energy_and_gradients(o["B"], o["H"], C, gam, pm, o["vnn"])
        E, g, gg = ctx.energy_grad(_t(C), _t(gam))
        assert abs(_n(E)[0] - want["E"]) < tol
        np.testing.assert_allclose(_n(g), want["g"], rtol=0, atol=tol)
        np.testing.assert_allclose(_n(gg), want["g_gamma"], rtol=0, atol=tol)


def test_softmax_step_trajectory_h4():
    import paper_2512_13550_gb300 as nof
    sysm = systems.h4()
    o = sysm.oracle
    pm = _pm(sysm)
    ctx = nof.Context(precision=0, ncwo=sysm.ncwo, isoftmax=1)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    C0, g0 = sysm.orbitals(0), inputs.uniform(9, pm.ngamma, -2.0, 0.5)
    st = step.State(C0, g0)
    Cd, gd = _t(C0), _t(g0)
    n = o["n"]
    m, v = _t(np.zeros((n, n))), _t(np.zeros((n, n)))
    for it in range(15):
        out = _n(ctx.step(Cd, gd, m, v))
        E, gn, _ = step.step(o["B"], o["H"], o["vnn"], st, pm)
        assert abs(out[0] - E) < 1e-10, it
        assert abs(out[1] - gn) < 1e-9, it
    np.testing.assert_allclose(_n(gd), st.gamma, atol=1e-9)
    np.testing.assert_allclose(_n(Cd), st.C, atol=1e-9)


def test_softmax_occupations_are_not_clamped_to_half():
    """The mapping lets a weak orbital hold more than half of its pair (no n_g >= 1/2): a large
    positive variable must still give the oracle's energy."""
    import paper_2512_13550_gb300 as nof
    sysm = systems.h4()
    o = sysm.oracle
    pm = _pm(sysm)
    ctx = nof.Context(precision=0, ncwo=1, isoftmax=1)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    C = sysm.orbitals(2)
    gam = np.array([3.0, -40.0])  # n_p1 = 0.953 in subspace 0, n_g ~ 1 - 4e-18 in subspace 1
    want = pnof.energy_and_gradients(o["B"], o["H"], C, gam, pm, o["vnn"])
    E, g, gg = ctx.energy_grad(_t(C), _t(gam))
    assert abs(_n(E)[0] - want["E"]) < 1e-10
    np.testing.assert_allclose(_n(gg), want["g_gamma"], rtol=0, atol=1e-10)
