"""Parity of the split-precision tensor-core path (exact BF16 digit planes on tcgen05) with the
CPU FP64 oracle, through the C ABI. Tolerance: 1e-6 Ha on E and 1e-6 max-abs on J, K and the
orbital and occupation gradients (the accuracy gate of the evaluation)."""
import numpy as np
import pytest

import systems
from oracle import pnof, ri
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-6


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _n(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


def _ctx(sysm, ipnof=7, digits=0):
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, ncwo=sysm.ncwo, ipnof=ipnof, digits=digits)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    return ctx


CASES = {
    "H4": lambda: systems.h4(),                    # n = a = 4: one digit atom, heavy padding
    "H10": lambda: systems.chain3s(10),            # n = 30, a = 10 (ragged everywhere)
    "H22": lambda: systems.chain3s(22),            # n = 66, a = 22 (a padded to 32)
    "H8_ncwo2": lambda: systems.chain3s(8, ncwo=2),  # two weak orbitals per pair
    "H50": lambda: systems.h50(),                  # the benchmark workload (n = 150, a = 50)
    "H64": lambda: systems.chain3s(64, seed=5),    # n = 192 > 160: two exact K accumulations
    "H66": lambda: systems.chain3s(66, seed=6),    # a = 66: several N tiles, the last one ragged
}


def test_digit_storage_reproduces_fitted_eri():
    sysm = systems.chain3s(6)
    o = sysm.oracle
    B = _n(_ctx(sysm).get_B())
    ref = ri.fitted_eri(o["B"])
    assert np.max(np.abs(ri.fitted_eri(B) - ref)) < 1e-8 * np.max(np.abs(ref))


@pytest.mark.parametrize("name,digits", [(k, 0) for k in CASES] + [("H10", 5), ("H22", 5), ("H66", 5),
                                                                   ("H8_ncwo2", 5)])
def test_split_jk_energy_gradients(name, digits):
    """digits 0 = automatic (4 for all of these sizes); 5 forces five BF16 digits per element."""
    sysm = CASES[name]()
    o = sysm.oracle
    ctx = _ctx(sysm, digits=digits)
    C, gam = sysm.orbitals(), sysm.gamma()
    Ct, gt = _t(C), _t(gam)
    J, K = ctx.jk(Ct)
    E, g, gg = ctx.energy_grad(Ct, gt)
    ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"])
    assert abs(_n(E)[0] - ref["E"]) < GATE
    assert np.max(np.abs(_n(J) - ref["J"])) < GATE
    assert np.max(np.abs(_n(K) - ref["K"])) < GATE
    assert np.max(np.abs(_n(g) - ref["g"])) < GATE
    assert np.max(np.abs(_n(gg) - ref["g_gamma"])) < GATE


def test_split_pnof5():
    sysm = systems.chain3s(10)
    o = sysm.oracle
    ctx = _ctx(sysm, ipnof=5)
    C, gam = sysm.orbitals(3), sysm.gamma(4)
    E, g, gg = ctx.energy_grad(_t(C), _t(gam))
    ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"], 5)
    assert abs(_n(E)[0] - ref["E"]) < GATE
    assert np.max(np.abs(_n(g) - ref["g"])) < GATE


def test_split_step_energy_matches_oracle_step():
    """One alternating step from a shared state: same ON update and the same energy."""
    from oracle import step
    sysm = systems.chain3s(10)
    o = sysm.oracle
    ctx = _ctx(sysm)
    C0, g0 = sysm.orbitals(0), sysm.gamma(1)
    st = step.State(C0, g0)
    n = o["n"]
    Cd, gd = _t(C0), _t(g0)
    m, v = _t(np.zeros((n, n))), _t(np.zeros((n, n)))
    out = _n(ctx.step(Cd, gd, m, v))
    E, gn, _ = step.step(o["B"], o["H"], o["vnn"], st, o["pm"])
    assert abs(out[0] - E) < GATE
    np.testing.assert_allclose(_n(gd), st.gamma, atol=1e-6)
    S = o["S"]
    Cn = _n(Cd)
    np.testing.assert_allclose(Cn.T @ S @ Cn, np.eye(n), atol=1e-10)


def test_split_chooses_tiles_per_shape():
    """Different shapes get independent autotuned plans and still agree with the oracle."""
    for name in ("H10", "H22"):
        sysm = CASES[name]()
        o = sysm.oracle
        ctx = _ctx(sysm)
        C, gam = sysm.orbitals(2), sysm.gamma(3)
        E, g, gg = ctx.energy_grad(_t(C), _t(gam))
        ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"])
        assert abs(_n(E)[0] - ref["E"]) < GATE
        assert np.max(np.abs(_n(g) - ref["g"])) < GATE
