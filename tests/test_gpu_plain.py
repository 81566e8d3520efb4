"""Parity of the plain FP64 GPU path (called through the C ABI) with the CPU oracle."""
import numpy as np
import pytest

import systems
from oracle import pnof, reference, ri, step
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 on both sides; only the summation order differs


def _ctx(sysm, precision=0, **kw):
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=precision, ncwo=sysm.ncwo, **kw)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    return ctx


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _n(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


@pytest.mark.parametrize("make", [systems.h4, lambda: systems.chain3s(6)])
def test_setup_matches_oracle(make):
    sysm = make()
    o = sysm.oracle
    ctx = _ctx(sysm)
    s = ctx.sizes
    assert s["nbf"] == o["n"] and s["naux"] == o["B"].shape[0]
    assert abs(s["vnn"] - o["vnn"]) < 1e-12
    S, H = ctx.get_SH()
    np.testing.assert_allclose(_n(S), o["S"], atol=1e-13)
    np.testing.assert_allclose(_n(H), o["H"], atol=1e-12)
    # the fitted 4-index tensor is independent of the square root of the metric
    B = _n(ctx.get_B())
    np.testing.assert_allclose(ri.fitted_eri(B), ri.fitted_eri(o["B"]), atol=1e-11)


def test_lowdin_orthonormal():
    sysm = systems.chain3s(6)
    o = sysm.oracle
    ctx = _ctx(sysm)
    Q = inputs.random_orthogonal(o["n"], 0)
    C = _n(ctx.lowdin(_t(Q)))
    np.testing.assert_allclose(C.T @ o["S"] @ C, np.eye(o["n"]), atol=1e-11)
    np.testing.assert_allclose(C, reference.orthonormal_orbitals(o["S"], Q), atol=1e-10)


@pytest.mark.parametrize("natom", [4, 10, 22])
def test_jk_parity(natom):
    sysm = systems.h4() if natom == 4 else systems.chain3s(natom)
    o = sysm.oracle
    ctx = _ctx(sysm)
    C = sysm.orbitals()
    J, K = ctx.jk(_t(C))
    Jo, Ko = pnof.jk(o["B"], C, o["pm"].nact)
    np.testing.assert_allclose(_n(J), Jo, atol=TOL)
    np.testing.assert_allclose(_n(K), Ko, atol=TOL)


@pytest.mark.parametrize("natom,ncwo,ipnof", [(4, 1, 7), (10, 1, 7), (10, 1, 5), (8, 2, 7)])
def test_energy_grad_parity(natom, ncwo, ipnof):
    sysm = systems.h4(ncwo) if natom == 4 else systems.chain3s(natom, ncwo=ncwo)
    o = sysm.oracle
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=0, ncwo=ncwo, ipnof=ipnof)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    C, gam = sysm.orbitals(), sysm.gamma()
    E, g, gg = ctx.energy_grad(_t(C), _t(gam))
    ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"], ipnof)
    assert abs(_n(E)[0] - ref["E"]) < TOL * max(1.0, abs(ref["E"]))
    np.testing.assert_allclose(_n(g), ref["g"], atol=TOL)
    np.testing.assert_allclose(_n(gg), ref["g_gamma"], atol=TOL)


def test_h50_plain_parity():
    sysm = systems.h50()
    o = sysm.oracle
    ctx = _ctx(sysm)
    C, gam = sysm.orbitals(), sysm.gamma()
    E, g, gg = ctx.energy_grad(_t(C), _t(gam))
    ref = pnof.energy_and_gradients(o["B"], o["H"], C, gam, o["pm"], o["vnn"])
    assert abs(_n(E)[0] - ref["E"]) < 1e-9
    np.testing.assert_allclose(_n(g), ref["g"], atol=1e-9)
    np.testing.assert_allclose(_n(gg), ref["g_gamma"], atol=1e-9)


def test_step_trajectory_h4():
    """H4 run: 20 alternating steps from a seeded orthonormal C and seeded gamma."""
    sysm = systems.h4()
    o = sysm.oracle
    ctx = _ctx(sysm)
    C0, g0 = sysm.orbitals(0), sysm.gamma(1)
    st = step.State(C0, g0)
    Cd, gd = _t(C0), _t(g0)
    n = o["n"]
    m, v = _t(np.zeros((n, n))), _t(np.zeros((n, n)))
    for it in range(20):
        out = _n(ctx.step(Cd, gd, m, v))
        E, gn, asym = step.step(o["B"], o["H"], o["vnn"], st, o["pm"])
        assert abs(out[0] - E) < TOL, it
        assert abs(out[1] - gn) < 1e-9, it
    np.testing.assert_allclose(_n(Cd), st.C, atol=1e-9)
    np.testing.assert_allclose(_n(gd), st.gamma, atol=1e-9)


def test_error_paths():
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=0)
    C = _t(np.eye(4))
    with pytest.raises(nof.NofError) as e:
        ctx.sizes = dict(nact=4, nbf=4, ngamma=2)
        ctx.jk(C)
    assert e.value.code == nof.NOF_ESTATE
    orb, aux = inputs.basis_h4()
    with pytest.raises(nof.NofError) as e:  # odd electron count
        ctx.build_B(inputs.chain(3), orb, aux)
    assert e.value.code == nof.NOF_EINVAL
    with pytest.raises(nof.NofError) as e:  # triplet
        ctx.build_B(inputs.chain(4), orb, aux, mult=3)
    assert e.value.code == nof.NOF_EINVAL
    bad_aux = inputs.Basis([((1.0,), (1,)), ((1.0 + 1e-12,), (1,))])
    with pytest.raises(nof.NofError) as e:  # numerically singular metric
        ctx.build_B(inputs.chain(4), orb, bad_aux)
    assert e.value.code == nof.NOF_EILLCOND
    with pytest.raises(nof.NofError) as e:
        nof.Context(precision=0, ipnof=3)
    assert e.value.code == nof.NOF_EINVAL
