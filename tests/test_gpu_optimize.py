"""The converged ON / NO loop on the GPU (nof_optimize) against the oracle's loop (oracle/optimize.py,
pinned to library minimisers and to two-electron full CI)."""
import ctypes

import numpy as np
import pytest

from oracle import integrals, optimize, pnof, reference, ri
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _system(natom, basis, spacing=1.8, ncwo=1):
    orb, aux = basis
    xyz = inputs.chain(natom, spacing)
    S, T, V = integrals.one_electron(orb, xyz)
    n = S.shape[0]
    return dict(orb=orb, aux=aux, xyz=xyz, S=S, H=T + V, B=ri.fitted_B(orb, aux, xyz),
                vnn=integrals.nuclear_repulsion(xyz), pm=pnof.PairMap(natom, ncwo, n), n=n)


def _ctx(s, precision):
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=precision, ncwo=s["pm"].ncwo)
    ctx.build_B(s["xyz"], s["orb"], s["aux"])
    return ctx


def _start(s, seed=9, scale=0.05):
    from oracle import step
    return reference.core_guess(s["S"], s["H"]) @ step.expm_antisym(inputs.random_antisymmetric(s["n"], seed) * scale)


@pytest.mark.parametrize("precision", [0, 1])
def test_on_convergence_matches_oracle(precision):
    """First outer iteration only: the ONs converged at the start orbitals by the one-block BFGS
    kernel, and the energy there, against the oracle's on_converge."""
    s = _system(8, inputs.basis_3s_10aux(), ncwo=2)
    ctx = _ctx(s, precision)
    C0 = _start(s)
    g0 = inputs.random_gamma(s["pm"].ngamma, 3)
    C, gam = _t(C0), _t(g0)
    r = ctx.optimize(C, gam, maxit=1, maxloop=1)
    a = s["pm"].nact
    J, K = pnof.jk(s["B"], C0, a)
    hpp = np.einsum("mp,mn,np->p", C0[:, :a], s["H"], C0[:, :a])
    ref_g, _, gmax = optimize.on_converge(hpp, J, K, g0, s["pm"])
    assert gmax < 1e-8
    E_ref = pnof.energy(s["B"], s["H"], C0, ref_g, s["pm"], s["vnn"])
    tol = 1e-9 if precision == 0 else 1e-6
    assert abs(r["history"][0, 0] - E_ref) < tol
    assert np.max(np.abs(gam.cpu().numpy() - ref_g)) < (1e-6 if precision == 0 else 1e-4)
    ctx.close()


@pytest.mark.parametrize("orbopt", [0, 1])
def test_fp64_trajectory_matches_oracle(orbopt):
    """15 outer iterations of the FP64 path and of the oracle from the same start, with ADAM blocks
    (orbopt 0) and with L-BFGS steps (orbopt 1): the energies, gradient norms and rates of every
    outer iteration agree (the same decisions are taken)."""
    s = _system(4, inputs.basis_3s_10aux())
    ctx = _ctx(s, 0)
    C0 = _start(s)
    g0 = np.full(s["pm"].ngamma, 0.3)
    r = ctx.optimize(_t(C0), _t(g0), maxit=15, orbopt=orbopt)
    ref = optimize.optimize(s["B"], s["H"], s["vnn"], C0, g0, s["pm"], maxit=15, orbopt=orbopt)
    h = np.array(ref["history"])
    assert r["iterations"] == len(h) == 15
    np.testing.assert_allclose(r["history"][:, 0], h[:, 0], atol=1e-9, rtol=0)
    np.testing.assert_allclose(r["history"][:, 1], h[:, 1], atol=1e-8, rtol=1e-6)
    np.testing.assert_array_equal(r["history"][:, 2], h[:, 2])
    assert r["evaluations"] == ref["evaluations"]
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_converged_energy_matches_oracle(precision):
    """H6 (3 s + 10 aux s per H) from a generic start to ||g|| < 1e-5: converged, symmetric
    lambda, and the oracle's converged energy (the same minimum) on both precisions."""
    s = _system(6, inputs.basis_3s_10aux())
    ctx = _ctx(s, precision)
    C0 = _start(s)
    g0 = np.full(s["pm"].ngamma, 0.3)
    C, gam = _t(C0), _t(g0)
    r = ctx.optimize(C, gam, gtol=1e-5, etol=1e-9)
    ref = optimize.optimize(s["B"], s["H"], s["vnn"], C0, g0, s["pm"], gtol=1e-5, etol=1e-9)
    print(f"precision {precision}: E {r['E']:.12f} (oracle {ref['E']:.12f}), ||g|| {r['gnorm']:.2e}, "
          f"{r['iterations']} iterations, {r['evaluations']} evaluations (oracle {ref['iterations']}, "
          f"{ref['evaluations']}), final rate {r['lr']:.2e}")
    assert r["converged"] and ref["converged"]
    assert r["gnorm"] < 1e-5 and r["lam_asym"] < 1e-5
    assert abs(r["E"] - ref["E"]) < (1e-9 if precision == 0 else 1e-7)
    # the returned state is the converged one: its energy evaluated afresh
    E_state = pnof.energy(s["B"], s["H"], C.cpu().numpy(), gam.cpu().numpy(), s["pm"], s["vnn"])
    assert abs(E_state - r["E"]) < (1e-10 if precision == 0 else 1e-6)
    ctx.close()


def test_two_electron_loop_reaches_full_ci():
    """H2 with every orbital in one subspace: the GPU loop's energy is two-electron full CI."""
    s = _system(2, inputs.basis_3s_10aux(), spacing=1.4, ncwo=5)
    ctx = _ctx(s, 0)
    C0 = reference.core_guess(s["S"], s["H"])
    r = ctx.optimize(_t(C0), _t(np.full(s["pm"].ngamma, 0.3)), gtol=1e-7, etol=1e-11, maxit=3000)
    assert r["converged"]
    eri = reference.mo_integrals(ri.fitted_eri(s["B"]), C0)
    e_fci = reference.fci_two_electron(C0.T @ s["H"] @ C0, eri) + s["vnn"]
    assert abs(r["E"] - e_fci) < 1e-8
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_orbitals_are_reported(precision):
    """A NaN in C reaches the energy: nof_energy_grad's status word gives NOF_ENONFINITE at
    nof_sync, and nof_optimize returns it; the context stays usable afterwards."""
    import paper_2512_13550_gb300 as nof
    s = _system(4, inputs.basis_3s_10aux())
    ctx = _ctx(s, precision)
    C0 = _start(s)
    bad = C0.copy()
    bad[3, 2] = np.nan
    gam = _t(np.full(s["pm"].ngamma, 0.3))
    ctx.energy_grad(_t(bad), gam)
    with pytest.raises(nof.NofError) as ei:
        ctx.sync()
    assert ei.value.code == nof.NOF_ENONFINITE
    with pytest.raises(nof.NofError) as ei:
        ctx.optimize(_t(bad), gam.clone(), maxit=3)
    assert ei.value.code == nof.NOF_ENONFINITE
    ctx.sync()  # the status word was read and cleared
    E, _, _ = ctx.energy_grad(_t(C0), gam)
    ctx.sync()
    assert np.isfinite(E.item())
    ctx.close()
