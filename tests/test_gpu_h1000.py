"""The H1000 chain (spacing 1.8 bohr, 1 contracted s + 3 aux s per H: nbf 1000, naux 3000,
nact 1000) on the split path through the C ABI:

* against the oracle's orbital-basis route (oracle/large.py, P-blocked, pinned to the plain route):
  E, J, K, the orbital gradient and the occupation gradient element by element at 1e-6. The
  oracle's integrals run in spawned worker processes (nuclear attraction over slices of nuclei,
  three-centre integrals over slices of aux functions); its fitted tensor in the orbital basis
  is one array of 24 GB on the host;
* properties that hold at any size: the invariants of J and K, and the gradients against
  fourth-order finite differences of the split path's own energy.

The orbitals are the oracle's Loewdin orbitals of its overlap matrix."""
import numpy as np
import pytest

import oracle_pool
from oracle import integrals, large, pnof, reference
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-6


@pytest.fixture(scope="module")
def h1000():
    import paper_2512_13550_gb300 as nof
    orb, aux = inputs.basis_h1000()
    xyz = inputs.chain(1000, 1.8)
    S = integrals.overlap(orb, xyz)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(S.shape[0], 0))
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16)
    ctx.build_B(xyz, orb, aux)
    yield dict(ctx=ctx, C=C, n=S.shape[0], orb=orb, aux=aux, xyz=xyz)
    ctx.close()


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_h1000_matches_oracle(h1000):
    ctx, C = h1000["ctx"], h1000["C"]
    s = ctx.sizes
    assert (s["nbf"], s["naux"], s["nact"], ctx.split_digits()) == (1000, 3000, 1000, 5)
    gam = inputs.random_gamma(s["ngamma"], 1)
    J, K = ctx.jk(_t(C))
    E, g, gg = ctx.energy_grad(_t(C), _t(gam))
    torch.cuda.synchronize()
    got = dict(E=E.item(), J=J.cpu().numpy(), K=K.cpu().numpy(), g=g.cpu().numpy(), g_gamma=gg.cpu().numpy())
    orb, aux, xyz = h1000["orb"], h1000["aux"], h1000["xyz"]
    S, H = oracle_pool.core_hamiltonian(orb, xyz)
    pm = pnof.PairMap(1000, 1, s["nbf"])
    bfull = oracle_pool.fitted_mo(orb, aux, xyz, C, pm.nact)
    ref = large.energy_and_gradients_mo_blocked(bfull, H, C, gam, pm, integrals.nuclear_repulsion(xyz))
    del bfull
    dev = {key: float(np.max(np.abs(np.asarray(got[key]) - ref[key]))) for key in ("E", "J", "K", "g", "g_gamma")}
    print("H1000 split path vs oracle, max |difference|:", dev)
    for key, d in dev.items():
        assert d < GATE, key


def test_h1000_jk_invariants(h1000):
    ctx = h1000["ctx"]
    J, K = ctx.jk(_t(h1000["C"]))
    torch.cuda.synchronize()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    assert np.max(np.abs(J - J.T)) < 1e-10
    assert np.max(np.abs(K - K.T)) < 1e-9
    assert np.max(np.abs(np.diag(J) - np.diag(K))) < 1e-10   # (pp|pp) both ways
    assert K.min() >= 0.0                                      # sums of squares
    dJ = np.sqrt(np.outer(np.diag(J), np.diag(J)))
    assert np.all(K <= dJ * (1 + 1e-9) + 1e-12)               # Cauchy-Schwarz of the fitted ERI
    w = np.linalg.eigvalsh(J)
    assert w.min() > -1e-9 * w.max()                            # J = d^T d is positive semidefinite


def test_h1000_gradients_match_finite_differences(h1000):
    """dE along a random orbital rotation C exp(t Y) and along a random gamma direction (fourth-
    order central differences of the split-path energy) against sum_{p<q} g_pq Y_pq and
    g_gamma . dgamma."""
    from scipy.linalg import expm
    ctx, C, n = h1000["ctx"], h1000["C"], h1000["n"]
    gam = inputs.random_gamma(ctx.sizes["ngamma"], 1)
    _, g, gg = ctx.energy_grad(_t(C), _t(gam))
    g = g.cpu().numpy()
    gg = gg.cpu().numpy()
    Y = inputs.random_antisymmetric(n, 7) * 1e-2
    dgam = inputs.normal(8, ctx.sizes["ngamma"]) * 1e-2
    eps = 1e-2

    def energy(Cx, gx):
        E, _, _ = ctx.energy_grad(_t(Cx), _t(gx))
        return E.item()

    def fd4(f):  # fourth-order central difference of f(t) at t = 0
        return (8.0 * (f(eps) - f(-eps)) - (f(2 * eps) - f(-2 * eps))) / (12.0 * eps)

    dE = fd4(lambda t: energy(C @ expm(t * Y), gam))
    pred = 0.5 * np.sum(g * Y)  # sum over the independent pairs p < q of g_pq Y_pq
    assert abs(dE - pred) < 1e-6 * max(1.0, abs(pred))
    dEg = fd4(lambda t: energy(C, gam + t * dgam))
    assert abs(dEg - gg @ dgam) < 1e-6 * max(1.0, abs(gg @ dgam))
