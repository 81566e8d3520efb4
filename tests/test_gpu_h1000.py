"""The H1000 chain (spacing 1.8 bohr, 1 contracted s + 3 aux s per H: nbf 1000, naux 3000,
nact 1000) on the split path, checked by properties that hold at any size (the oracle's
integrals are too slow at this size): the invariants of J and K, and the orbital and occupation
gradients against fourth-order finite differences of the energy. The orbitals are the oracle's
Loewdin orbitals of its overlap matrix."""
import numpy as np
import pytest

from oracle import integrals, reference
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h1000():
    import paper_2512_13550_gb300 as nof
    orb, aux = inputs.basis_h1000()
    xyz = inputs.chain(1000, 1.8)
    S = integrals.overlap(orb, xyz)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(S.shape[0], 0))
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16)
    ctx.build_B(xyz, orb, aux)
    return dict(ctx=ctx, C=C, n=S.shape[0])


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_h1000_jk_invariants(h1000):
    ctx = h1000["ctx"]
    assert (ctx.sizes["nbf"], ctx.sizes["naux"], ctx.sizes["nact"]) == (1000, 3000, 1000)
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
