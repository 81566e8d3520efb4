"""Nuclear gradient on the GPU (FP64 path) against the oracle, at arbitrary states (C, gamma) on
non-collinear geometries; translation and rotation invariance; split-precision contexts refuse."""
import numpy as np
import pytest

from oracle import gradient, integrals, pnof, reference
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _geometry(natom, seed):
    xyz = inputs.chain(natom, 1.6)
    return xyz + inputs.uniform(seed, natom * 3, -0.35, 0.35).reshape(natom, 3)


@pytest.mark.parametrize("natom,basis,ncwo,ipnof", [
    (4, "h4", 1, 7), (4, "h4", 1, 5), (4, "et2", 2, 7), (8, "3s10aux", 1, 7)])
def test_nuclear_gradient_matches_oracle(natom, basis, ncwo, ipnof):
    import paper_2512_13550_gb300 as nof
    if basis == "h4":
        orb, aux = inputs.basis_h4()
    elif basis == "et2":
        orb, aux = inputs.Basis(inputs.even_tempered_shells(0.3, 4.0, 2)), inputs.basis_h4()[1]
    else:
        orb, aux = inputs.basis_3s_10aux()
    xyz = _geometry(natom, 11 + natom)
    S, _, _ = integrals.one_electron(orb, xyz)
    n = S.shape[0]
    pm = pnof.PairMap(natom, ncwo, n)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 21))
    gam = inputs.random_gamma(pm.ngamma, 22)
    want = gradient.nuclear_gradient(orb, aux, xyz, C, gam, pm, ipnof=ipnof)
    ctx = nof.Context(precision=nof.PREC_FP64, ncwo=ncwo, ipnof=ipnof)
    ctx.build_B(xyz, orb, aux)
    for _ in range(2):  # the second call reuses the workspaces
        got = ctx.nuclear_gradient(_t(C), _t(gam)).cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
    np.testing.assert_allclose(got.sum(axis=0), 0.0, atol=1e-9)
    np.testing.assert_allclose(np.cross(xyz, got).sum(axis=0), 0.0, atol=1e-9)


def test_split_precision_context_refuses():
    import paper_2512_13550_gb300 as nof
    orb, aux = inputs.basis_h4()
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16)
    ctx.build_B(_geometry(4, 3), orb, aux)
    n, ng = ctx.sizes["nbf"], ctx.sizes["ngamma"]
    with pytest.raises(nof.NofError) as e:
        ctx.nuclear_gradient(_t(np.eye(n)), _t(np.zeros(ng)))
    assert e.value.code == nof.NOF_EINVAL
