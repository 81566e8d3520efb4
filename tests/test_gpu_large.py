"""Full-size parity on the H200 lattice (10 x 20, spacing 2.0 bohr, 3 s + 10 aux s per H:
nbf 600, naux 2000, nact 200) through the C ABI, split-precision and FP64 paths, against the
oracle's orbital-basis route (oracle/large.py, pinned to the plain route), whose three-centre
integrals are generated in parallel slices by spawned processes."""
import numpy as np
import pytest

import oracle_pool
from oracle import integrals, large, pnof, reference
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-6


@pytest.fixture(scope="module")
def h200():
    orb, aux = inputs.basis_3s_10aux()
    xyz = inputs.lattice(10, 20, 2.0)
    S, T, V = integrals.one_electron(orb, xyz)
    n = S.shape[0]
    pm = pnof.PairMap(xyz.shape[0], 1, n)
    C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 0))
    gam = inputs.random_gamma(pm.ngamma, 1)
    bfull = oracle_pool.fitted_mo(orb, aux, xyz, C, pm.nact)
    ref = large.energy_and_gradients_mo(bfull, T + V, C, gam, pm, integrals.nuclear_repulsion(xyz))
    return dict(orb=orb, aux=aux, xyz=xyz, C=C, gam=gam, ref=ref)


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [1, 0])
def test_h200_energy_gradients(h200, precision):
    import paper_2512_13550_gb300 as nof
    ctx = nof.Context(precision=precision)
    ctx.build_B(h200["xyz"], h200["orb"], h200["aux"])
    assert (ctx.sizes["nbf"], ctx.sizes["naux"], ctx.sizes["nact"]) == (600, 2000, 200)
    C, gam = _t(h200["C"]), _t(h200["gam"])
    J, K = ctx.jk(C)
    E, g, gg = ctx.energy_grad(C, gam)
    torch.cuda.synchronize()
    ref = h200["ref"]
    assert abs(E.item() - ref["E"]) < GATE
    assert np.max(np.abs(J.cpu().numpy() - ref["J"])) < GATE
    assert np.max(np.abs(K.cpu().numpy() - ref["K"])) < GATE
    assert np.max(np.abs(g.cpu().numpy() - ref["g"])) < GATE
    assert np.max(np.abs(gg.cpu().numpy() - ref["g_gamma"])) < GATE
    if precision == 1:
        bn1, bn2, bn3, chunk = ctx.tuned_tiles()
        assert {bn1, bn2, bn3} <= {16, 32, 48, 64, 80, 96} and chunk >= 8
    ctx.close()
