"""Core-Hamiltonian guess on the device (Jacobi eigensolver) against the oracle's library eigh."""
import numpy as np
import pytest

import systems
from oracle import pnof, reference

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("natom", [10, 50])
def test_core_guess(natom):
    import paper_2512_13550_gb300 as nof
    sysm = systems.chain3s(natom)
    o = sysm.oracle
    ctx = nof.Context(precision=0)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    C, eps = ctx.core_guess()
    torch.cuda.synchronize()
    C, eps = C.cpu().numpy(), eps.cpu().numpy()
    S, H = o["S"], o["H"]
    X = reference.lowdin(S)
    w_ref = np.linalg.eigvalsh(X.T @ H @ X)
    np.testing.assert_allclose(eps, w_ref, atol=1e-10)
    np.testing.assert_allclose(C.T @ S @ C, np.eye(o["n"]), atol=1e-10)
    np.testing.assert_allclose(C.T @ H @ C, np.diag(w_ref), atol=1e-9)
    # the occupied space (no degeneracy at the Fermi level) fixes the RHF energy
    e_dev = reference.rhf_energy_ao(o["B"], H, C, natom // 2, o["vnn"])
    e_ref = reference.rhf_energy_ao(o["B"], H, reference.core_guess(S, H), natom // 2, o["vnn"])
    assert abs(e_dev - e_ref) < 1e-9
