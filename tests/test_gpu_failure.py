"""Failure detection on the GPU without a fault: bounded device waits that run out, and non-finite
inputs, each reported as a status the host reads, with the device still usable afterwards."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nd,bn", [(4, 64), (5, 48)])
def test_digit_gemm_wait_limit_reports_timeout(nd, bn):
    """A digit GEMM launch whose producer issues no copies: its MMA warp's wait for the first
    stage, the producer's wait for a free slot and the epilogue's wait for an accumulator run out
    at the 2 ms limit; the call returns NOF_ETIMEOUT within milliseconds and the next launches are
    correct."""
    import paper_2512_13550_gb300 as nof
    lib = nof.load_library()
    ms = ctypes.c_double(-1.0)
    rc = lib.nof_selftest_digit_gemm_timeout(1024, 128, bn, nd, 16, 2.0, ctypes.byref(ms))
    assert rc == nof.NOF_ETIMEOUT, lib.nof_last_error()
    assert b"timed out" in lib.nof_last_error()
    assert 1.9 <= ms.value < 100.0
    # the device is still usable: the same product with its copies is exact
    assert nof.selftest_digit_gemm(1024, 128, bn, 16, 16, seed=5, nd=nd) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_gamma_is_reported(precision):
    """A NaN occupation angle reaches the energy: nof_sync returns NOF_ENONFINITE once, then the
    status word is clear and a finite evaluation follows."""
    import paper_2512_13550_gb300 as nof
    from oracle import integrals, reference
    from paper_2512_13550_gb300 import inputs
    orb, aux = inputs.basis_3s_10aux()
    xyz = inputs.chain(6, 1.8)
    ctx = nof.Context(precision=precision)
    ctx.build_B(xyz, orb, aux)
    S = integrals.overlap(orb, xyz)
    C = torch.tensor(reference.orthonormal_orbitals(S, inputs.random_orthogonal(S.shape[0], 2)),
                     dtype=torch.float64, device="cuda")
    gam = np.full(ctx.sizes["ngamma"], 0.4)
    gam[1] = np.nan
    ctx.energy_grad(C, torch.tensor(gam, dtype=torch.float64, device="cuda"))
    with pytest.raises(nof.NofError) as ei:
        ctx.sync()
    assert ei.value.code == nof.NOF_ENONFINITE
    ctx.sync()
    gam[1] = 0.4
    E, _, _ = ctx.energy_grad(C, torch.tensor(gam, dtype=torch.float64, device="cuda"))
    ctx.sync()
    assert np.isfinite(E.item())
    ctx.close()
