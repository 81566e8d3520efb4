"""The allocation-free JK entry point (nof_jk_static) against the context-based nof_jk.

nof_jk_static serves callers that cannot call cudaMalloc (their device memory belongs to
another allocator, or an allocation must not stall or fail mid-run): it keeps its scratch in a
fixed array inside the library. This file is collected last so that a failure here leaves every
other test already run; it must pass alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 on both sides, the same kernels' arithmetic


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("make", [lambda: systems.chain3s(10), systems.h50])
def test_jk_static_matches_nof_jk_on_two_calls(make):
    import paper_2512_13550_gb300 as nof
    lib = nof.load_library()
    sysm = make()
    ctx = nof.Context(precision=nof.PREC_FP64)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    s = ctx.sizes
    X, n, a = s["naux"], s["nbf"], s["nact"]
    B = ctx.get_B()
    stream = torch.cuda.current_stream()
    # every tensor of both calls exists before the first call, so that free device memory can only
    # change inside the library
    Cs = [_t(sysm.orbitals(seed)) for seed in (0, 7)]  # two calls in a row, different orbitals
    refs = [ctx.jk(C) for C in Cs]
    outs = [(torch.full((a, a), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((a, a), float("nan"), dtype=torch.float64, device="cuda")) for _ in Cs]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    for C, (J0, K0), (J, K) in zip(Cs, refs, outs):
        rc = lib.nof_jk_static(X, n, a, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                               ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(K.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream))
        assert rc == nof.NOF_OK, lib.nof_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert torch.max(torch.abs(J - J0)).item() < TOL
        assert torch.max(torch.abs(K - K0)).item() < TOL
    # the call after the first allocates nothing; the first may reserve the fixed array (the
    # library's module loads lazily) and never more than the array plus its module's code
    assert free[2] == free[1]
    first = free[0] - free[1]
    print(f"free device memory taken by the first call: {first / 2**20:.1f} MiB")
    assert 0 <= first <= 64 * 2**20


def test_jk_static_rejects_sizes_beyond_its_scratch():
    import paper_2512_13550_gb300 as nof
    lib = nof.load_library()
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    # 2000 * 600 * 200 doubles is far beyond the 48 MiB array: refused before any launch
    rc = lib.nof_jk_static(2000, 600, 200, p, p, p, p, None)
    assert rc == nof.NOF_EINVAL
    assert b"exceeds" in lib.nof_last_error()
