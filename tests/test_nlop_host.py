"""The host-side NLOP entry points of the C ABI (no device work, no GPU): centred differences
and the Romberg-Richardson triangle against the oracle on the same inputs."""
import numpy as np
import pytest

from oracle import nlop as onlop
from paper_2512_13550_gb300 import inputs

nof = pytest.importorskip("paper_2512_13550_gb300")


@pytest.fixture(scope="module")
def lib():
    try:
        return nof.load_library()
    except ImportError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("npoint", [1, 4, 9])
def test_field_differences_match_oracle(lib, npoint):
    step = 1e-3
    fields = onlop.field_points(step, npoint)
    vals = inputs.uniform(11 + npoint, fields.size, -1.0, 1.0)
    mu = dict(zip(fields, vals))
    want = onlop.differences(mu, step, npoint)
    got = nof.field_differences(vals, npoint, step)
    for w, g in zip(want, got):
        np.testing.assert_allclose(g, w, rtol=1e-14, atol=0)


@pytest.mark.parametrize("N", [1, 2, 5, 9])
def test_romberg_matches_oracle(lib, N):
    for seed in range(4):
        D = inputs.uniform(30 + seed + 7 * N, N, -5.0, 5.0)
        Rw, bw = onlop.romberg(D)
        Rg, bg = nof.romberg(D)
        np.testing.assert_array_equal(np.isnan(Rg), np.isnan(Rw))
        np.testing.assert_allclose(Rg[~np.isnan(Rw)], Rw[~np.isnan(Rw)], rtol=1e-15, atol=0)
        assert bg[2:] == bw[2:]
        assert bg[0] == bw[0] and (np.isnan(bw[1]) and np.isnan(bg[1]) or bg[1] == bw[1])
    # the tie rule on the hand-made case of the oracle's pins
    _, b = nof.romberg([-2.0, -1.0, 0.0, 7.0])
    assert b[2:] == (2, 1)


def test_host_entry_points_reject_bad_arguments(lib):
    d = np.zeros(4)
    p = d.ctypes.data_as(__import__("ctypes").c_void_p)
    assert lib.nof_romberg(p, 0, p, p, p) == nof.NOF_EINVAL
    assert lib.nof_romberg(None, 3, p, p, p) == nof.NOF_EINVAL
    assert lib.nof_field_differences(p, 0, 1e-3, p, p, p) == nof.NOF_EINVAL
    assert lib.nof_field_differences(p, 1, -1.0, p, p, p) == nof.NOF_EINVAL
    assert lib.nof_set_field(None, p) == nof.NOF_EINVAL
    assert lib.nof_dipole(None, p, p, p) == nof.NOF_EINVAL
    assert lib.nof_step_batch(None, 0, None, None, None, None, None, None, None) == nof.NOF_EINVAL


def test_polarizability_invariants_match_oracle(lib):
    for seed in range(5):
        a = inputs.uniform(70 + seed, 3, 0.5, 9.0)
        got = nof.polarizability_invariants(*a)
        want = onlop.polarizability_invariants(*a)
        assert abs(got[0] - want[0]) < 1e-15 * abs(want[0]) + 1e-300
        assert abs(got[1] - want[1]) < 1e-14 * max(1.0, want[1])
