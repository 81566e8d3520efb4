"""Bit-exactness of the tcgen05 digit-plane GEMM against a SIMT integer reference."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,katoms,splits", [
    (128, 64, 2, 1),     # one tile, one pipeline stage
    (300, 64, 10, 1),    # ragged M, K = 160 (the exactness limit of one accumulation)
    (128, 16, 5, 1),     # narrowest N, odd atom count (partial last stage)
    (257, 48, 9, 1),     # ragged M, N not a power of two
    (200, 128, 8, 1),    # widest N (512 TMEM columns)
    (256, 64, 20, 4),    # split-K with integer atomics, 5 atoms per chunk
    (300, 64, 12, 1),    # K = 192 > 160: two exact accumulations of 6 atoms summed in the epilogue
    (150, 32, 20, 1),    # K = 320: two parts of 10 atoms
    (256, 64, 24, 2),    # two K parts per tile and split-K atomics together
])
def test_digit_gemm_exact(M, N, katoms, splits):
    import paper_2512_13550_gb300 as nof
    assert nof.selftest_digit_gemm(M, N, katoms, splits, seed=M * 7 + N) == 0
