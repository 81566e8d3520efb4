"""Bit-exactness of the tcgen05 digit-plane GEMM against a SIMT integer reference."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,bn,katoms,chunk,nd", [
    (128, 64, 64, 2, 2, 4),      # one tile, one pipeline stage
    (300, 64, 64, 10, 10, 4),    # ragged M, K = 160 (the exactness limit of one accumulation)
    (128, 16, 16, 5, 5, 4),      # narrowest tile, odd atom count (partial last stage)
    (257, 48, 16, 9, 9, 4),      # three N tiles of 16
    (257, 48, 32, 9, 9, 4),      # ragged last N tile (48 = 32 + 16 valid of 32)
    (257, 48, 64, 9, 9, 4),      # one N tile, 16 padding columns
    (200, 208, 64, 8, 8, 4),     # four N tiles, the last one 16 of 64 columns
    (256, 64, 64, 20, 5, 4),     # split-K with integer atomics, 5 atoms per chunk
    (300, 64, 32, 12, 12, 4),    # K = 192: two exact parts (10 + 2) summed in the epilogue
    (150, 32, 32, 38, 38, 4),    # K = 608: four parts (10, 10, 10, 8), like nbf = 600
    (256, 80, 16, 24, 14, 4),    # split-K with a ragged last chunk (14 + 10) and two parts per chunk
    (130, 96, 64, 63, 63, 4),    # seven parts (K = 1008, like nbf = 1000), two N tiles
    (128, 32, 32, 8, 8, 5),      # 5 digits: 15 products, one part of 8 atoms
    (300, 80, 16, 38, 38, 5),    # 5 digits, five parts (8 + 8 + 8 + 8 + 6), five N tiles
    (257, 64, 32, 24, 9, 5),     # 5 digits, split-K with ragged chunks (9, 9, 6) and two N tiles
    (130, 208, 32, 63, 63, 5),   # 5 digits, K = 1008 (eight parts), seven N tiles
    (300, 208, 64, 38, 38, 5),   # 5 digits, BN 64 with one TMEM set (five parts drained in turn)
    (256, 64, 64, 24, 10, 5),    # 5 digits, BN 64, one TMEM set, split-K (chunks 10, 10, 4)
    (300, 208, 48, 38, 38, 5),   # 5 digits, BN 48 (24-column halves: chunks of 16 and 8), five tiles
    (257, 100, 48, 12, 12, 4),   # 4 digits, BN 48, ragged last tile (100 = 2 x 48 + 4)
])
def test_digit_gemm_exact(M, N, bn, katoms, chunk, nd):
    import paper_2512_13550_gb300 as nof
    assert nof.selftest_digit_gemm(M, N, bn, katoms, chunk, seed=M * 7 + N + bn, nd=nd) == 0
