"""The tcgen05 digit-plane GEMM against a SIMT integer reference.

Digits lie in [-128, 128], the leading one in [-256, 256] with 4 digits. The leading levels 0 .. nd - 3 of every accumulation are exact; the
last two levels may round once a part's FP32 sum passes 2^24. The bound below counts one FP32
rounding (half an ulp of the largest possible partial sum, taken as a whole ulp for the tensor
core's internal sum) per accumulation into those levels, weighted by the level's place in V. With
random digits the sums stay far below 2^24, so the results are bit-identical in practice."""
import math

import pytest

pytestmark = pytest.mark.gpu


def _bound(nd, katoms):
    amax = 20 if nd == 5 else 16             # atoms per accumulation
    top = [128 if nd == 5 else 256] + [128] * (nd - 1)  # largest |digit| per plane
    total = 0
    for lvl in range(nd - 2, nd):  # the two levels allowed to round
        smax = amax * 16 * sum(top[i] * top[lvl - i] for i in range(lvl + 1))
        ulp = 2 ** max(0, math.ceil(math.log2(smax)) - 24)
        total += katoms * (lvl + 1) * ulp * 256 ** (nd - 1 - lvl)
    return total


@pytest.mark.parametrize("M,N,bn,katoms,chunk,nd", [
    (128, 64, 64, 2, 2, 4),      # one tile, one pipeline stage
    (300, 64, 64, 10, 10, 4),    # ragged M, K = 160 (one part)
    (128, 16, 16, 5, 5, 4),      # narrowest tile, odd atom count (partial last stage)
    (257, 48, 16, 9, 9, 4),      # three N tiles of 16
    (257, 48, 32, 9, 9, 4),      # ragged last N tile (48 = 32 + 16 valid of 32)
    (257, 48, 64, 9, 9, 4),      # one N tile, 16 padding columns
    (200, 208, 64, 8, 8, 4),     # four N tiles, the last one 16 of 64 columns
    (256, 64, 64, 20, 5, 4),     # split-K with integer atomics, 5 atoms per chunk
    (300, 64, 32, 12, 12, 4),    # K = 192: one part
    (150, 32, 32, 38, 38, 4),    # K = 608: three parts (14, 14, 10), like nbf = 600
    (256, 80, 16, 24, 14, 4),    # split-K with a ragged last chunk (14 + 10)
    (130, 96, 64, 63, 63, 4),    # four parts (16, 16, 16, 15; K = 1008 like nbf = 1000), two N tiles
    (128, 32, 32, 8, 8, 5),      # 5 digits: 15 products, one part of 8 atoms
    (300, 80, 16, 38, 38, 5),    # 5 digits, two parts (20 + 18), five N tiles
    (257, 64, 32, 24, 9, 5),     # 5 digits, split-K with ragged chunks (9, 9, 6) and two N tiles
    (130, 208, 32, 63, 63, 5),   # 5 digits, K = 1008 (four parts of 16), seven N tiles
    (300, 208, 64, 38, 38, 5),   # 5 digits, BN 64 with one TMEM set (two parts drained in turn)
    (256, 64, 64, 24, 10, 5),    # 5 digits, BN 64, one TMEM set, split-K (chunks 10, 10, 4)
    (300, 208, 48, 38, 38, 5),   # 5 digits, BN 48 (24-column halves: chunks of 16 and 8), five tiles
    (257, 100, 48, 12, 12, 4),   # 4 digits, BN 48, ragged last tile (100 = 2 x 48 + 4)
    (300, 64, 32, 70, 70, 4),    # 4 digits, K = 1120: five parts of 14
    (256, 48, 48, 41, 41, 5),    # 5 digits, K = 656: three parts (14 + 14 + 13), odd count
    (300, 208, 80, 38, 38, 5),   # 5 digits, BN 80 (40-column halves), one TMEM set, ragged last tile
    (257, 100, 80, 24, 9, 4),    # 4 digits, BN 80, split-K (9, 9, 6), ragged last tile (100 = 80 + 20)
    (130, 1000, 80, 60, 60, 5),  # 5 digits, BN 80, 13 N tiles (the last 40 of 80), three scale parts
    (257, 100, 80, 24, 24, 4),   # 4 digits, BN 80, three scale parts of 8 atoms
    (300, 208, 96, 38, 38, 5),   # 5 digits, BN 96 (48-column halves), last tile 16 of 96 columns
    (130, 1000, 96, 80, 80, 5),  # 5 digits, BN 96, 11 N tiles, four scale parts
    (257, 100, 96, 24, 9, 4),    # 4 digits, BN 96, split-K (9, 9, 6)
])
def test_digit_gemm_exact(M, N, bn, katoms, chunk, nd):
    """The int64 output (single CTAs, round-robin and dynamic tiles) within the last levels' rounding
    of the exact V; with one K chunk and an even N, the scaled double-float output too, and with K in
    whole scale parts the per-part FP64 output (the self-test reports 2^62 if either is off)."""
    import paper_2512_13550_gb300 as nof
    assert 0 <= nof.selftest_digit_gemm(M, N, bn, katoms, chunk, seed=M * 7 + N + bn, nd=nd) <= _bound(nd, katoms)
