"""Timing sweep of the digit-plane tensor-core GEMM over the shapes of the JK step's three
contractions (zero operands; measurement only). Prints one markdown table row per case:

    python -m paper_2512_13550_gb300.gemm_sweep

Shapes: the half transform (M = naux nbf rows, N = nact, K = nbf), also with L2 flushed before
each launch (mode flag 4) and with dynamic tiles (mode flag 8), the full transform (M = naux
nact) and the Lagrangian
contraction (M = nbf, N = nact, K = naux nact) of the H50 chain (nbf 150, naux 500, nact 50), a
long-K stream (600000 x 64 x 640) that shows the steady state, and the H200 half transform
(1.2e6 x 208 x 608) with 4 and 5 digits.
"""
from __future__ import annotations

from . import bench_digit_gemm

CASES = [
    # name, M, N, bn, nd, katoms, chunk, mode
    ("H50 half transform, int64 out", 75000, 64, 64, 4, 10, 10, 0),
    ("H50 half transform, scaled out", 75000, 64, 64, 4, 10, 10, 1),
    ("H50 half transform, scaled out, L2 flushed", 75000, 64, 64, 4, 10, 10, 1 + 4),
    ("H50 half transform, scaled out, L2 flushed, dynamic tiles", 75000, 64, 64, 4, 10, 10, 1 + 4 + 8),
    ("H50 full transform, scaled out", 32000, 64, 64, 4, 10, 10, 1),
    ("H50 full transform, scaled out, dynamic tiles", 32000, 64, 64, 4, 10, 10, 1 + 8),
    ("H50 Lagrangian, chunk 16", 150, 50, 64, 4, 2000, 16, 2),
    ("H50 Lagrangian, chunk 32", 150, 50, 64, 4, 2000, 32, 2),
    ("H50 Lagrangian, chunk 32, dynamic tiles", 150, 50, 64, 4, 2000, 32, 2 + 8),
    ("H50 Lagrangian, chunk 64", 150, 50, 64, 4, 2000, 64, 2),
    ("stream 600000 x 64 x 640, BN 64", 600000, 64, 64, 4, 40, 40, 0),
    ("stream 600000 x 64 x 640, BN 32", 600000, 64, 32, 4, 40, 40, 0),
    ("stream 600000 x 64 x 640, BN 16", 600000, 64, 16, 4, 40, 40, 0),
    ("stream 600000 x 64 x 640, 5 digits, BN 32", 600000, 64, 32, 5, 40, 40, 0),
    ("H200 half transform, 5 digits, BN 32", 1200000, 208, 32, 5, 38, 38, 1),
    ("H200 half transform, 5 digits, BN 48", 1200000, 208, 48, 5, 38, 38, 1),
    ("H200 half transform, 5 digits, BN 64 (one TMEM set)", 1200000, 208, 64, 5, 38, 38, 1),
    ("stream 600000 x 64 x 640, 5 digits, BN 64 (one TMEM set)", 600000, 64, 64, 5, 40, 40, 0),
    ("H200 half transform, 4 digits, BN 64", 1200000, 208, 64, 4, 38, 38, 1),
]


def main():
    print("| case | M x N x K | digits | BN | us/launch | MMAs/SM/us | digit-product TFLOP/s |")
    print("|---|---|---|---|---|---|---|")
    for name, M, N, bn, nd, katoms, chunk, mode in CASES:
        us = bench_digit_gemm(M, N, bn, nd, katoms, chunk, mode, reps=10)
        prods = nd * (nd + 1) // 2
        # MMAs per K atom: A plane i meets B planes 0 .. nd - 1 - i two at a time (one MMA of
        # width 2 BN per pair, a single one of width BN for an odd count)
        per_atom = sum((nd - i + 1) // 2 for i in range(nd))
        mmas = ((M + 127) // 128) * ((N + bn - 1) // bn) * katoms * per_atom
        tflops = 2.0 * M * N * katoms * 16 * prods / us / 1e6
        print(f"| {name} | {M} x {N} x {16 * katoms} | {nd} | {bn} | {us:.1f} | {mmas / 152 / us:.1f} | {tflops:.0f} |")


if __name__ == "__main__":
    main()
