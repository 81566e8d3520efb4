"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's tests.

This module generates *inputs only*: random numbers, hydrogen geometries, s-only basis
specifications, random orthogonal matrices and starting occupation angles. It holds none of
the method's arithmetic (no integrals, no fitting, no functional, no gradient), so the CUDA
path and the CPU oracle can both consume identical bytes without sharing any computation.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of stream `seed` is
mix64(seed + (i + 1) * 0x9E3779B97F4A7C15). Normals use the Box-Muller transform.

Workload recipes (hydrogen systems standing in for the paper's Gaussian-basis molecules):
  * H4 chain, spacing 1.8 bohr, one 3-primitive contracted s per H (STO-3G-like fit, zeta=1.24),
    8 even-tempered aux s per H (alpha = 0.1 * 3^k).
  * H50 chain, spacing 1.8 + U(-0.1, 0.1) bohr per bond, 3 even-tempered s per H
    (alpha = 0.2 * 4^k) and 10 aux s per H (alpha = 0.1 * 3^k).
  * H200 10 x 20 square lattice, spacing 2.0 bohr, same basis as H50.
  * Batches of H8..H64 chains (even N), Gaussian displacements sigma = 0.05 bohr.
  * H1000 chain, spacing 1.8 bohr, the contracted s per H and 3 aux s per H.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based splitmix64: element i is mix64(seed + (offset + i + 1) * golden)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of splitmix64."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller over consecutive pairs of uniforms."""
    m = (count + 1) // 2
    u = (splitmix64(seed, 2 * m) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# ----------------------------------------------------------------------------------------
# Basis specifications: a shell is (exponents, contraction coefficients). All s type.
# ----------------------------------------------------------------------------------------

# Hehre-Stewart-Pople STO-3G least-squares fit of a zeta = 1 Slater 1s (textbook constants).
_STO3G_EXP = (0.109818, 0.405771, 2.227660)
_STO3G_COEF = (0.444635, 0.535328, 0.154329)


def sto3g_like_shell(zeta: float = 1.24):
    return (tuple(e * zeta * zeta for e in _STO3G_EXP), _STO3G_COEF)


def even_tempered_shells(alpha0: float, beta: float, count: int):
    return [((alpha0 * beta ** k,), (1.0,)) for k in range(count)]


class Basis:
    """Per-atom list of contracted s shells, identical on every hydrogen."""

    def __init__(self, shells):
        self.shells = [(tuple(map(float, e)), tuple(map(float, c))) for e, c in shells]

    @property
    def per_atom(self) -> int:
        return len(self.shells)

    def flat(self, natom: int):
        """Flattened arrays for the C ABI: per function (atom index, first primitive, nprim)
        plus primitive exponent and coefficient arrays. Functions are ordered atom-major."""
        fn_atom, fn_first, fn_nprim, pexp, pcoef = [], [], [], [], []
        for A in range(natom):
            for e, c in self.shells:
                fn_atom.append(A)
                fn_first.append(len(pexp))
                fn_nprim.append(len(e))
                pexp.extend(e)
                pcoef.extend(c)
        return (np.array(fn_atom, np.int32), np.array(fn_first, np.int32),
                np.array(fn_nprim, np.int32), np.array(pexp, np.float64),
                np.array(pcoef, np.float64))


def basis_h4():
    return Basis([sto3g_like_shell(1.24)]), Basis(even_tempered_shells(0.1, 3.0, 8))


def basis_3s_10aux():
    return Basis(even_tempered_shells(0.2, 4.0, 3)), Basis(even_tempered_shells(0.1, 3.0, 10))


def basis_h1000():
    return Basis([sto3g_like_shell(1.24)]), Basis(even_tempered_shells(0.1, 3.0, 3))


# ----------------------------------------------------------------------------------------
# Geometries (bohr), hydrogen only (Z = 1).
# ----------------------------------------------------------------------------------------

def chain(natom: int, spacing: float = 1.8) -> np.ndarray:
    xyz = np.zeros((natom, 3))
    xyz[:, 2] = spacing * np.arange(natom)
    return xyz


def jittered_chain(natom: int, seed: int, spacing: float = 1.8, jitter: float = 0.1) -> np.ndarray:
    bonds = spacing + uniform(seed, natom - 1, -jitter, jitter)
    xyz = np.zeros((natom, 3))
    xyz[1:, 2] = np.cumsum(bonds)
    return xyz


def lattice(nx: int = 10, ny: int = 20, spacing: float = 2.0) -> np.ndarray:
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    xyz = np.zeros((nx * ny, 3))
    xyz[:, 0] = spacing * ix.ravel()
    xyz[:, 1] = spacing * iy.ravel()
    return xyz


def displaced_chain(natom: int, seed: int, sigma: float = 0.05, spacing: float = 1.8) -> np.ndarray:
    return chain(natom, spacing) + sigma * normal(seed, 3 * natom).reshape(natom, 3)


def batch_sizes(count: int = 256, seed: int = 3, lo: int = 8, hi: int = 64) -> np.ndarray:
    """Even chain lengths drawn uniformly from {lo, lo+2, ..., hi}."""
    choices = np.arange(lo, hi + 1, 2)
    idx = (splitmix64(seed, count) % np.uint64(len(choices))).astype(np.int64)
    return choices[idx]


def batch_geometries(count: int = 256, size_seed: int = 3, disp_seed: int = 4):
    sizes = batch_sizes(count, size_seed)
    return [displaced_chain(int(N), disp_seed * 1000003 + i) for i, N in enumerate(sizes)]


# ----------------------------------------------------------------------------------------
# Orbital / occupation inputs.
# ----------------------------------------------------------------------------------------

def random_orthogonal(n: int, seed: int = 0) -> np.ndarray:
    """Q from the QR factorisation of an n x n N(0,1) matrix, columns signed so diag(R) > 0."""
    G = normal(seed, n * n).reshape(n, n)
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def random_antisymmetric(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    G = normal(seed, n * n).reshape(n, n)
    return scale * (np.triu(G, 1) - np.triu(G, 1).T)


def random_gamma(count: int, seed: int = 1, lo: float = 0.1, hi: float = 1.2) -> np.ndarray:
    return uniform(seed, count, lo, hi)
