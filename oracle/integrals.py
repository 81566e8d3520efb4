"""Integrals over contracted s Gaussians (oracle; test infrastructure only).

The paper defines the one-electron integrals h_ki (kinetic energy plus the external potential
of the nuclei) and the two-electron integrals <kl|ij> in its Theory section; it obtains them
from libcint. For s-only Gaussian bases the integrals have closed forms (the standard
Gaussian-product results): with p = a + b, P = (aA + bB)/p, K_AB = exp(-ab/p |A-B|^2),

    overlap      S  = (pi/p)^{3/2} K_AB
    kinetic      T  = (ab/p) (3 - 2 (ab/p) |A-B|^2) S
    nuclear      V  = -Z_C (2 pi / p) K_AB F0(p |P-C|^2)
    repulsion    (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD F0(pq/(p+q) |P-Q|^2)

with F0(t) = (1/2) sqrt(pi/t) erf(sqrt(t)) and F0(0) = 1. The three-centre (ab|c) and
two-centre (c|d) integrals are the repulsion formula with single-Gaussian charge
distributions (q = c, K_CD = 1; p = c, q = d). Primitives are normalised with
(2a/pi)^{3/4}; a contracted function is renormalised after contraction.

Parity: pinned by the textbook H2/STO-3G integrals at R = 1.4 bohr, by the Gaussian
charge-cloud electrostatics identity checked by radial quadrature, and by F0's limits.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def boys_f0(t):
    """F0(t) = int_0^1 exp(-t u^2) du. Series below 1e-8, erf closed form above."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    small = t < 1e-8
    ts = t[small]
    out[small] = 1.0 - ts / 3.0 + ts * ts / 10.0
    tl = t[~small]
    out[~small] = 0.5 * np.sqrt(np.pi / tl) * erf(np.sqrt(tl))
    return out


def _functions(basis, xyz):
    """List of (centre, exponents, coefficients*primitive norms) per basis function."""
    funcs = []
    for A in range(xyz.shape[0]):
        for exps, coefs in basis.shells:
            e = np.array(exps)
            c = np.array(coefs) * (2.0 * e / np.pi) ** 0.75
            funcs.append((xyz[A], e, c))
    # renormalise each contraction: <chi|chi> = sum_ab c_a c_b (pi/(a+b))^{3/2}
    out = []
    for R, e, c in funcs:
        p = e[:, None] + e[None, :]
        s = np.sum(c[:, None] * c[None, :] * (np.pi / p) ** 1.5)
        out.append((R, e, c / np.sqrt(s)))
    return out


def _prim_table(basis, xyz):
    """Flattened primitives: function index, centre, exponent, scaled coefficient."""
    fidx, cen, ex, co = [], [], [], []
    for i, (R, e, c) in enumerate(_functions(basis, xyz)):
        for a, w in zip(e, c):
            fidx.append(i)
            cen.append(R)
            ex.append(a)
            co.append(w)
    return np.array(fidx), np.array(cen), np.array(ex), np.array(co)


def nbf(basis, xyz) -> int:
    return basis.per_atom * xyz.shape[0]


def overlap(basis, xyz):
    """S alone (the first matrix of one_electron) for systems where the nuclear-attraction sum
    over all nuclei is too slow: S_ab = (pi/p)^{3/2} exp(-ab/p |AB|^2) per primitive pair."""
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    AB2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    Sp = (np.pi / p) ** 1.5 * np.exp(-a * b / p * AB2)
    S = np.zeros((n, n))
    np.add.at(S, (fi[:, None], fi[None, :]), co[:, None] * co[None, :] * Sp)
    return S


def kinetic(basis, xyz):
    """T alone (the second matrix of one_electron): T_ab = mu (3 - 2 mu |AB|^2) S_ab per primitive
    pair, mu = ab/p."""
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    mu = a * b / p
    AB2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    Tp = mu * (3.0 - 2.0 * mu * AB2) * (np.pi / p) ** 1.5 * np.exp(-mu * AB2)
    T = np.zeros((n, n))
    np.add.at(T, (fi[:, None], fi[None, :]), co[:, None] * co[None, :] * Tp)
    return T


def nuclear_attraction(basis, xyz, Z=None, centres=None):
    """The nuclear-attraction part of one_electron's V from the nuclei listed in `centres` only
    (all by default): V_ab = -sum_C Z_C (2 pi / p) K_AB F0(p |PC|^2) per primitive pair. Summed over
    a partition of the nuclei it gives V (the sum over C split into slices)."""
    natom = xyz.shape[0]
    Z = np.ones(natom) if Z is None else np.asarray(Z, np.float64)
    centres = range(natom) if centres is None else centres
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    Kab = np.exp(-a * b / p * np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1))
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    Vp = np.zeros_like(Kab)
    for C in centres:
        PC2 = np.sum((Pc - xyz[C]) ** 2, axis=-1)
        Vp += -Z[C] * (2.0 * np.pi / p) * Kab * boys_f0(p * PC2)
    V = np.zeros((n, n))
    np.add.at(V, (fi[:, None], fi[None, :]), co[:, None] * co[None, :] * Vp)
    return V


def one_electron(basis, xyz, Z=None):
    """S, T and V (nuclear attraction of all nuclei) as n x n FP64 matrices."""
    natom = xyz.shape[0]
    Z = np.ones(natom) if Z is None else np.asarray(Z, np.float64)
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    mu = a * b / p
    AB2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    Kab = np.exp(-mu * AB2)
    Sp = (np.pi / p) ** 1.5 * Kab
    Tp = mu * (3.0 - 2.0 * mu * AB2) * Sp
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    Vp = np.zeros_like(Sp)
    for C in range(natom):
        PC2 = np.sum((Pc - xyz[C]) ** 2, axis=-1)
        Vp += -Z[C] * (2.0 * np.pi / p) * Kab * boys_f0(p * PC2)
    w = co[:, None] * co[None, :]
    S = np.zeros((n, n)); T = np.zeros((n, n)); V = np.zeros((n, n))
    np.add.at(S, (fi[:, None], fi[None, :]), w * Sp)
    np.add.at(T, (fi[:, None], fi[None, :]), w * Tp)
    np.add.at(V, (fi[:, None], fi[None, :]), w * Vp)
    return S, T, V


def nuclear_repulsion(xyz, Z=None) -> float:
    natom = xyz.shape[0]
    Z = np.ones(natom) if Z is None else np.asarray(Z, np.float64)
    e = 0.0
    for A in range(natom):
        for B in range(A + 1, natom):
            e += Z[A] * Z[B] / np.linalg.norm(xyz[A] - xyz[B])
    return e


def _aux_table(aux, xyz):
    """Aux functions are uncontracted primitives; returns centre, exponent, norm."""
    cen, ex, nm = [], [], []
    for A in range(xyz.shape[0]):
        for exps, _ in aux.shells:
            for e in exps:
                cen.append(xyz[A]); ex.append(e); nm.append((2.0 * e / np.pi) ** 0.75)
    return np.array(cen), np.array(ex), np.array(nm)


def naux(aux, xyz) -> int:
    return sum(len(e) for e, _ in aux.shells) * xyz.shape[0]


def two_center(aux, xyz):
    """Coulomb metric V_PQ = (P|Q), X x X."""
    cen, ex, nm = _aux_table(aux, xyz)
    p = ex[:, None]; q = ex[None, :]
    R2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    pre = 2.0 * np.pi ** 2.5 / (p * q * np.sqrt(p + q))
    return nm[:, None] * nm[None, :] * pre * boys_f0(p * q / (p + q) * R2)


def three_center(basis, aux, xyz, P_slice=None):
    """(P|mu nu) as an array [X][n][n] (or the rows P_slice of it)."""
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    acen, aex, anm = _aux_table(aux, xyz)
    if P_slice is not None:
        acen, aex, anm = acen[P_slice], aex[P_slice], anm[P_slice]
    a = ex[:, None]; b = ex[None, :]
    p = a + b
    Kab = np.exp(-a * b / p * np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1))
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    w = co[:, None] * co[None, :] * Kab
    out = np.zeros((len(aex), n, n))
    for k in range(len(aex)):
        q = aex[k]
        PQ2 = np.sum((Pc - acen[k]) ** 2, axis=-1)
        val = anm[k] * w * 2.0 * np.pi ** 2.5 / (p * q * np.sqrt(p + q)) * boys_f0(p * q / (p + q) * PQ2)
        blk = np.zeros((n, n))
        np.add.at(blk, (fi[:, None], fi[None, :]), val)
        out[k] = blk
    return out


def four_center(basis, xyz):
    """Exact (mu nu|lam sig), n^4 array. Tiny systems only."""
    fi, cen, ex, co = _prim_table(basis, xyz)
    n = nbf(basis, xyz)
    npr = len(ex)
    a = ex[:, None]; b = ex[None, :]
    p = a + b
    Kab = np.exp(-a * b / p * np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1))
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    w = co[:, None] * co[None, :] * Kab
    P1 = p.reshape(npr * npr); W1 = w.reshape(npr * npr); C1 = Pc.reshape(npr * npr, 3)
    pp = P1[:, None]; qq = P1[None, :]
    R2 = np.sum((C1[:, None, :] - C1[None, :, :]) ** 2, axis=-1)
    val = W1[:, None] * W1[None, :] * 2.0 * np.pi ** 2.5 / (pp * qq * np.sqrt(pp + qq)) \
        * boys_f0(pp * qq / (pp + qq) * R2)
    val = val.reshape(npr, npr, npr, npr)
    out = np.zeros((n, n, n, n))
    np.add.at(out, (fi[:, None, None, None], fi[None, :, None, None],
                    fi[None, None, :, None], fi[None, None, None, :]), val)
    return out
