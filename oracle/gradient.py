"""Nuclear gradient of the RI-PNOF energy for s-only bases (oracle; test infrastructure only).

The paper lists analytic nuclear gradients among DoNOF's capabilities (geometry optimisation and
the molecular-dynamics interface) without printing them; they follow from the energy it defines
(Eq. PNOF with the RI integrals of the Single Point Energy section):

    E = sum_p n_p 2 h_pp + sum_pq (A_pq J_pq - B_pq K_pq) + V_nn,
    J_pq = sum_PQ (pp|P) (V^-1)_PQ (Q|qq),   K_pq = sum_PQ (pq|P) (V^-1)_PQ (Q|pq).

Reading (the paper gives no formula): the orbitals follow the geometry through the Loewdin-type
connection C(x) = C0 (C0^T S(x) C0)^{-1/2}, which keeps them S(x)-orthonormal. With
dC/dx = -C0 M^x / 2 at x0 (M^x = C0^T S^x C0) and dE/dC = 4 Lambda (so that C^T dE/dC = 4 lambda,
the Lagrangian of the Natural Orbital Optimization subsection), at any (C, gamma):

    dE/dx = sum_uv P_uv h^x_uv - 2 sum_uv (C lambda C^T)_uv S^x_uv
            + sum_P sum_uv Gamma^P_uv (uv|P)^x - sum_PQ Z_PQ V^x_PQ + V_nn^x,

with P = 2 C diag(n) C^T (active columns), c^P_pq = sum_Q (V^-1)_PQ (Q|pq),
Y^P_pq = 2 delta_pq sum_r A_pr c^P_rr - 2 B_pq c^P_pq, Gamma^P = C Y^P C^T and
Z_PQ = sum_pq (A_pq c^P_pp c^Q_qq - B_pq c^P_pq c^Q_pq). At a converged state (lambda
symmetric, dE/dgamma = 0) this is the physical gradient.

Integral derivatives of s Gaussians (p = a + b, mu = ab/p, P = (aA + bB)/p, K = exp(-mu |A-B|^2),
F1(t) = -dF0/dt):
    dS/dA = -2 mu (A-B) S;  dT/dA = -2 mu^2 (A-B) (5 - 2 mu |A-B|^2) S;
    V^C = -Z_C (2 pi/p) K F0(t), t = p|P-C|^2:  dV/dA = -Z_C (2 pi/p) (-2 mu (A-B) K F0 - 2a K F1 (P-C)),
        dV/dC = -Z_C (2 pi/p) 2p K F1 (P-C);
    (ab|c) = N 2 pi^{5/2} / (p c sqrt(p+c)) K F0(rho |P-C|^2), rho = pc/(p+c):
        d/dA = N pre (-2 mu (A-B) K F0 - 2 rho (a/p) K F1 (P-C)),  d/dC = N pre 2 rho K F1 (P-C);
    (c|d) = N N' 2 pi^{5/2} / (c d sqrt(c+d)) F0(rho' |C-D|^2): d/dC = -N N' pre 2 rho' F1 (C-D);
the derivative with respect to B follows by symmetry, and every integral is translation
invariant (the derivatives over its centres sum to zero).

Parity: every integral derivative is pinned by finite differences of the integral routines of
integrals.py, and the gradient by finite differences of the energy along the connection, and by
its translational and rotational invariance (tests/test_oracle_gradient.py).
"""
from __future__ import annotations

import numpy as np

from . import integrals, pnof, ri


def boys_f1(t):
    """F1(t) = int_0^1 u^2 exp(-t u^2) du = (F0(t) - exp(-t)) / (2t); series below 1e-4."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    small = t < 1e-4
    ts = t[small]
    out[small] = 1.0 / 3.0 - ts / 5.0 + ts * ts / 14.0
    tl = t[~small]
    out[~small] = (integrals.boys_f0(tl) - np.exp(-tl)) / (2.0 * tl)
    return out


def _atom_of_functions(basis, xyz):
    return np.repeat(np.arange(xyz.shape[0]), basis.per_atom)


def _prim_atoms(basis, xyz):
    fi, cen, ex, co = integrals._prim_table(basis, xyz)
    atom = _atom_of_functions(basis, xyz)[fi]
    return fi, atom, cen, ex, co


def one_electron_derivatives(basis, xyz, Z=None):
    """dS, dT, dV: [natom][3][n][n], derivatives of S, T and V (all nuclei) with respect to R_A,k."""
    natom = xyz.shape[0]
    Z = np.ones(natom) if Z is None else np.asarray(Z, np.float64)
    fi, at, cen, ex, co = _prim_atoms(basis, xyz)
    n = integrals.nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    mu = a * b / p
    AB = cen[:, None, :] - cen[None, :, :]
    AB2 = np.sum(AB ** 2, axis=-1)
    K = np.exp(-mu * AB2)
    Sp = (np.pi / p) ** 1.5 * K
    w = co[:, None] * co[None, :]
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    dS = np.zeros((natom, 3, n, n)); dT = np.zeros_like(dS); dV = np.zeros_like(dS)
    I, J = np.meshgrid(np.arange(len(ex)), np.arange(len(ex)), indexing="ij")
    for k in range(3):
        dSa = -2.0 * mu * AB[..., k] * Sp                              # d/dA; d/dB = -d/dA
        dTa = -2.0 * mu * mu * AB[..., k] * (5.0 - 2.0 * mu * AB2) * Sp
        np.add.at(dS, (at[I], k, fi[I], fi[J]), w * dSa)
        np.add.at(dS, (at[J], k, fi[I], fi[J]), -w * dSa)
        np.add.at(dT, (at[I], k, fi[I], fi[J]), w * dTa)
        np.add.at(dT, (at[J], k, fi[I], fi[J]), -w * dTa)
    for C in range(natom):
        PC = Pc - xyz[C]
        t = p * np.sum(PC ** 2, axis=-1)
        F0 = integrals.boys_f0(t)
        F1 = boys_f1(t)
        pre = -Z[C] * 2.0 * np.pi / p
        for k in range(3):
            dA = pre * (-2.0 * mu * AB[..., k] * K * F0 - 2.0 * a * K * F1 * PC[..., k])
            dB = pre * (2.0 * mu * AB[..., k] * K * F0 - 2.0 * b * K * F1 * PC[..., k])
            dC = pre * (2.0 * p * K * F1 * PC[..., k])
            np.add.at(dV, (at[I], k, fi[I], fi[J]), w * dA)
            np.add.at(dV, (at[J], k, fi[I], fi[J]), w * dB)
            dV[C, k] += np.bincount((fi[I] * n + fi[J]).ravel(), (w * dC).ravel(), n * n).reshape(n, n)
    return dS, dT, dV


def three_center_derivatives(basis, aux, xyz):
    """d(P|uv)/dR_A,k as [natom][3][X][n][n] (small systems)."""
    natom = xyz.shape[0]
    fi, at, cen, ex, co = _prim_atoms(basis, xyz)
    n = integrals.nbf(basis, xyz)
    acen, aex, anm = integrals._aux_table(aux, xyz)
    aat = np.repeat(np.arange(natom), integrals.naux(aux, xyz) // natom)
    X = len(aex)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    mu = a * b / p
    AB = cen[:, None, :] - cen[None, :, :]
    K = np.exp(-mu * np.sum(AB ** 2, axis=-1))
    Pc = (a[..., None] * cen[:, None, :] + b[..., None] * cen[None, :, :]) / p[..., None]
    w = co[:, None] * co[None, :]
    I, J = np.meshgrid(np.arange(len(ex)), np.arange(len(ex)), indexing="ij")
    out = np.zeros((natom, 3, X, n, n))
    for P in range(X):
        q = aex[P]
        rho = p * q / (p + q)
        PC = Pc - acen[P]
        t = rho * np.sum(PC ** 2, axis=-1)
        F0 = integrals.boys_f0(t)
        F1 = boys_f1(t)
        pre = anm[P] * w * 2.0 * np.pi ** 2.5 / (p * q * np.sqrt(p + q))
        for k in range(3):
            dA = pre * (-2.0 * mu * AB[..., k] * K * F0 - 2.0 * rho * (a / p) * K * F1 * PC[..., k])
            dB = pre * (2.0 * mu * AB[..., k] * K * F0 - 2.0 * rho * (b / p) * K * F1 * PC[..., k])
            np.add.at(out, (at[I], k, P, fi[I], fi[J]), dA)
            np.add.at(out, (at[J], k, P, fi[I], fi[J]), dB)
            blk = np.bincount((fi[I] * n + fi[J]).ravel(), (-(dA + dB)).ravel(), n * n).reshape(n, n)
            out[aat[P], k, P] += blk
    return out


def two_center_derivatives(aux, xyz):
    """d(P|Q)/dR_A,k as [natom][3][X][X]."""
    natom = xyz.shape[0]
    cen, ex, nm = integrals._aux_table(aux, xyz)
    aat = np.repeat(np.arange(natom), integrals.naux(aux, xyz) // natom)
    X = len(ex)
    p = ex[:, None]
    q = ex[None, :]
    rho = p * q / (p + q)
    D = cen[:, None, :] - cen[None, :, :]
    t = rho * np.sum(D ** 2, axis=-1)
    pre = nm[:, None] * nm[None, :] * 2.0 * np.pi ** 2.5 / (p * q * np.sqrt(p + q))
    F1 = boys_f1(t)
    out = np.zeros((natom, 3, X, X))
    I, J = np.meshgrid(np.arange(X), np.arange(X), indexing="ij")
    for k in range(3):
        dP = -pre * 2.0 * rho * F1 * D[..., k]       # d/dR of the first centre; the second gets -dP
        np.add.at(out, (aat[I], k, I, J), dP)
        np.add.at(out, (aat[J], k, I, J), -dP)
    return out


def nuclear_repulsion_gradient(xyz, Z=None):
    natom = xyz.shape[0]
    Z = np.ones(natom) if Z is None else np.asarray(Z, np.float64)
    g = np.zeros((natom, 3))
    for A in range(natom):
        for B in range(natom):
            if A != B:
                d = xyz[A] - xyz[B]
                g[A] -= Z[A] * Z[B] * d / np.linalg.norm(d) ** 3
    return g


def connected_orbitals(C0, S):
    """C0 (C0^T S C0)^{-1/2}: the orbitals at a displaced geometry (overlap S) on the connection."""
    M = C0.T @ S @ C0
    w, U = np.linalg.eigh(M)
    return C0 @ (U / np.sqrt(w)) @ U.T


def nuclear_gradient(orb, aux, xyz, C, gamma, pm: pnof.PairMap, Z=None, ipnof: int = 7):
    """dE/dR_A,k [natom][3] along the connection, at the state (C, gamma)."""
    a = pm.nact
    S, T, V = integrals.one_electron(orb, xyz, Z)
    H = T + V
    V2 = integrals.two_center(aux, xyz)
    M3 = integrals.three_center(orb, aux, xyz)
    B = ri.fitted_B(orb, aux, xyz)
    Ca = C[:, :a]
    nocc = pnof.occupation_numbers(gamma, pm)
    A, Bc = pnof.coefficients(gamma, pm, ipnof)
    Q3mo = np.einsum("up,Puv,vq->Ppq", Ca, M3, Ca)
    cfit = np.linalg.solve(V2, Q3mo.reshape(len(V2), -1)).reshape(Q3mo.shape)   # c^P_pq
    cdiag = np.einsum("Ppp->Pp", cfit)
    Y = -2.0 * Bc[None, :, :] * cfit
    Y[:, np.arange(a), np.arange(a)] += 2.0 * cdiag @ A.T
    Gam = np.einsum("up,Ppq,vq->Puv", Ca, Y, Ca)
    Zm = cdiag @ A @ cdiag.T - np.einsum("pq,Ppq,Qpq->PQ", Bc, cfit, cfit)
    Pao = 2.0 * (Ca * nocc[None, :]) @ Ca.T
    lam = pnof.lagrangian(B, H, C, gamma, pm, ipnof)
    Wao = C @ lam @ C.T
    dS, dT, dV = one_electron_derivatives(orb, xyz, Z)
    d3 = three_center_derivatives(orb, aux, xyz)
    d2 = two_center_derivatives(aux, xyz)
    g = np.einsum("uv,Akuv->Ak", Pao, dT + dV)
    g -= 2.0 * np.einsum("uv,Akuv->Ak", Wao, dS)
    g += np.einsum("Puv,AkPuv->Ak", Gam, d3)
    g -= np.einsum("PQ,AkPQ->Ak", Zm, d2)
    g += nuclear_repulsion_gradient(xyz, Z)
    return g
