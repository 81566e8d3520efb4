"""Finite-field polarizability and hyperpolarizabilities (oracle; test infrastructure only).

Follows the NLOPs subsection (Polarizabilities and Hyperpolarizabilities) of DoNOF 2.0
(arXiv 2512.13550):
  * a static field along one axis, with strengths on the dyadic ladder h_k = STEP 2^{k-1}
    (k = 1 .. NPOINT); the dipole moment is evaluated at -2h, -h, 0, h, 2h for every h_k;
  * centred differences of order h^2:
        alpha(h) = (mu(h) - mu(-h)) / (2h),
        beta(h)  = (mu(h) - 2 mu(0) + mu(-h)) / h^2,
        gamma(h) = (mu(2h) - 2 mu(h) + 2 mu(-h) - mu(-2h)) / (2 h^3);
  * a Romberg-Richardson triangle with p = 2: R(k, 1) = D(h_k) and
        R(k, j) = R(k, j-1) + (R(k, j-1) - R(k+1, j-1)) / (4^{j-1} - 1),  k <= NPOINT - j + 1;
  * the value reported: over every column j and every vertical pair (k, k+1) of it, the pair
    with the smallest Delta_{k,j} = |R(k+1, j) - R(k, j)| selects R(k, j+1), with Delta as its
    uncertainty; equal Deltas are resolved towards the candidate of smallest magnitude;
  * ISOALPHA: alpha_xx, alpha_yy, alpha_zz from fields along x, y, z, the isotropic mean and the
    anisotropy in the Raman convention.

Readings (the paper leaves these to the code it describes):
  * the field couples through the dipole operator mu = -sum_i r_i + sum_A Z_A R_A: the
    Hamiltonian gains -mu.F, so h_uv -> h_uv + F.<u|r|v> and V_nn -> V_nn - F.sum_A Z_A R_A (the
    EVEC keyword's field);
  * mu of a state is the expectation value of that operator with the NOF 1RDM (diagonal in the
    natural orbitals): mu = -2 sum_p n_p <phi_p|r|phi_p> + sum_A Z_A R_A;
  * at fixed orbitals and occupations E(F) = E(0) - F.mu, exactly;
  * 2 h_k = h_{k+1}, so the 5 NPOINT field points hold 2 NPOINT + 3 distinct fields; each is
    computed once;
  * the state at each field is what the library's alternating steps reach from one common
    starting point. The paper converges each field to tight thresholds (NTHRESHL on the
    symmetry of the Lagrange multipliers, NTHRESHE on the energy). Here a field stops at the
    first check (every `check` steps) where the step reports ||g|| < gtol, or after `nsteps`
    steps. Stopping matters: once converged, further ADAM steps eventually leave the minimum,
    at a point that depends on rounding.

Parity: the dipole integrals are pinned by quadrature and by their origin dependence, the field
term by the exact linearity of E(F), the differences and the triangle by polynomials they must
reproduce exactly, and the whole pipeline by beta = 0 for a centrosymmetric chain
(tests/test_oracle_nlop.py).
"""
from __future__ import annotations

import numpy as np

from . import integrals, pnof, step


def dipole_integrals(basis, xyz):
    """D [3][n][n]: D_k,uv = <u|r_k|v> over contracted s Gaussians. For a primitive pair the
    product is a Gaussian at P = (aA + bB)/(a + b), so <a|r_k|b> = P_k <a|b>."""
    fi, cen, ex, co = integrals._prim_table(basis, xyz)
    n = integrals.nbf(basis, xyz)
    a = ex[:, None]
    b = ex[None, :]
    p = a + b
    AB2 = np.sum((cen[:, None, :] - cen[None, :, :]) ** 2, axis=-1)
    Sp = (np.pi / p) ** 1.5 * np.exp(-a * b / p * AB2)
    D = np.zeros((3, n, n))
    for k in range(3):
        Pk = (a * cen[:, None, k] + b * cen[None, :, k]) / p
        np.add.at(D[k], (fi[:, None], fi[None, :]), co[:, None] * co[None, :] * Sp * Pk)
    return D


def nuclear_dipole(xyz, Z=None):
    Z = np.ones(xyz.shape[0]) if Z is None else np.asarray(Z, np.float64)
    return Z @ xyz


def field_hamiltonian(H, D, F, xyz, vnn, Z=None):
    """h(F) = h + sum_k F_k D_k and V_nn(F) = V_nn - F . sum_A Z_A R_A."""
    F = np.asarray(F, np.float64)
    return H + np.einsum("k,kuv->uv", F, D), vnn - float(F @ nuclear_dipole(xyz, Z))


def dipole(C, gamma, pm: pnof.PairMap, D, xyz, Z=None):
    """mu = -2 sum_p n_p (C^T D_k C)_pp + sum_A Z_A R_A, for k = x, y, z."""
    a = pm.nact
    n = pnof.occupation_numbers(gamma, pm)
    Ca = C[:, :a]
    w = np.einsum("up,kuv,vp->kp", Ca, D, Ca)
    return -2.0 * w @ n + nuclear_dipole(xyz, Z)


def field_points(step_size: float, npoint: int):
    """The distinct field strengths: 0 and +-STEP 2^{k-1} for k = 1 .. NPOINT + 1."""
    h = step_size * 2.0 ** np.arange(npoint + 1)
    return np.concatenate([[0.0], h, -h])


def differences(mu, step_size: float, npoint: int):
    """alpha(h_k), beta(h_k), gamma(h_k) for k = 1 .. NPOINT from mu(F), a dict field -> value."""
    al, be, ga = [], [], []
    for k in range(npoint):
        h = step_size * 2.0 ** k
        m2, m1, m0, p1, p2 = mu[-2 * h], mu[-h], mu[0.0], mu[h], mu[2 * h]
        al.append((p1 - m1) / (2.0 * h))
        be.append((p1 - 2.0 * m0 + m1) / (h * h))
        ga.append((p2 - 2.0 * p1 + 2.0 * m1 - m2) / (2.0 * h ** 3))
    return np.array(al), np.array(be), np.array(ga)


def romberg(D):
    """Triangle R [NPOINT][NPOINT] (R[k-1][j-1] = R(k, j); unused entries NaN) and the selected
    (value, Delta, k, j) by the minimum-Delta rule (1-based k, j of the selecting pair)."""
    D = np.asarray(D, np.float64)
    N = D.size
    R = np.full((N, N), np.nan)
    R[:, 0] = D
    for j in range(2, N + 1):
        for k in range(1, N - j + 2):
            prev, nxt = R[k - 1, j - 2], R[k, j - 2]
            R[k - 1, j - 1] = prev + (prev - nxt) / (4.0 ** (j - 1) - 1.0)
    best = None
    for j in range(1, N):
        for k in range(1, N - j + 1):
            delta = abs(R[k, j - 1] - R[k - 1, j - 1])
            value = R[k - 1, j]
            cand = (delta, abs(value), value, k, j)
            if best is None or cand[:2] < best[:2]:
                best = cand
    if best is None:
        return R, (float(D[0]), float("nan"), 1, 1)
    return R, (best[2], best[0], best[3], best[4])


def polarizability_invariants(axx: float, ayy: float, azz: float):
    """ISOALPHA: the isotropic polarizability (axx + ayy + azz) / 3 and the anisotropy (Raman
    convention) sqrt(((axx - ayy)^2 + (ayy - azz)^2 + (azz - axx)^2) / 2)."""
    iso = (axx + ayy + azz) / 3.0
    aniso = np.sqrt(((axx - ayy) ** 2 + (ayy - azz) ** 2 + (azz - axx) ** 2) / 2.0)
    return iso, aniso


def run(B, H, D, xyz, vnn, pm: pnof.PairMap, axis: int, step_size: float, npoint: int, nsteps: int,
        C0, gamma0, ipnof: int = 7, Z=None, gtol=None, check: int = 25, **opt):
    """The whole workload: alternating steps at every distinct field from (C0, gamma0) (at most
    nsteps; with gtol, stopping at the first multiple of `check` steps whose step reported
    ||g|| < gtol), the dipole along `axis` at each final state, the differences and the three
    triangles. `steps` holds the step count of each field."""
    mu, steps = {}, {}
    for f in field_points(step_size, npoint):
        F = np.zeros(3)
        F[axis] = f
        Hf, vf = field_hamiltonian(H, D, F, xyz, vnn, Z)
        st = step.State(C0, gamma0)
        done = 0
        for it in range(nsteps):
            _, gn, _ = step.step(B, Hf, vf, st, pm, ipnof, **opt)
            done = it + 1
            if gtol is not None and done % check == 0 and gn < gtol:
                break
        mu[f] = dipole(st.C, st.gamma, pm, D, xyz, Z)[axis]
        steps[f] = done
    al, be, ga = differences(mu, step_size, npoint)
    return dict(mu=mu, steps=steps, alpha=romberg(al), beta=romberg(be), gamma=romberg(ga), D=(al, be, ga))
