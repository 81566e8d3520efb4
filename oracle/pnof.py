"""PNOF pairing, occupations, energy, Lagrangian and gradients (oracle; test infrastructure only).

Follows DoNOF 2.0 (arXiv 2512.13550):
  * pairing: a closed-shell singlet has N_I = 0 and N_II/2 = N/2 subspaces Omega_g, each
    holding one strongly occupied orbital g < N/2 and N_g weakly occupied orbitals above
    N_Omega = N/2 (Eq. OmegaG). Reading of Fig. 1: subspace g takes, in every block of N/2
    weak orbitals, the orbital counted from the top of the block, so for N_g = 1 the pairs are
    HOMO<->LUMO, HOMO-1<->LUMO+1, ... Orbitals past N/2 (N_g + 1) have zero occupation.
  * sum rule n_g + sum_i n_{p_i} = 1 per subspace (Eq. sum1), trace 2 sum n = N.
  * trigonometric mapping (Occupation Number Optimization subsection):
        n_g = (1 + cos^2 gamma_g)/2,  h_g = 1 - n_g,
        n_{p_i} = h_g cos^2 gamma_{p_1} ... cos^2 gamma_{p_{i-1}} sin^2 gamma_{p_i}  (i < N_g),
        n_{p_{N_g}} = h_g cos^2 gamma_{p_1} ... cos^2 gamma_{p_{N_g - 1}}.
    Angles are stored slot-major: gamma[i * npair + g], slot 0 = gamma_g, slot i = gamma_{p_i}.
  * softmax mapping (same subsection, ISOFTMAX = 1), N_g variables per subspace, one per weak
    orbital, stored slot-major too: gamma[k * npair + g] = gamma_{p_{k+1}};
        n_g = 1 / (1 + sum_k exp(gamma_{p_k})),   n_{p_i} = n_g exp(gamma_{p_i}).
  * JKL-only energy (Eq. PNOF), with L = K for real orbitals:
        E = 2 sum_p n_p h_pp + sum_pq A_pq J_pq - sum_pq B_pq K_pq + V_nn.
    The paper defers A and B to the PNOF5/PNOF7 publications. Reading (spin-restricted
    singlet, c_p = +sqrt(n_p) strong, -sqrt(n_p) weak, Phi_p = sqrt(n_p (1 - n_p))):
        A_pp = n_p;  A_pq = 2 n_p n_q (different subspaces);  0 within a subspace;
        B_pp = 0;    B_pq = -c_p c_q (same subspace);  B_pq = n_p n_q + Phi_p Phi_q
        (different subspaces; PNOF5 drops the Phi term).
  * Lagrangian L = E - 2 sum lambda_qp (<p|q> - delta_pq) and orbital gradient
    g_pq = dE/dy_pq = 4 (lambda_pq - lambda_qp) (Natural Orbital Optimization subsection).
    With phi_p = sum_mu C_mu,p chi_mu and C' = C exp(y), dE = 4 sum_pq lambda_qp y_qp where
        lambda = C^T Lambda,  Lambda_mu,p = n_p (H C)_mu,p + sum_P T^P_mu,p D^P_p
                                           - sum_P sum_q T^P_mu,q B_pq b^P_qp,
    T^P = B^P C, b^P = C^T T^P, d^P_p = b^P_pp, D^P = A d^P.

The square roots sqrt(n_p) and sqrt(1 - n_p) are formed directly from |sin| and |cos| of the
angles so that their derivatives never divide by a vanishing occupation; the one-sided
derivative from gamma > 0 is taken at the kink gamma = 0 (sign(0) := +1).

Parity: pinned by the RHF limit (AO-form RHF energy), the two-electron DOCI/FCI cases, the
sum rule and trace, finite differences of E in y and in gamma, and by the 2RDM route of rdm.py:
the energy assembled here from A and B equals Eq. (Energy) contracted with the spin-orbital 2RDM
of the Theory section's cumulant expansion, element by element, for PNOF5 and PNOF7 with N_g = 1
and 2 (which pins every factor and sign of the A/B bookkeeping, the inter-pair Phi term's
included). The values of Delta and Pi, and with them Phi_p = sqrt(n_p (1 - n_p)), are the
functionals' readings (the paper defers them); the value of Phi is parity unpinned.
"""
from __future__ import annotations

import numpy as np


class PairMap:
    """Closed-shell pairing structure for N electrons, N_g weak orbitals per subspace, and the
    ON mapping (isoftmax = 0: trigonometric, 1: softmax)."""

    def __init__(self, nelec: int, ncwo: int, nbf: int, isoftmax: int = 0):
        if nelec % 2 or nelec <= 0:
            raise ValueError("closed-shell singlet needs an even, positive electron count")
        if isoftmax not in (0, 1):
            raise ValueError("isoftmax must be 0 (trigonometric) or 1 (softmax)")
        self.isoftmax = isoftmax
        self.npair = nelec // 2
        self.ncwo = ncwo
        self.nact = self.npair * (ncwo + 1)
        if self.nact > nbf:
            raise ValueError("not enough orbitals for the requested pairing")
        self.ngamma = self.npair * ncwo
        self.pair = np.full(self.nact, -1)
        self.slot = np.full(self.nact, -1)  # 0 strong, i >= 1 weak orbital p_i
        for g in range(self.npair):
            self.pair[g] = g
            self.slot[g] = 0
            for i in range(1, ncwo + 1):
                p = self.npair + (i - 1) * self.npair + (self.npair - 1 - g)
                self.pair[p] = g
                self.slot[p] = i
        self.strong = self.slot == 0
        self.same = self.pair[:, None] == self.pair[None, :]

    def weak_orbital(self, g: int, i: int) -> int:
        return self.npair + (i - 1) * self.npair + (self.npair - 1 - g)


def _sgn(x):
    return 1.0 if x >= 0.0 else -1.0


def occupations(gamma, pm: PairMap):
    """sqrt(n_p), sqrt(1 - n_p) and their derivatives with respect to every gamma, for the
    mapping pm.isoftmax selects.

    Returns s, t (length nact) and ds, dt (nact x ngamma)."""
    if pm.isoftmax:
        return occupations_softmax(gamma, pm)
    gamma = np.asarray(gamma, np.float64)
    a, ng, P, Ng = pm.nact, pm.ngamma, pm.npair, pm.ncwo
    s = np.zeros(a); t = np.zeros(a)
    ds = np.zeros((a, ng)); dt = np.zeros((a, ng))
    for g in range(P):
        k0 = g  # index of gamma_g
        th0 = gamma[k0]
        sg = np.sqrt(0.5 * (1.0 + np.cos(th0) ** 2))
        tg = abs(np.sin(th0)) / np.sqrt(2.0)
        dsg = (-np.sin(th0) * np.cos(th0)) / (2.0 * sg)
        dtg = _sgn(np.sin(th0)) * np.cos(th0) / np.sqrt(2.0)
        s[g], t[g] = sg, tg
        ds[g, k0], dt[g, k0] = dsg, dtg
        # weak orbitals: s_{p_i} = t_g * prod_{j<i} |cos th_j| * (|sin th_i| if i < N_g)
        for i in range(1, Ng + 1):
            p = pm.weak_orbital(g, i)
            factors = [(k0, tg, dtg)]
            for j in range(1, i):
                kj = j * P + g
                th = gamma[kj]
                factors.append((kj, abs(np.cos(th)), -_sgn(np.cos(th)) * np.sin(th)))
            if i < Ng:
                ki = i * P + g
                th = gamma[ki]
                factors.append((ki, abs(np.sin(th)), _sgn(np.sin(th)) * np.cos(th)))
            val = np.prod([f[1] for f in factors])
            s[p] = val
            for m, (km, fm, dfm) in enumerate(factors):
                others = np.prod([f[1] for q, f in enumerate(factors) if q != m])
                ds[p, km] += dfm * others
            t[p] = np.sqrt(1.0 - val * val)
            dt[p, :] = -val * ds[p, :] / t[p]
    return s, t, ds, dt


def occupations_softmax(gamma, pm: PairMap):
    """The softmax mapping: per subspace g with variables x_k = gamma_{p_k} (k = 1..N_g),
        Z = 1 + sum_k exp(x_k),  n_g = 1 / Z,  n_{p_i} = n_g exp(x_i),
    so that sqrt(n_g) = Z^{-1/2}, sqrt(n_{p_i}) = exp(x_i / 2) Z^{-1/2}, and
        d sqrt(n_q) / d x_j = sqrt(n_q) (delta_{q, p_j} - n_{p_j}) / 2
    for every orbital q of the subspace (with delta_{g, p_j} = 0). sqrt(1 - n) follows from
    1 - n_g = sum_k n_{p_k} and 1 - n_{p_i} = n_g + sum_{k != i} n_{p_k}, and
    d sqrt(1 - n) = -sqrt(n) d sqrt(n) / sqrt(1 - n).

    Returns s, t (length nact) and ds, dt (nact x ngamma) as occupations() does."""
    gamma = np.asarray(gamma, np.float64)
    a, ng, P, Ng = pm.nact, pm.ngamma, pm.npair, pm.ncwo
    s = np.zeros(a); t = np.zeros(a)
    ds = np.zeros((a, ng)); dt = np.zeros((a, ng))
    for g in range(P):
        keys = [k * P + g for k in range(Ng)]              # gamma index of x_{k+1}
        ex = np.array([np.exp(gamma[k]) for k in keys])
        Z = 1.0 + ex.sum()
        n_g = 1.0 / Z
        n_w = n_g * ex                                     # n_{p_1} .. n_{p_Ng}
        orbs = [g] + [pm.weak_orbital(g, i) for i in range(1, Ng + 1)]
        occ = [n_g] + list(n_w)
        rest = [n_w.sum()] + [n_g + n_w.sum() - n_w[i] for i in range(Ng)]  # 1 - n, per orbital
        for m, q in enumerate(orbs):
            s[q] = np.sqrt(occ[m])
            t[q] = np.sqrt(rest[m])
            for j, kj in enumerate(keys):
                own = 1.0 if m == j + 1 else 0.0
                ds[q, kj] = 0.5 * s[q] * (own - n_w[j])
                dt[q, kj] = -s[q] * ds[q, kj] / t[q]
    return s, t, ds, dt


def occupation_numbers(gamma, pm: PairMap):
    s, _, _, _ = occupations(gamma, pm)
    return s * s


def coefficients(gamma, pm: PairMap, ipnof: int = 7):
    """A and B coefficient matrices (nact x nact) of Eq. PNOF for PNOF7 (or PNOF5)."""
    s, t, _, _ = occupations(gamma, pm)
    n = s * s
    c = np.where(pm.strong, s, -s)
    phi = s * t
    diff = ~pm.same
    A = np.where(diff, 2.0 * np.outer(n, n), 0.0)
    np.fill_diagonal(A, n)
    Bc = np.where(pm.same, -np.outer(c, c), np.outer(n, n))
    if ipnof == 7:
        Bc = Bc + np.where(diff, np.outer(phi, phi), 0.0)
    elif ipnof != 5:
        raise ValueError("only PNOF5 and PNOF7 are defined here")
    np.fill_diagonal(Bc, 0.0)
    return A, Bc


def transform(B, C, nact):
    """Half and full transforms: T^P = B^P C_a (n x a), b^P = C_a^T T^P (a x a)."""
    Ca = C[:, :nact]
    T = np.einsum("Pmn,na->Pma", B, Ca)
    b = np.einsum("mq,Pmp->Pqp", Ca, T)
    return T, b


def jk(B, C, nact):
    """J_pq = sum_P b^P_pp b^P_qq and K_pq = sum_P (b^P_pq)^2 for the active orbitals."""
    _, b = transform(B, C, nact)
    d = np.einsum("Ppp->Pp", b)
    J = d.T @ d
    K = np.einsum("Ppq,Ppq->pq", b, b)
    return J, K


def energy_from_jk(hpp, J, K, gamma, pm: PairMap, vnn: float, ipnof: int = 7) -> float:
    A, Bc = coefficients(gamma, pm, ipnof)
    n = occupation_numbers(gamma, pm)
    return 2.0 * np.dot(n, hpp) + np.sum(A * J) - np.sum(Bc * K) + vnn


def energy(B, H, C, gamma, pm: PairMap, vnn: float, ipnof: int = 7) -> float:
    a = pm.nact
    J, K = jk(B, C, a)
    hpp = np.einsum("mp,mn,np->p", C[:, :a], H, C[:, :a])
    return energy_from_jk(hpp, J, K, gamma, pm, vnn, ipnof)


def lagrangian(B, H, C, gamma, pm: PairMap, ipnof: int = 7):
    """lambda (n x n; columns >= nact are zero) = C^T Lambda."""
    a = pm.nact
    n_bf = C.shape[0]
    A, Bc = coefficients(gamma, pm, ipnof)
    nocc = occupation_numbers(gamma, pm)
    T, b = transform(B, C, a)
    d = np.einsum("Ppp->Pp", b)
    D = d @ A.T                                   # D^P_p = sum_r A_pr d^P_r
    Lam = (H @ C[:, :a]) * nocc[None, :]
    Lam += np.einsum("Pmp,Pp->mp", T, D)
    Lam -= np.einsum("Pmq,pq,Pqp->mp", T, Bc, b)
    lam = np.zeros((n_bf, n_bf))
    lam[:, :a] = C.T @ Lam
    return lam


def orbital_gradient(lam):
    return 4.0 * (lam - lam.T)


def gamma_gradient(hpp, J, K, gamma, pm: PairMap, ipnof: int = 7):
    """dE/dgamma by the chain rule through sqrt(n), c = +-sqrt(n), Phi = sqrt(n) sqrt(1-n)."""
    s, t, ds, dt = occupations(gamma, pm)
    n = s * s
    sign = np.where(pm.strong, 1.0, -1.0)
    c = sign * s
    phi = s * t
    diff = ~pm.same
    offd = pm.same & ~np.eye(pm.nact, dtype=bool)
    dE_dn = 2.0 * hpp + np.diag(J) + 2.0 * np.sum(np.where(diff, n[None, :] * (2.0 * J - K), 0.0), axis=1)
    dE_dc = 2.0 * np.sum(np.where(offd, c[None, :] * K, 0.0), axis=1)
    dE_dphi = -2.0 * np.sum(np.where(diff, phi[None, :] * K, 0.0), axis=1)
    if ipnof == 5:
        dE_dphi = np.zeros_like(dE_dphi)
    dn = 2.0 * s[:, None] * ds
    dc = sign[:, None] * ds
    dphi = ds * t[:, None] + s[:, None] * dt
    return dE_dn @ dn + dE_dc @ dc + dE_dphi @ dphi


def energy_and_gradients(B, H, C, gamma, pm: PairMap, vnn: float, ipnof: int = 7):
    """One energy+gradient evaluation at fixed (C, gamma): E, J, K, lambda, g_orb, g_gamma."""
    a = pm.nact
    J, K = jk(B, C, a)
    hpp = np.einsum("mp,mn,np->p", C[:, :a], H, C[:, :a])
    E = energy_from_jk(hpp, J, K, gamma, pm, vnn, ipnof)
    lam = lagrangian(B, H, C, gamma, pm, ipnof)
    return dict(E=E, J=J, K=K, hpp=hpp, lam=lam, g=orbital_gradient(lam),
                g_gamma=gamma_gradient(hpp, J, K, gamma, pm, ipnof))
