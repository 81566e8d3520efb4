"""Seeded test systems: geometry + basis from the shared input generators, oracle results on
demand. Only tests import this module."""
import functools

import numpy as np

from oracle import integrals, pnof, reference, ri
from paper_2512_13550_gb300 import inputs


class System:
    def __init__(self, name, xyz, orb, aux, ncwo=1):
        self.name, self.xyz, self.orb, self.aux, self.ncwo = name, xyz, orb, aux, ncwo

    @functools.cached_property
    def oracle(self):
        S, T, V = integrals.one_electron(self.orb, self.xyz)
        B = ri.fitted_B(self.orb, self.aux, self.xyz)
        n = S.shape[0]
        pm = pnof.PairMap(self.xyz.shape[0], self.ncwo, n)
        return dict(S=S, H=T + V, B=B, vnn=integrals.nuclear_repulsion(self.xyz), pm=pm, n=n)

    def orbitals(self, seed=0):
        o = self.oracle
        return reference.orthonormal_orbitals(o["S"], inputs.random_orthogonal(o["n"], seed))

    def gamma(self, seed=1):
        return inputs.random_gamma(self.oracle["pm"].ngamma, seed)


def h4(ncwo=1):
    orb, aux = inputs.basis_h4()
    return System("H4", inputs.chain(4, 1.8), orb, aux, ncwo)


def chain3s(natom, seed=2, ncwo=1):
    orb, aux = inputs.basis_3s_10aux()
    return System(f"H{natom}", inputs.jittered_chain(natom, seed), orb, aux, ncwo)


def h50():
    return chain3s(50, seed=2)
