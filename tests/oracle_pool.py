"""Process pool for the oracle's slice-by-slice orbital-basis route (test infrastructure).

Workers are started with `spawn` (safe after CUDA is initialised in the parent) and run with
single-threaded BLAS; each computes (P|q p) for one slice of aux functions."""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from oracle import integrals, large, ri


def _slice(args):
    orb, aux, xyz, C, nact, lo, hi = args
    return large.mo_three_center(orb, aux, xyz, C, nact, slice(lo, hi))


def fitted_mo(orb, aux, xyz, C, nact, workers=None):
    """b^P_{qp} [X][n][nact] of the oracle, (P|q p) computed in parallel slices, written into one
    preallocated array and fitted in place (one array of X n nact doubles)."""
    X = integrals.naux(aux, xyz)
    n = C.shape[0]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    step = max(1, -(-X // (4 * workers)))
    jobs = [(orb, aux, xyz, C, nact, lo, min(X, lo + step)) for lo in range(0, X, step)]
    Q3 = np.empty((X, n, nact))
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            for (_, _, _, _, _, lo, hi), part in zip(jobs, ex.map(_slice, jobs)):
                Q3[lo:hi] = part
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return large.fit_inplace(Q3, integrals.two_center(aux, xyz))


def _nuclear_slice(args):
    orb, xyz, lo, hi = args
    return integrals.nuclear_attraction(orb, xyz, None, range(lo, hi))


def core_hamiltonian(orb, xyz, workers=None):
    """S and H = T + V of the oracle, V summed over slices of nuclei computed in parallel."""
    natom = xyz.shape[0]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    step = max(1, -(-natom // workers))
    jobs = [(orb, xyz, lo, min(natom, lo + step)) for lo in range(0, natom, step)]
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        V = sum(ex.map(_nuclear_slice, jobs))
    return integrals.overlap(orb, xyz), integrals.kinetic(orb, xyz) + V


def _slice_cols(args):
    orb, aux, xyz, Cs, lo, hi = args
    M = integrals.three_center(orb, aux, xyz, slice(lo, hi))
    return np.matmul(Cs.T[None, :, :], np.matmul(M, Cs))


def fitted_columns(orb, aux, xyz, Cs, workers=None):
    """b^P_{ij} = sum_Q (V^{-1/2})_{PQ} (Q|i j) for the orbitals given as the columns of Cs only
    ([X][k][k]); the three-centre integrals are generated in parallel slices of aux functions."""
    X = integrals.naux(aux, xyz)
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    step = max(1, -(-X // (4 * workers)))
    jobs = [(orb, aux, xyz, Cs, lo, min(X, lo + step)) for lo in range(0, X, step)]
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            Q3 = np.concatenate(list(ex.map(_slice_cols, jobs)))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    k = Q3.shape[1]
    return (ri.inverse_sqrt_metric(integrals.two_center(aux, xyz)) @ Q3.reshape(X, k * k)).reshape(X, k, k)


def _frame(args):
    orb, aux, xyz, Q, gam = args
    S, T, V = integrals.one_electron(orb, xyz)
    B = ri.fitted_B(orb, aux, xyz)
    from oracle import pnof, reference
    n = S.shape[0]
    pm = pnof.PairMap(xyz.shape[0], 1, n)
    C = reference.orthonormal_orbitals(S, Q)
    r = pnof.energy_and_gradients(B, T + V, C, gam, pm, integrals.nuclear_repulsion(xyz))
    return C, r["E"], r["g"], r["g_gamma"]


def frames(jobs, workers=None):
    """The oracle's (C, E, g, g_gamma) for every (orb, aux, xyz, Q, gamma) job, C = S^{-1/2} Q, in
    spawned worker processes with single-threaded BLAS."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_frame, jobs, chunksize=4))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
