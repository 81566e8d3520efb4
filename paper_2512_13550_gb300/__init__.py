"""GB300 library for the density-fitted PNOF JK step (DoNOF 2.0, arXiv 2512.13550).

This module is a thin ctypes binding over the C ABI in include/nof.h: it marshals torch CUDA
tensors (device memory and the current stream) into plain pointers and turns status codes into
exceptions. Every step of the computation runs in the library's own CUDA kernels; there is no
CPU fallback, and importing this package fails loudly if libnof.so has not been built
(python -m paper_2512_13550_gb300.build).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (re-exported: seeded synthetic inputs)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnof.so")

PREC_FP64 = 0
PREC_SPLIT_BF16 = 1

NOF_OK, NOF_EINVAL, NOF_ENOMEM, NOF_ECUDA = 0, -1, -2, -3
NOF_ETIMEOUT, NOF_ENONFINITE, NOF_EILLCOND, NOF_ENOTCONV, NOF_ESTATE = -4, -5, -6, -7, -8
ERROR_NAMES = {
    -1: "NOF_EINVAL", -2: "NOF_ENOMEM", -3: "NOF_ECUDA", -4: "NOF_ETIMEOUT",
    -5: "NOF_ENONFINITE", -6: "NOF_EILLCOND", -7: "NOF_ENOTCONV", -8: "NOF_ESTATE",
}


class NofError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("ipnof", ctypes.c_int), ("isoftmax", ctypes.c_int), ("ncwo", ctypes.c_int),
                ("precision", ctypes.c_int), ("on_iters", ctypes.c_int), ("on_lr", ctypes.c_double),
                ("lr", ctypes.c_double), ("b1", ctypes.c_double), ("b2", ctypes.c_double),
                ("eps", ctypes.c_double), ("digits", ctypes.c_int), ("graphs", ctypes.c_int)]


class OptParams(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("maxloop", ctypes.c_int), ("gtol", ctypes.c_double),
                ("etol", ctypes.c_double), ("lr", ctypes.c_double), ("lr_min", ctypes.c_double),
                ("on_tol", ctypes.c_double), ("on_maxit", ctypes.c_int), ("eps_rel", ctypes.c_double),
                ("lr_grow", ctypes.c_double), ("orbopt", ctypes.c_int), ("memory", ctypes.c_int),
                ("lbfgs_after", ctypes.c_double)]


class CBasis(ctypes.Structure):
    _fields_ = [("nshell", ctypes.c_int), ("nprim", ctypes.POINTER(ctypes.c_int)),
                ("exps", ctypes.POINTER(ctypes.c_double)), ("coefs", ctypes.POINTER(ctypes.c_double))]


_lib = None

# name -> (restype, argtypes); mirrors include/nof.h
_P = ctypes.c_void_p
SIGNATURES = {
    "nof_default_options": (None, [ctypes.POINTER(Options)]),
    "nof_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Options), _P]),
    "nof_destroy": (ctypes.c_int, [_P]),
    "nof_build_B": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(CBasis), ctypes.POINTER(CBasis)]),
    "nof_query": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "nof_get_SH": (ctypes.c_int, [_P, _P, _P]),
    "nof_get_B": (ctypes.c_int, [_P, _P]),
    "nof_tuned_tiles": (ctypes.c_int, [_P, _P]),
    "nof_split_digits": (ctypes.c_int, [_P, _P]),
    "nof_lowdin": (ctypes.c_int, [_P, _P, _P]),
    "nof_core_guess": (ctypes.c_int, [_P, _P, _P]),
    "nof_jk": (ctypes.c_int, [_P, _P, _P, _P]),
    "nof_energy_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "nof_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "nof_sync": (ctypes.c_int, [_P]),
    "nof_default_opt_params": (None, [ctypes.POINTER(OptParams)]),
    "nof_optimize": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(OptParams), _P, _P]),
    "nof_energy_grad_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]),
    "nof_kernel_launches": (ctypes.c_longlong, []),
    "nof_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "nof_profile_read": (ctypes.c_int, [_P, _P, _P, _P]),
    "nof_selftest_digit_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_uint, _P]),
    "nof_bench_digit_gemm": (ctypes.c_int, [ctypes.c_int] * 8 + [_P]),
    "nof_selftest_digit_gemm_timeout": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.c_double, _P]),
    "nof_jk_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "nof_mlp_param_count": (ctypes.c_longlong, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "nof_mlp_work_size": (ctypes.c_longlong, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "nof_mlp_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "nof_mlp_loss_grad": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P,
                                         _P, _P]),
    "nof_mlp_to_bf16": (ctypes.c_int, [ctypes.c_longlong, _P, _P, _P]),
    "nof_mlp_forward_bf16": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                            _P, _P]),
    "nof_mlp_adam": (ctypes.c_int, [ctypes.c_longlong, _P, _P, _P, _P, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "nof_nuclear_gradient": (ctypes.c_int, [_P, _P, _P, _P]),
    "nof_set_field": (ctypes.c_int, [_P, _P]),
    "nof_dipole": (ctypes.c_int, [_P, _P, _P, _P]),
    "nof_field_differences": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _P, _P, _P]),
    "nof_romberg": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "nof_step_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "nof_polarizability_invariants": (ctypes.c_int, [_P, _P]),
    "nof_last_error": (ctypes.c_char_p, []),
}


def load_library():
    """Load libnof.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2512_13550_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by libnof so far in this process (counted at every launch site)."""
    return int(load_library().nof_kernel_launches())


def selftest_digit_gemm(M: int, N: int, bn: int, katoms: int, chunk_atoms: int = 0, seed: int = 1,
                        nd: int = 4) -> int:
    """Largest |difference| between the tcgen05 digit GEMM (nd digits, N tiles of bn, K chunks of
    chunk_atoms atoms; 0 = one chunk) and a SIMT integer reference."""
    out = ctypes.c_longlong(-1)
    chunk = chunk_atoms if chunk_atoms > 0 else katoms
    _check(load_library().nof_selftest_digit_gemm(M, N, bn, nd, katoms, chunk, seed, ctypes.byref(out)))
    return out.value


def bench_digit_gemm(M: int, N: int, bn: int, nd: int, katoms: int, chunk_atoms: int = 0, mode: int = 0,
                     reps: int = 10) -> float:
    """Microseconds per launch of the digit GEMM on zero operands (see nof_bench_digit_gemm)."""
    us = ctypes.c_double(-1.0)
    chunk = chunk_atoms if chunk_atoms > 0 else katoms
    _check(load_library().nof_bench_digit_gemm(M, N, bn, nd, katoms, chunk, mode, reps, ctypes.byref(us)))
    return us.value


def field_differences(mu, npoint: int, step: float):
    """alpha(h_k), beta(h_k), gamma(h_k), k = 1 .. npoint, from the dipoles at the 2 npoint + 3
    distinct fields 0, +h_1 .. +h_{npoint+1}, -h_1 .. -h_{npoint+1} (nof_field_differences)."""
    mu = np.ascontiguousarray(mu, np.float64)
    if mu.size != 2 * npoint + 3:
        raise ValueError("expected 2 npoint + 3 dipoles")
    out = [np.zeros(npoint) for _ in range(3)]
    _check(load_library().nof_field_differences(mu.ctypes.data_as(ctypes.c_void_p), npoint, float(step),
                                                *(o.ctypes.data_as(ctypes.c_void_p) for o in out)))
    return tuple(out)


def romberg(D):
    """Romberg-Richardson triangle of D(h_k) and the selected (value, Delta, k, j) (nof_romberg)."""
    D = np.ascontiguousarray(D, np.float64)
    N = D.size
    R = np.zeros((N, N))
    best = np.zeros(2)
    sel = np.zeros(2, np.int32)
    _check(load_library().nof_romberg(D.ctypes.data_as(ctypes.c_void_p), N, R.ctypes.data_as(ctypes.c_void_p),
                                      best.ctypes.data_as(ctypes.c_void_p), sel.ctypes.data_as(ctypes.c_void_p)))
    return R, (float(best[0]), float(best[1]), int(sel[0]), int(sel[1]))


def polarizability_invariants(axx: float, ayy: float, azz: float):
    """Isotropic polarizability and anisotropy (Raman convention) (nof_polarizability_invariants)."""
    a = np.array([axx, ayy, azz], np.float64)
    out = np.zeros(2)
    _check(load_library().nof_polarizability_invariants(a.ctypes.data_as(ctypes.c_void_p),
                                                         out.ctypes.data_as(ctypes.c_void_p)))
    return float(out[0]), float(out[1])


def step_batch(contexts, Cs, gammas, ms, vs, outs, stream=None, device_counter: bool = False):
    """One nof_step on every context concurrently (each on its own stream), forked from `stream`.
    device_counter: the contexts' device-side step counters (the call is then capturable)."""
    import torch
    n = len(contexts)
    stream = stream if stream is not None else torch.cuda.current_stream()
    arr = lambda ts: (ctypes.c_void_p * n)(*[_dptr(t).value for t in ts])
    hs = (ctypes.c_void_p * n)(*[c._h.value for c in contexts])
    ts = None if device_counter else (ctypes.c_void_p * n)(*[ctypes.addressof(c.t) for c in contexts])
    _check(load_library().nof_step_batch(hs, n, arr(Cs), arr(gammas), arr(ms), arr(vs), ts, arr(outs),
                                         ctypes.c_void_p(stream.cuda_stream)))


def energy_grad_batch(contexts, Cs, gammas, Es, gs=None, ggs=None, stream=None):
    """Evaluate several contexts concurrently (each on its own stream), forked from `stream`."""
    import torch
    n = len(contexts)
    stream = stream if stream is not None else torch.cuda.current_stream()
    arr = lambda ts: (ctypes.c_void_p * n)(*[None if t is None else _dptr(t).value for t in ts])
    hs = (ctypes.c_void_p * n)(*[c._h.value for c in contexts])
    _check(load_library().nof_energy_grad_batch(hs, n, arr(Cs), arr(gammas), arr(Es),
                                                None if gs is None else arr(gs),
                                                None if ggs is None else arr(ggs),
                                                ctypes.c_void_p(stream.cuda_stream)))


def _check(rc: int):
    if rc != NOF_OK:
        raise NofError(rc, load_library().nof_last_error().decode())


def _basis_struct(b: "inputs.Basis"):
    nprim = np.array([len(e) for e, _ in b.shells], np.int32)
    exps = np.array([x for e, _ in b.shells for x in e], np.float64)
    coefs = np.array([x for _, c in b.shells for x in c], np.float64)
    st = CBasis(len(b.shells), nprim.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                exps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                coefs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, (nprim, exps, coefs)


def _dptr(t):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One system (geometry + basis) on the current CUDA device and stream."""

    def __init__(self, precision: int = PREC_FP64, ipnof: int = 7, ncwo: int = 1, stream=None,
                 **opts):
        import torch
        lib = load_library()
        o = Options()
        lib.nof_default_options(ctypes.byref(o))
        o.precision, o.ipnof, o.ncwo = precision, ipnof, ncwo
        known = {name for name, _ in Options._fields_}
        for k, v in opts.items():
            if k not in known:  # a misspelt option would otherwise be ignored silently
                raise ValueError(f"unknown option {k!r}; the options are {sorted(known)}")
            setattr(o, k, v)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        _check(lib.nof_create(ctypes.byref(self._h), ctypes.byref(o), ctypes.c_void_p(self.stream.cuda_stream)))
        self.opts = o
        self.t = ctypes.c_int(0)
        self.sizes = None

    def close(self):
        if self._h:
            load_library().nof_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_B(self, xyz, orb, aux, Z=None, charge: int = 0, mult: int = 1):
        xyz = np.ascontiguousarray(xyz, np.float64)
        zarr = None if Z is None else np.ascontiguousarray(Z, np.float64)
        ob, keep1 = _basis_struct(orb)
        ab, keep2 = _basis_struct(aux)
        _check(load_library().nof_build_B(self._h, xyz.shape[0], xyz.ctypes.data_as(ctypes.c_void_p),
                                          None if zarr is None else zarr.ctypes.data_as(ctypes.c_void_p),
                                          charge, mult, ctypes.byref(ob), ctypes.byref(ab)))
        self.sizes = self.query()
        self.natom = int(xyz.shape[0])
        self.t = ctypes.c_int(0)
        return self.sizes

    def query(self):
        nbf, naux, nact, ng = (ctypes.c_int() for _ in range(4))
        vnn = ctypes.c_double()
        _check(load_library().nof_query(self._h, ctypes.byref(nbf), ctypes.byref(naux), ctypes.byref(nact),
                                        ctypes.byref(ng), ctypes.byref(vnn)))
        return dict(nbf=nbf.value, naux=naux.value, nact=nact.value, ngamma=ng.value, vnn=vnn.value)

    def _empty(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def get_SH(self):
        n = self.sizes["nbf"]
        S, H = self._empty(n, n), self._empty(n, n)
        _check(load_library().nof_get_SH(self._h, _dptr(S), _dptr(H)))
        return S, H

    def get_B(self):
        s = self.sizes
        B = self._empty(s["naux"], s["nbf"], s["nbf"])
        _check(load_library().nof_get_B(self._h, _dptr(B)))
        return B

    def split_digits(self) -> int:
        """Digits per operand element of the split path (4 or 5)."""
        nd = ctypes.c_int(0)
        _check(load_library().nof_split_digits(self._h, ctypes.byref(nd)))
        return nd.value

    def tuned_tiles(self):
        """(N tile of GEMM1, of GEMM2, of GEMM3, GEMM3 split-K chunk in atoms) chosen by the autotuner."""
        out = (ctypes.c_int * 4)()
        _check(load_library().nof_tuned_tiles(self._h, out))
        return tuple(out)

    def lowdin(self, Q):
        n = self.sizes["nbf"]
        C = self._empty(n, n)
        _check(load_library().nof_lowdin(self._h, _dptr(Q), _dptr(C)))
        return C

    def core_guess(self):
        """Core-Hamiltonian orbitals C0 and their energies (ascending)."""
        n = self.sizes["nbf"]
        C, eps = self._empty(n, n), self._empty(n)
        _check(load_library().nof_core_guess(self._h, _dptr(C), _dptr(eps)))
        return C, eps

    def jk(self, C, J=None, K=None):
        a = self.sizes["nact"]
        J = self._empty(a, a) if J is None else J
        K = self._empty(a, a) if K is None else K
        _check(load_library().nof_jk(self._h, _dptr(C), _dptr(J), _dptr(K)))
        return J, K

    def energy_grad(self, C, gamma, E=None, g=None, gg=None, grad: bool = True):
        s = self.sizes
        E = self._empty(1) if E is None else E
        if grad:
            g = self._empty(s["nbf"], s["nbf"]) if g is None else g
            gg = self._empty(s["ngamma"]) if gg is None else gg
        _check(load_library().nof_energy_grad(self._h, _dptr(C), _dptr(gamma), _dptr(E),
                                              _dptr(g) if grad else None, _dptr(gg) if grad else None))
        return E, g, gg

    def step(self, C, gamma, m, v, out=None, device_counter: bool = False):
        """One alternating step (nof_step). device_counter: keep the ADAM step counter on the
        device (t == NULL), which makes the call capturable in a CUDA graph."""
        out = self._empty(3) if out is None else out
        _check(load_library().nof_step(self._h, _dptr(C), _dptr(gamma), _dptr(m), _dptr(v),
                                       None if device_counter else ctypes.byref(self.t), _dptr(out)))
        return out

    def optimize(self, C, gamma, **params):
        """The converged ON / NO loop (nof_optimize) from (C, gamma), in place. params: fields of
        nof_opt_params. Returns dict(E, gnorm, lam_asym, iterations, evaluations, converged, lr,
        on_steps, history [iterations][3] of (E_k, ||g_k||, lr_k))."""
        lib = load_library()
        p = OptParams()
        lib.nof_default_opt_params(ctypes.byref(p))
        known = {name for name, _ in OptParams._fields_}
        for k, v in params.items():
            if k not in known:
                raise ValueError(f"unknown parameter {k!r}; the parameters are {sorted(known)}")
            setattr(p, k, v)
        hist = np.zeros((p.maxit, 3))
        res = np.zeros(8)
        _check(lib.nof_optimize(self._h, _dptr(C), _dptr(gamma), ctypes.byref(p),
                                hist.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p)))
        it = int(res[3])
        return dict(E=float(res[0]), gnorm=float(res[1]), lam_asym=float(res[2]), iterations=it,
                    evaluations=int(res[4]), converged=bool(res[5]), lr=float(res[6]), on_steps=int(res[7]),
                    history=hist[:it].copy())

    def nuclear_gradient(self, C, gamma, grad=None):
        """dE/dR [natom][3] at (C, gamma) along the orbital connection (nof_nuclear_gradient)."""
        import torch
        natom = self.natom
        grad = torch.empty(natom, 3, dtype=torch.float64, device="cuda") if grad is None else grad
        _check(load_library().nof_nuclear_gradient(self._h, _dptr(C), _dptr(gamma), _dptr(grad)))
        return grad

    def set_field(self, F):
        """Static field F = (Fx, Fy, Fz) in atomic units for every later call (nof_set_field)."""
        f = np.ascontiguousarray(F, np.float64)
        if f.shape != (3,):
            raise ValueError("F has three components")
        _check(load_library().nof_set_field(self._h, f.ctypes.data_as(ctypes.c_void_p)))

    def dipole(self, C, gamma, mu=None):
        """Dipole moment (3,) of the state (C, gamma) as a device tensor (nof_dipole)."""
        mu = self._empty(3) if mu is None else mu
        _check(load_library().nof_dipole(self._h, _dptr(C), _dptr(gamma), _dptr(mu)))
        return mu

    def profile(self, which: int = 1):
        """Time one contraction of every later evaluation (1 half transform, 2 full transform,
        3 Lagrangian contraction; 0 or False: off) with CUDA events (nof_profile)."""
        _check(load_library().nof_profile(self._h, int(which)))

    def profile_read(self):
        ms, cnt, name = ctypes.c_double(), ctypes.c_int(), ctypes.c_char_p()
        _check(load_library().nof_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(name)))
        return ms.value, cnt.value, (name.value or b"").decode()

    def sync(self):
        _check(load_library().nof_sync(self._h))
