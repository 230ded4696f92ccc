"""ctypes wrapper over the plain serial FP64 UA-AMG oracle (``uaamg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU-baseline leg
of the benchmark.  The product package never imports this module.

Every function mirrors one routine of the C file; see that file for the passages of the
paper each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "uaamg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_uaamg.so")

MAXIMAL, SINGLE_ROUND = 0, 1
OR_OK, OR_ERR_NO_CONVERGENCE = 0, 4


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain C, no FP contraction, same bits on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("coarse_size", C.c_int32), ("max_levels", C.c_int32),
                ("max_agg_size", C.c_int32), ("pass_mode", C.c_int32), ("seed", C.c_uint64),
                ("pre", C.c_int32), ("post", C.c_int32), ("kcycle_inner", C.c_int32),
                ("kcycle_tau", C.c_double), ("max_iter", C.c_int32), ("agg_repeat", C.c_int32),
                ("kcycle_ratio", C.c_double), ("min_coarsening", C.c_double),
                ("jacobi_omega", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P, I32, I64, U64, D = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double)
        sig = {
            "or_fmix32": (C.c_uint32, [C.c_uint32]),
            "or_level_salt": (C.c_uint32, [U64, I32]),
            "or_priorities": (None, [I32, P, P, U64, I32, P]),
            "or_paa": (I32, [I32, P, P, P, I32, I32, P, P]),
            "or_renumber": (I32, [I32, P, P]),
            "or_coarse": (I64, [I32, P, P, P, P, I32, P, P, P, I64]),
            "or_minv": (None, [I32, P, P, P, P]),
            "or_cholesky": (I32, [I32, P]),
            "or_cholesky_solve": (None, [I32, P, P, P]),
            "or_setup": (P, [I32, P, P, P, C.POINTER(_Params), C.POINTER(I32)]),
            "or_free": (None, [P]),
            "or_num_levels": (I32, [P]),
            "or_level_n": (I32, [P, I32]),
            "or_level_nnz": (I64, [P, I32]),
            "or_level_passes": (I32, [P, I32]),
            "or_level_csr": (None, [P, I32, P, P, P]),
            "or_level_agg": (None, [P, I32, P]),
            "or_level_pass_of": (None, [P, I32, P]),
            "or_level_minv": (None, [P, I32, P]),
            "or_apply_B": (None, [P, I32, P, P]),
            "or_apply_K": (None, [P, I32, P, P]),
            "or_solve": (I32, [P, P, P, D, I32, C.POINTER(I32), C.POINTER(D), P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def fmix32(h: int) -> int:
    return int(lib().or_fmix32(h & 0xFFFFFFFF))


def level_salt(seed: int, level: int) -> int:
    return int(lib().or_level_salt(seed, level))


def priorities(rowptr, col, seed: int, level: int = 0) -> np.ndarray:
    rowptr, col = _i32(rowptr), _i32(col)
    n = len(rowptr) - 1
    P = np.empty(n, dtype=np.uint64)
    lib().or_priorities(n, _p(rowptr), _p(col), seed, level, _p(P))
    return P


def paa(rowptr, col, P, t: int = 5, mode: int = MAXIMAL):
    """Algorithm 2: returns (root_of, pass_of, npasses)."""
    rowptr, col = _i32(rowptr), _i32(col)
    P = np.ascontiguousarray(P, dtype=np.uint64)
    n = len(rowptr) - 1
    root_of = np.empty(n, np.int32)
    pass_of = np.empty(n, np.int32)
    npass = lib().or_paa(n, _p(rowptr), _p(col), _p(P), t, mode, _p(root_of), _p(pass_of))
    if npass < 0:
        raise ValueError("or_paa: bad argument")
    return root_of, pass_of, int(npass)


def renumber(root_of):
    root_of = _i32(root_of)
    agg = np.empty(len(root_of), np.int32)
    nc = lib().or_renumber(len(root_of), _p(root_of), _p(agg))
    return agg, int(nc)


def coarse(rowptr, col, val, agg, nc: int):
    """Eq. (2.4): returns (rowptr_c, col_c, val_c)."""
    rowptr, col, val, agg = _i32(rowptr), _i32(col), _f64(val), _i32(agg)
    n = len(rowptr) - 1
    cap = max(1, len(col))
    rc = np.empty(nc + 1, np.int32)
    cc = np.empty(cap, np.int32)
    vc = np.empty(cap, np.float64)
    z = lib().or_coarse(n, _p(rowptr), _p(col), _p(val), _p(agg), nc, _p(rc), _p(cc), _p(vc), cap)
    if z < 0:
        raise RuntimeError("or_coarse: capacity")
    return rc, cc[:z].copy(), vc[:z].copy()


def minv(rowptr, col, val):
    rowptr, col, val = _i32(rowptr), _i32(col), _f64(val)
    out = np.empty(len(rowptr) - 1)
    lib().or_minv(len(rowptr) - 1, _p(rowptr), _p(col), _p(val), _p(out))
    return out


def cholesky(A):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    rc = lib().or_cholesky(A.shape[0], _p(A))
    if rc != 0:
        raise np.linalg.LinAlgError(f"pivot {-rc - 1} not positive")
    return np.tril(A)


def cholesky_solve(L, b):
    L, b = _f64(L), _f64(b)
    x = np.empty_like(b)
    lib().or_cholesky_solve(len(b), _p(L), _p(b), _p(x))
    return x


@dataclass
class Params:
    coarse_size: int = 64
    max_levels: int = 25
    max_agg_size: int = 5
    pass_mode: int = SINGLE_ROUND
    seed: int = 0x5EED
    pre: int = 1
    post: int = 1
    kcycle_inner: int = 2
    kcycle_tau: float = 0.0
    max_iter: int = 200
    agg_repeat: int = 1
    kcycle_ratio: float = 0.0
    min_coarsening: float = 0.0
    jacobi_omega: float = 0.0

    def c(self) -> _Params:
        return _Params(self.coarse_size, self.max_levels, self.max_agg_size, self.pass_mode,
                       self.seed, self.pre, self.post, self.kcycle_inner, self.kcycle_tau,
                       self.max_iter, self.agg_repeat, self.kcycle_ratio, self.min_coarsening,
                       self.jacobi_omega)


class Hierarchy:
    """Algorithm 1 setup in FP64; owns the C-side hierarchy."""

    def __init__(self, rowptr, col, val, params: Params | None = None):
        self.params = params or Params()
        rowptr, col, val = _i32(rowptr), _i32(col), _f64(val)
        st = C.c_int32(0)
        cp = self.params.c()
        self._h = lib().or_setup(len(rowptr) - 1, _p(rowptr), _p(col), _p(val), C.byref(cp),
                                 C.byref(st))
        if not self._h:
            raise RuntimeError(f"or_setup failed with status {st.value}")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_free(self._h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return int(lib().or_num_levels(self._h))

    def n(self, l: int) -> int:
        return int(lib().or_level_n(self._h, l))

    def nnz(self, l: int) -> int:
        return int(lib().or_level_nnz(self._h, l))

    def passes(self, l: int) -> int:
        return int(lib().or_level_passes(self._h, l))

    def csr(self, l: int):
        n, z = self.n(l), self.nnz(l)
        rp, cc, vv = np.empty(n + 1, np.int32), np.empty(z, np.int32), np.empty(z)
        lib().or_level_csr(self._h, l, _p(rp), _p(cc), _p(vv))
        return rp, cc, vv

    def agg(self, l: int):
        a = np.empty(self.n(l), np.int32)
        lib().or_level_agg(self._h, l, _p(a))
        return a

    def pass_of(self, l: int):
        a = np.empty(self.n(l), np.int32)
        lib().or_level_pass_of(self._h, l, _p(a))
        return a

    def minv(self, l: int):
        a = np.empty(self.n(l))
        lib().or_level_minv(self._h, l, _p(a))
        return a

    def apply_B(self, l: int, r):
        r = _f64(r)
        x = np.empty_like(r)
        lib().or_apply_B(self._h, l, _p(r), _p(x))
        return x

    def apply_K(self, m: int, rho):
        rho = _f64(rho)
        e = np.empty_like(rho)
        lib().or_apply_K(self._h, m, _p(rho), _p(e))
        return e

    def solve(self, b, tol: float = 1e-8, x0=None):
        """Returns (x, iters, relres, status, history)."""
        b = _f64(b)
        x = _f64(x0).copy() if x0 is not None else np.zeros_like(b)
        it, rr = C.c_int32(0), C.c_double(0.0)
        hist = np.zeros(self.params.max_iter + 1)
        st = lib().or_solve(self._h, _p(b), _p(x), tol, int(x0 is not None), C.byref(it),
                            C.byref(rr), _p(hist))
        return x, int(it.value), float(rr.value), int(st), hist[: it.value + 1].copy()
