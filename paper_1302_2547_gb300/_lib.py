"""ctypes binding of libuaamg (include/uaamg.h): the same entry points, argument
marshalling only.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
every computation runs in the library's CUDA kernels.  Importing this module does not load
the library; the first call does, and raises if the CUDA library has not been built."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libuaamg.so")

UAAMG_OK = 0
UAAMG_ERR_NO_CONVERGENCE = 4
UAAMG_ERR_TIMEOUT = 8
UAAMG_ERR_CANCELLED = 10
UAAMG_FP64, UAAMG_MIXED = 0, 1
UAAMG_PASS_MAXIMAL, UAAMG_PASS_SINGLE_ROUND = 0, 1
UAAMG_KCLASS_SMOOTH0, UAAMG_KCLASS_SPMV64, UAAMG_KCLASS_PAA, UAAMG_KCLASS_COARSE = 1, 2, 3, 4
UAAMG_KCLASS_SRA = 5

# every symbol declared in include/uaamg.h
EXPORTS = [
    "uaamg_default_params", "uaamg_setup", "uaamg_solve", "uaamg_free", "uaamg_num_levels",
    "uaamg_level_info", "uaamg_get_aggregates", "uaamg_get_level_csr", "uaamg_get_priorities",
    "uaamg_get_pass_of", "uaamg_get_minv", "uaamg_apply_B", "uaamg_apply_K",
    "uaamg_residual_history", "uaamg_get_stats", "uaamg_set_profiling", "uaamg_get_profile",
    "uaamg_total_launches", "uaamg_set_memory_budget", "uaamg_memory_in_use",
    "uaamg_status_string", "uaamg_aggregate_static", "uaamg_solve_many",
    "uaamg_server_create", "uaamg_server_submit", "uaamg_server_poll", "uaamg_server_wait",
    "uaamg_server_stats", "uaamg_server_destroy", "uaamg_server_cancel",
    "uaamg_solve_batch", "uaamg_setup_batch", "uaamg_measure_fp64_fma",
    "uaamg_server_wait_answer", "uaamg_level_kernel",
]


class uaamg_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int32)]


class uaamg_params(C.Structure):
    _fields_ = [("coarse_size", C.c_int32), ("max_levels", C.c_int32),
                ("max_agg_size", C.c_int32), ("pass_mode", C.c_int32), ("seed", C.c_uint64),
                ("pre", C.c_int32), ("post", C.c_int32), ("kcycle_inner", C.c_int32),
                ("kcycle_tau", C.c_double), ("precision", C.c_int32), ("max_iter", C.c_int32),
                ("use_graphs", C.c_int32), ("profile_class", C.c_int32),
                ("agg_repeat", C.c_int32), ("kcycle_ratio", C.c_double),
                ("min_coarsening", C.c_double), ("jacobi_omega", C.c_double),
                ("tma_rows", C.c_int32), ("sell_rows", C.c_int32), ("fuse_below", C.c_int32),
                ("sra_rounds", C.c_int32), ("restrict_fuse_below", C.c_int32),
                ("autotune", C.c_int32), ("cluster_below", C.c_int32),
                ("wait_limit_ns", C.c_int64)]


class uaamg_stats(C.Structure):
    _fields_ = [("setup_ms", C.c_double), ("solve_ms", C.c_double), ("launches", C.c_int64),
                ("graph_nodes", C.c_int64), ("opc", C.c_double),
                ("grid_complexity", C.c_double), ("device_bytes", C.c_uint64),
                ("tail_level", C.c_int32), ("tail_blocks", C.c_int32)]


class uaamg_answer(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("batch", C.c_int32),
                ("cache_hit", C.c_int32), ("relres", C.c_double), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


class UaamgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib = None


def lib() -> C.CDLL:
    """Loads libuaamg.so; raises when it has not been built (there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libuaamg.so is not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "uaamg_default_params": (None, [C.POINTER(uaamg_params)]),
            "uaamg_setup": (C.c_int, [C.POINTER(uaamg_csr), C.POINTER(uaamg_params), P,
                                      C.POINTER(P)]),
            "uaamg_solve": (C.c_int, [P, P, P, D, I32, C.POINTER(I32), C.POINTER(D)]),
            "uaamg_free": (None, [P]),
            "uaamg_num_levels": (C.c_int, [P, C.POINTER(I32)]),
            "uaamg_level_info": (C.c_int, [P, I32, C.POINTER(I32), C.POINTER(I32),
                                           C.POINTER(I32)]),
            "uaamg_get_aggregates": (C.c_int, [P, I32, P]),
            "uaamg_get_level_csr": (C.c_int, [P, I32, P, P, P]),
            "uaamg_get_priorities": (C.c_int, [P, I32, P]),
            "uaamg_get_pass_of": (C.c_int, [P, I32, P]),
            "uaamg_get_minv": (C.c_int, [P, I32, P]),
            "uaamg_apply_B": (C.c_int, [P, I32, P, P]),
            "uaamg_apply_K": (C.c_int, [P, I32, P, P]),
            "uaamg_residual_history": (C.c_int, [P, P, I32, C.POINTER(I32)]),
            "uaamg_get_stats": (C.c_int, [P, C.POINTER(uaamg_stats)]),
            "uaamg_set_profiling": (C.c_int, [P, I32]),
            "uaamg_get_profile": (C.c_int, [P, C.POINTER(I64), C.POINTER(D), C.POINTER(D)]),
            "uaamg_total_launches": (I64, []),
            "uaamg_set_memory_budget": (C.c_int, [U64]),
            "uaamg_memory_in_use": (U64, []),
            "uaamg_status_string": (C.c_char_p, [C.c_int]),
            "uaamg_aggregate_static": (C.c_int, [C.POINTER(uaamg_csr), I32, I32, U64, P,
                                                 C.POINTER(I32), P]),
            "uaamg_solve_many": (C.c_int, [P, I32, P, P, D, P, P]),
            "uaamg_server_create": (C.c_int, [C.POINTER(uaamg_params), U64, I32, I32,
                                              C.POINTER(P)]),
            "uaamg_server_submit": (C.c_int, [P, C.POINTER(uaamg_csr), U64, P, D,
                                              C.POINTER(U64)]),
            "uaamg_server_poll": (C.c_int, [P, U64, C.POINTER(I32)]),
            "uaamg_server_wait": (C.c_int, [P, U64, P, C.POINTER(I32), C.POINTER(D),
                                            C.POINTER(D), C.POINTER(I32)]),
            "uaamg_server_stats": (C.c_int, [P, C.POINTER(U64), C.POINTER(U64), C.POINTER(U64),
                                             C.POINTER(U64), C.POINTER(U64), C.POINTER(I32)]),
            "uaamg_server_destroy": (None, [P]),
            "uaamg_server_cancel": (C.c_int, [P, U64, C.POINTER(I32)]),
            "uaamg_solve_batch": (C.c_int, [P, I32, P, P, P, D, P, P, P]),
            "uaamg_setup_batch": (C.c_int, [I32, P, P, I32, P, P]),
            "uaamg_measure_fp64_fma": (C.c_int, [I32, C.POINTER(D)]),
            "uaamg_server_wait_answer": (C.c_int, [P, U64, P, C.POINTER(uaamg_answer)]),
            "uaamg_level_kernel": (C.c_int, [P, I32, C.POINTER(I32), C.POINTER(I32), P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().uaamg_status_string(status).decode()


def check(status: int, where: str = "uaamg") -> int:
    if status != UAAMG_OK:
        raise UaamgError(status, where)
    return status


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):  # torch.cuda.Stream
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def uaamg_default_params(**overrides) -> uaamg_params:
    p = uaamg_params()
    lib().uaamg_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def uaamg_setup(rowptr, col, val, params: uaamg_params | None = None, stream=None):
    """Returns a handle (c_void_p).  rowptr/col int32, val float64; all host or all device."""
    (rp, d0), (cp, d1), (vp, d2) = _ptr(rowptr), _ptr(col), _ptr(val)
    if not (d0 == d1 == d2):
        raise ValueError("rowptr, col and val must all be host or all device arrays")
    n = int(rowptr.shape[0]) - 1
    A = uaamg_csr(n, int(col.shape[0]), rp, cp, vp, d0)
    h = C.c_void_p()
    check(lib().uaamg_setup(C.byref(A), C.byref(params) if params is not None else None,
                            _stream(stream), C.byref(h)), "uaamg_setup")
    return h


def uaamg_solve(h, b, x, tol: float = 1e-8, use_guess: bool = False):
    """Returns (status, iters, relres); status may be UAAMG_ERR_NO_CONVERGENCE."""
    it, rr = C.c_int32(0), C.c_double(0.0)
    st = lib().uaamg_solve(h, _ptr(b)[0], _ptr(x)[0], tol, int(use_guess), C.byref(it),
                           C.byref(rr))
    if st not in (UAAMG_OK, UAAMG_ERR_NO_CONVERGENCE):
        check(st, "uaamg_solve")
    return st, int(it.value), float(rr.value)


def uaamg_solve_many(h, B, X, tol: float = 1e-8):
    """B, X: [n][nrhs] float64 (numpy or torch, host or device).  Returns
    (status, iters[nrhs], relres[nrhs])."""
    nrhs = int(B.shape[1])
    it = np.zeros(nrhs, np.int32)
    rr = np.zeros(nrhs)
    st = lib().uaamg_solve_many(h, nrhs, _ptr(B)[0], _ptr(X)[0], tol, it.ctypes.data,
                                rr.ctypes.data)
    if st not in (UAAMG_OK, UAAMG_ERR_NO_CONVERGENCE):
        check(st, "uaamg_solve_many")
    return st, it, rr


def uaamg_solve_batch(handles, Bs, Xs, tol: float = 1e-8, stream=None):
    """Solves len(handles) systems together.  Bs[s], Xs[s]: [n_s][nrhs_s] float64 (numpy or
    torch, host or device; a 1-D array is one right-hand side).  Returns (status,
    iters list of arrays, relres list of arrays), one array per system."""
    ns = len(handles)
    if not (len(Bs) == len(Xs) == ns) or ns < 1:
        raise ValueError("one B and one X per handle")
    nr = np.array([1 if len(B.shape) == 1 else int(B.shape[1]) for B in Bs], np.int32)
    hp = (C.c_void_p * ns)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    bp = (C.c_void_p * ns)(*[_ptr(B)[0] for B in Bs])
    xp = (C.c_void_p * ns)(*[_ptr(X)[0] for X in Xs])
    it = np.zeros(int(nr.sum()), np.int32)
    rr = np.zeros(int(nr.sum()))
    st = lib().uaamg_solve_batch(hp, ns, nr.ctypes.data, bp, xp, tol, it.ctypes.data,
                                 rr.ctypes.data, _stream(stream))
    if st not in (UAAMG_OK, UAAMG_ERR_NO_CONVERGENCE):
        check(st, "uaamg_solve_batch")
    off = np.concatenate([[0], np.cumsum(nr)])
    return st, [it[off[s]:off[s + 1]] for s in range(ns)], [rr[off[s]:off[s + 1]]
                                                              for s in range(ns)]


def uaamg_setup_batch(mats, params=None, threads: int = 8, stream=None):
    """uaamg_setup of every (rowptr, col, val) in `mats` on `threads` host threads; each
    triple is all host (numpy) or all device (torch CUDA) arrays.  `params` is one
    uaamg_params for all or a list of one per matrix.  Returns the list of handles."""
    ns = len(mats)
    keep = []
    csr = (uaamg_csr * ns)()
    for s, (rp, cc, vv) in enumerate(mats):
        if not hasattr(rp, "data_ptr"):
            rp = np.ascontiguousarray(rp, np.int32)
            cc = np.ascontiguousarray(cc, np.int32)
            vv = np.ascontiguousarray(vv, np.float64)
        keep += [rp, cc, vv]
        (a, d0), (b, d1), (c, d2) = _ptr(rp), _ptr(cc), _ptr(vv)
        if not (d0 == d1 == d2):
            raise ValueError("rowptr, col and val must all be host or all device arrays")
        csr[s] = uaamg_csr(int(rp.shape[0]) - 1, int(cc.shape[0]), a, b, c, d0)
    if params is None:
        pp = None
    else:
        plist = params if isinstance(params, (list, tuple)) else [params] * ns
        pp = (uaamg_params * ns)(*plist)
    out = (C.c_void_p * ns)()
    check(lib().uaamg_setup_batch(ns, csr, pp, threads, _stream(stream), out),
          "uaamg_setup_batch")
    return [C.c_void_p(out[s]) for s in range(ns)]


def uaamg_free(h):
    if h:
        lib().uaamg_free(h)


def uaamg_num_levels(h) -> int:
    v = C.c_int32(0)
    check(lib().uaamg_num_levels(h, C.byref(v)), "uaamg_num_levels")
    return v.value


def uaamg_level_info(h, l: int):
    n, z, p = C.c_int32(), C.c_int32(), C.c_int32()
    check(lib().uaamg_level_info(h, l, C.byref(n), C.byref(z), C.byref(p)), "uaamg_level_info")
    return n.value, z.value, p.value


def uaamg_get_aggregates(h, l: int) -> np.ndarray:
    n, _, _ = uaamg_level_info(h, l)
    a = np.empty(n, np.int32)
    check(lib().uaamg_get_aggregates(h, l, a.ctypes.data), "uaamg_get_aggregates")
    return a


def uaamg_get_level_csr(h, l: int):
    n, z, _ = uaamg_level_info(h, l)
    rp, cc, vv = np.empty(n + 1, np.int32), np.empty(z, np.int32), np.empty(z)
    check(lib().uaamg_get_level_csr(h, l, rp.ctypes.data, cc.ctypes.data, vv.ctypes.data),
          "uaamg_get_level_csr")
    return rp, cc, vv


def uaamg_get_priorities(h, l: int) -> np.ndarray:
    n, _, _ = uaamg_level_info(h, l)
    a = np.empty(n, np.uint64)
    check(lib().uaamg_get_priorities(h, l, a.ctypes.data), "uaamg_get_priorities")
    return a


def uaamg_get_pass_of(h, l: int) -> np.ndarray:
    n, _, _ = uaamg_level_info(h, l)
    a = np.empty(n, np.int32)
    check(lib().uaamg_get_pass_of(h, l, a.ctypes.data), "uaamg_get_pass_of")
    return a


def uaamg_level_kernel(h, l: int) -> dict:
    """{"path": 0 row-block / 1 TMA / 2 ELLPACK, "rows": rows per block, "tune_us": the
    autotuner's six first-sweep timings (-1 = not timed)}."""
    p, r = C.c_int32(), C.c_int32()
    us = np.zeros(6)
    check(lib().uaamg_level_kernel(h, l, C.byref(p), C.byref(r), us.ctypes.data),
          "uaamg_level_kernel")
    return {"path": p.value, "rows": r.value, "tune_us": [round(float(u), 2) for u in us]}


def uaamg_get_minv(h, l: int) -> np.ndarray:
    n, _, _ = uaamg_level_info(h, l)
    a = np.empty(n)
    check(lib().uaamg_get_minv(h, l, a.ctypes.data), "uaamg_get_minv")
    return a


def uaamg_apply_B(h, l: int, v) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    check(lib().uaamg_apply_B(h, l, v.ctypes.data, out.ctypes.data), "uaamg_apply_B")
    return out


def uaamg_apply_K(h, m: int, v) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    check(lib().uaamg_apply_K(h, m, v.ctypes.data, out.ctypes.data), "uaamg_apply_K")
    return out


def uaamg_residual_history(h, cap: int = 4096) -> np.ndarray:
    a = np.empty(cap)
    k = C.c_int32(0)
    check(lib().uaamg_residual_history(h, a.ctypes.data, cap, C.byref(k)),
          "uaamg_residual_history")
    return a[: k.value].copy()


def uaamg_get_stats(h) -> dict:
    s = uaamg_stats()
    check(lib().uaamg_get_stats(h, C.byref(s)), "uaamg_get_stats")
    return {k: getattr(s, k) for k, _ in uaamg_stats._fields_}


def uaamg_set_profiling(h, kclass: int):
    check(lib().uaamg_set_profiling(h, kclass), "uaamg_set_profiling")


def uaamg_get_profile(h):
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    check(lib().uaamg_get_profile(h, C.byref(n), C.byref(ms), C.byref(by)), "uaamg_get_profile")
    return n.value, ms.value, by.value


def uaamg_measure_fp64_fma(chains: int = 8) -> float:
    """FP64 FMA per second of the current device (1 or 8 independent chains per thread)."""
    v = C.c_double(0.0)
    check(lib().uaamg_measure_fp64_fma(chains, C.byref(v)), "uaamg_measure_fp64_fma")
    return v.value


def uaamg_total_launches() -> int:
    return int(lib().uaamg_total_launches())


def uaamg_set_memory_budget(nbytes: int):
    check(lib().uaamg_set_memory_budget(nbytes), "uaamg_set_memory_budget")


def uaamg_memory_in_use() -> int:
    return int(lib().uaamg_memory_in_use())


def _dtype_name(a) -> str:
    return str(a.dtype).replace("torch.", "")


def uaamg_aggregate_static(rowptr, col, val, agg, max_agg_size: int = 5,
                           pass_mode: int = UAAMG_PASS_SINGLE_ROUND, seed: int = 0x5EED,
                           stream=None) -> int:
    """Level-0 aggregation into the caller's device buffer `agg` (int32[n]) with no device
    allocation by the library; returns the number of aggregates.  All arrays are CUDA
    tensors on the current device: rowptr int32[n+1], col int32[nnz], val float64[nnz],
    agg int32 with at least n entries.  Anything else raises ValueError before the C call
    (the library cannot see the length of a device buffer)."""
    arrs = {"rowptr": rowptr, "col": col, "val": val, "agg": agg}
    want = {"rowptr": "int32", "col": "int32", "val": "float64", "agg": "int32"}
    for k, a in arrs.items():
        if not hasattr(a, "dtype") or _dtype_name(a) != want[k]:
            raise ValueError(f"{k} must be {want[k]}, not {getattr(a, 'dtype', type(a))}")
        if len(a.shape) != 1:
            raise ValueError(f"{k} must be one-dimensional")
    n = int(rowptr.shape[0]) - 1
    if n < 1:
        raise ValueError("rowptr must hold n + 1 >= 2 entries")
    if int(col.shape[0]) != int(val.shape[0]):
        raise ValueError("col and val must have the same length")
    if int(agg.shape[0]) < n:
        raise ValueError(f"agg holds {int(agg.shape[0])} entries, fewer than n = {n}")
    for k, a in arrs.items():
        if not hasattr(a, "is_cuda") or not a.is_cuda:
            raise ValueError(f"uaamg_aggregate_static takes CUDA tensors only ({k})")
    import torch

    cur = torch.cuda.current_device()
    for k, a in arrs.items():
        if a.device.index != cur:
            raise ValueError(f"{k} is on cuda:{a.device.index}, not the current cuda:{cur}")
    (rp, _), (cp, _), (vp, _), (ap, _) = _ptr(rowptr), _ptr(col), _ptr(val), _ptr(agg)
    A = uaamg_csr(n, int(col.shape[0]), rp, cp, vp, 1)
    nc = C.c_int32(0)
    check(lib().uaamg_aggregate_static(C.byref(A), max_agg_size, pass_mode, seed, ap,
                                       C.byref(nc), _stream(stream)), "uaamg_aggregate_static")
    return nc.value


class Server:
    """uaamg_server_*: queued solves with a device-resident hierarchy cache and batching of
    requests for the same matrix.  Arrays are host numpy arrays (copied at submit)."""

    def __init__(self, params: uaamg_params | None = None, budget_bytes: int = 0,
                 workers: int = 2, max_batch: int = 16):
        self._s = C.c_void_p()
        check(lib().uaamg_server_create(C.byref(params) if params is not None else None,
                                        budget_bytes, workers, max_batch, C.byref(self._s)),
              "uaamg_server_create")
        self._n = {}

    def submit(self, rowptr, col, val, b, tol: float = 1e-8, key: int = 0) -> int:
        rowptr = np.ascontiguousarray(rowptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        A = uaamg_csr(len(rowptr) - 1, len(col), rowptr.ctypes.data, col.ctypes.data,
                      val.ctypes.data, 0)
        t = C.c_uint64(0)
        check(lib().uaamg_server_submit(self._s, C.byref(A), key, b.ctypes.data, tol,
                                        C.byref(t)), "uaamg_server_submit")
        self._n[t.value] = len(rowptr) - 1
        return t.value

    def poll(self, ticket: int) -> bool:
        d = C.c_int32(0)
        check(lib().uaamg_server_poll(self._s, ticket, C.byref(d)), "uaamg_server_poll")
        return bool(d.value)

    def wait(self, ticket: int):
        """Returns (status, x, iters, relres, latency_ms, batch)."""
        x = np.zeros(self._n.pop(ticket))
        it, rr, lat, bt = C.c_int32(), C.c_double(), C.c_double(), C.c_int32()
        st = lib().uaamg_server_wait(self._s, ticket, x.ctypes.data, C.byref(it), C.byref(rr),
                                     C.byref(lat), C.byref(bt))
        return st, x, it.value, rr.value, lat.value, bt.value

    def cancel(self, ticket: int) -> bool:
        """True when the request was withdrawn before any worker took it."""
        c = C.c_int32(0)
        check(lib().uaamg_server_cancel(self._s, ticket, C.byref(c)), "uaamg_server_cancel")
        return bool(c.value)

    def wait_answer(self, ticket: int):
        """Returns (x, answer dict with status, iters, batch, cache_hit, relres, latency_ms,
        queue_ms, setup_ms, solve_ms)."""
        x = np.zeros(self._n.pop(ticket))
        a = uaamg_answer()
        lib().uaamg_server_wait_answer(self._s, ticket, x.ctypes.data, C.byref(a))
        return x, {k: getattr(a, k) for k, _ in uaamg_answer._fields_}

    def stats(self) -> dict:
        v = [C.c_uint64() for _ in range(5)]
        c = C.c_int32()
        check(lib().uaamg_server_stats(self._s, *[C.byref(x) for x in v], C.byref(c)),
              "uaamg_server_stats")
        keys = ("done", "batches", "cache_hits", "setups", "rejected")
        out = {k: x.value for k, x in zip(keys, v)}
        out["cached"] = c.value
        return out

    def close(self):
        if self._s:
            lib().uaamg_server_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()
