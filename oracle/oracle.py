"""CPU oracle for the exact ddKS statistic (arXiv 2106.13706) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The product
library never loads it, and it shares no code with the CUDA path: the plain C
loops live in ``ddks_oracle.c`` next to this file and are compiled with gcc.

Functions and the passages they follow:

* :func:`ddks` -- Sec. 2.1, Eq. (ddks_tensor_definition) with the loop method
  of Sec. 2.1 and the ">=" split of Eq. (g) (Sec. 2.2.1); the normalised
  difference of Eq. (abs_difference) kept as the integer |cP*NT - cT*NP|.
* :func:`perm_key`, :func:`perm_labels`, :func:`permutation_test` --
  the permutation test of Sec. 4.2 (Philox4x64-10 relabelling).
* :func:`significance` -- Sec. 3, Eq. (binomial_probability) and
  Eq. (ddks_significance).
* :func:`brute_force_ddks` -- a pure-Python/numpy restatement of the same
  definition for tiny inputs (used to pin the C loops).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

ORC_OK = 0
_ERRORS = {-1: "invalid argument", -2: "NaN in input", -3: "NP*NT too large", -4: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {_ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ddks_oracle.c with gcc (OpenMP when available) into liboracle.so."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # no fused multiply-add: the rdKS distances are summed as written
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
            vp = ctypes.c_void_p
            lib.oracle_ddks.argtypes = [vp, i64, vp, i64, i32, i32, i64, i64, i32,
                                        ctypes.POINTER(u64), ctypes.POINTER(i64),
                                        ctypes.POINTER(ctypes.c_int32), vp]
            lib.oracle_ddks.restype = i32
            lib.oracle_philox4x64_10.argtypes = [vp, vp, vp]
            lib.oracle_philox4x64_10.restype = None
            lib.oracle_perm_key.argtypes = [u64, i64, i64]
            lib.oracle_perm_key.restype = u64
            lib.oracle_perm_labels.argtypes = [u64, i64, i64, i64, vp]
            lib.oracle_perm_labels.restype = i32
            lib.oracle_permutation_test.argtypes = [vp, i64, vp, i64, i32, i32, i64, u64, i32,
                                                    ctypes.POINTER(u64), vp,
                                                    ctypes.POINTER(ctypes.c_double)]
            lib.oracle_permutation_test.restype = i32
            lib.oracle_cell_p_le.argtypes = [i64, i64, u64, ctypes.c_double, i32]
            lib.oracle_cell_p_le.restype = ctypes.c_double
            lib.oracle_significance.argtypes = [vp, i64, vp, i64, i32, i32, u64, i32, i32,
                                                ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double)]
            lib.oracle_significance.restype = i32
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = i32
            lib.oracle_vdks.argtypes = [vp, i64, vp, i64, i32, i32, i32, ctypes.POINTER(u64),
                                        ctypes.POINTER(i64), ctypes.POINTER(i32)]
            lib.oracle_vdks.restype = i32
            lib.oracle_rdks.argtypes = [vp, i64, vp, i64, i32, i32, ctypes.POINTER(u64), vp]
            lib.oracle_rdks.restype = i32
            _lib = lib
    return _lib


def _prep(P, T):
    P = np.asarray(P)
    T = np.asarray(T)
    if P.ndim == 1:
        P = P[:, None]
    if T.ndim == 1:
        T = T[:, None]
    if P.dtype not in (np.float32, np.float64):
        P = P.astype(np.float64)
    dt = np.float64 if (P.dtype == np.float64 or T.dtype == np.float64) else np.float32
    P = np.ascontiguousarray(P, dtype=dt)
    T = np.ascontiguousarray(T, dtype=dt)
    if P.shape[1] != T.shape[1]:
        raise ValueError("P and T must have the same dimension")
    return P, T, int(dt == np.float64)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def ddks(P, T, origins=None, nthreads: int = 0, per_origin: bool = False):
    """Exact ddKS over the pooled origins [o_begin, o_end).

    Returns dict(num_max, denom, D, argmax_origin, argmax_orthant[, per_origin]).
    """
    lib = _load()
    P, T, f64 = _prep(P, T)
    NP, d = P.shape
    NT = T.shape[0]
    N = NP + NT
    ob, oe = (0, N) if origins is None else (int(origins[0]), int(origins[1]))
    num = ctypes.c_uint64(0)
    ak = ctypes.c_int64(-1)
    aj = ctypes.c_int32(0)
    po = np.zeros(max(oe - ob, 1), dtype=np.uint64) if per_origin else None
    rc = lib.oracle_ddks(P.ctypes.data, NP, T.ctypes.data, NT, d, f64, ob, oe, int(nthreads),
                         ctypes.byref(num), ctypes.byref(ak), ctypes.byref(aj),
                         po.ctypes.data if po is not None else None)
    if rc != ORC_OK:
        raise OracleError(rc)
    out = dict(num_max=int(num.value), denom=NP * NT, D=int(num.value) / float(NP * NT),
               argmax_origin=int(ak.value), argmax_orthant=int(aj.value))
    if per_origin:
        out["per_origin"] = po[: oe - ob]
    return out


def philox4x64_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib.oracle_philox4x64_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def perm_key(seed: int, b: int, i: int) -> int:
    return int(_load().oracle_perm_key(seed, b, i))


def perm_labels(seed: int, b: int, NP: int, NT: int) -> np.ndarray:
    """is_p[i] = 1 if pooled point i belongs to the permuted P of permutation b."""
    out = np.zeros(NP + NT, dtype=np.uint8)
    rc = _load().oracle_perm_labels(seed, b, NP, NT, out.ctypes.data)
    if rc != ORC_OK:
        raise OracleError(rc)
    return out


def permutation_test(P, T, B: int, seed: int, nthreads: int = 0):
    lib = _load()
    P, T, f64 = _prep(P, T)
    NP, d = P.shape
    NT = T.shape[0]
    obs = ctypes.c_uint64(0)
    pm = np.zeros(max(B, 1), dtype=np.uint64)
    pv = ctypes.c_double(0.0)
    rc = lib.oracle_permutation_test(P.ctypes.data, NP, T.ctypes.data, NT, d, f64, B, seed,
                                     int(nthreads), ctypes.byref(obs), pm.ctypes.data,
                                     ctypes.byref(pv))
    if rc != ORC_OK:
        raise OracleError(rc)
    return dict(num_obs=int(obs.value), perm_num_max=pm[:B], p_value=float(pv.value))


def cell_p_le(NP: int, NT: int, num_max: int, lam: float, model: int = 0) -> float:
    return float(_load().oracle_cell_p_le(NP, NT, num_max, lam, model))


def significance(P, T, num_max: int, estimator: int = 1, model: int = 0):
    """Eq. (ddks_significance): returns (S, log of the product)."""
    lib = _load()
    P, T, f64 = _prep(P, T)
    NP, d = P.shape
    NT = T.shape[0]
    S = ctypes.c_double(0.0)
    lp = ctypes.c_double(0.0)
    rc = lib.oracle_significance(P.ctypes.data, NP, T.ctypes.data, NT, d, f64, int(num_max),
                                 estimator, model, ctypes.byref(S), ctypes.byref(lp))
    if rc != ORC_OK:
        raise OracleError(rc)
    return float(S.value), float(lp.value)


def vdks(P, T, voxels_per_dim: int):
    """Alg. vdKS (voxel approximation): returns dict(num_max, denom, D,
    argmax_voxel, argmax_orthant), the arg-max being the lowest filled voxel
    (linear index sum_m c_m V^m) and then the lowest orthant reaching num_max."""
    lib = _load()
    P, T, f64 = _prep(P, T)
    NP, d = P.shape
    NT = T.shape[0]
    num = ctypes.c_uint64(0)
    av = ctypes.c_int64(0)
    aj = ctypes.c_int32(0)
    rc = lib.oracle_vdks(P.ctypes.data, NP, T.ctypes.data, NT, d, f64, int(voxels_per_dim), ctypes.byref(num),
                         ctypes.byref(av), ctypes.byref(aj))
    if rc != ORC_OK:
        raise OracleError(rc)
    return dict(num_max=int(num.value), denom=NP * NT, D=int(num.value) / float(NP * NT),
                argmax_voxel=int(av.value), argmax_orthant=int(aj.value))


def rdks(P, T):
    """Alg. rdKS (radial approximation): returns dict(num_max, denom, D, per_corner)."""
    lib = _load()
    P, T, f64 = _prep(P, T)
    NP, d = P.shape
    NT = T.shape[0]
    num = ctypes.c_uint64(0)
    pc = np.zeros(d + 1, dtype=np.uint64)
    rc = lib.oracle_rdks(P.ctypes.data, NP, T.ctypes.data, NT, d, f64, ctypes.byref(num), pc.ctypes.data)
    if rc != ORC_OK:
        raise OracleError(rc)
    return dict(num_max=int(num.value), denom=NP * NT, D=int(num.value) / float(NP * NT), per_corner=pc)


def brute_force_ddks(P, T):
    """Pure-Python restatement of the definition for tiny inputs.

    For every pooled test point o and every orthant j, count the points x of P
    (and of T) with [x_m >= o_m] == bit m of j for all m, and keep the largest
    |cP*NT - cT*NP|.  Returns (num_max, NP*NT).
    """
    P = [list(map(float, r)) for r in np.atleast_2d(np.asarray(P, dtype=np.float64))]
    T = [list(map(float, r)) for r in np.atleast_2d(np.asarray(T, dtype=np.float64))]
    NP, NT = len(P), len(T)
    d = len(P[0])
    best = 0
    for o in P + T:
        for j in range(2 ** d):
            def inside(x):
                return all((x[m] >= o[m]) == bool((j >> m) & 1) for m in range(d))
            cP = sum(1 for x in P if inside(x))
            cT = sum(1 for x in T if inside(x))
            best = max(best, abs(cP * NT - cT * NP))
    return best, NP * NT
