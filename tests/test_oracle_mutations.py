"""Planted mistakes: each plausible slip in the oracle's loops must be caught by
the pins of test_oracle.py.  The mistake is planted in a temporary copy of the
C source (never in the oracle itself), compiled with gcc, and the same kinds of
checks are run against it through ctypes."""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

from paper_2106_13706_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "ddks_oracle.c")
GOLDEN = os.path.join(HERE, "golden", "hand_cases.json")

# (name, text in the source, replacement); every occurrence is replaced
MUTATIONS = [
    ("strict_compare", "if (x >= o) code", "if (x > o) code"),
    ("swapped_compare", "if (x >= o) code", "if (o >= x) code"),
    ("swapped_normalisation", "int64_t diff = cP[j] * NT - cT[j] * NP;", "int64_t diff = cP[j] * NP - cT[j] * NT;"),
    ("unnormalised_counts", "int64_t diff = cP[j] * NT - cT[j] * NP;", "int64_t diff = cP[j] - cT[j];"),
    ("drop_T_points", "    for (int64_t i = 0; i < N; ++i) {\n      uint64_t code = 0;",
     "    for (int64_t i = 0; i < NP; ++i) {\n      uint64_t code = 0;"),
    ("skip_self", "    for (int64_t i = 0; i < N; ++i) {\n      uint64_t code = 0;",
     "    for (int64_t i = 0; i < N; ++i) {\n      if (i == k) continue;\n      uint64_t code = 0;"),
    ("origins_from_P_only", "for (int64_t k = o_begin; k < o_end; ++k) {\n        po[k - o_begin]",
     "for (int64_t k = o_begin; k < o_end; ++k) {\n        if (k >= NP) { po[k - o_begin] = 0; pj[k - o_begin] = 0; continue; }\n        po[k - o_begin]"),
    ("wrong_bit_index", "code |= (uint64_t)1 << m;", "code |= (uint64_t)1 << (m / 2);"),
    ("transposed_points", "double x = pooled_coord(P, T, NP, d, is_f64, i, m);",
     "double x = pooled_coord(P, T, NP, d, is_f64, m < d ? i : i, (m + 1) % d);"),
]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation {name}: target text not found in the oracle"
    mut = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_ddks.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
    lib.oracle_ddks.restype = ctypes.c_int
    return lib


def _num(lib, P, T):
    P = np.ascontiguousarray(P, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    if P.ndim == 1:
        P, T = P[:, None], T[:, None]
    n = ctypes.c_uint64(0)
    k = ctypes.c_int64(0)
    j = ctypes.c_int32(0)
    N = len(P) + len(T)
    rc = lib.oracle_ddks(P.ctypes.data, len(P), T.ctypes.data, len(T), P.shape[1], 1, 0, N, 1,
                         ctypes.byref(n), ctypes.byref(k), ctypes.byref(j), None)
    assert rc == 0
    return int(n.value)


def _pins_pass(lib):
    """The pin checks of test_oracle.py in compact form; False at the first miss."""
    from oracle import oracle as orc
    for c in json.load(open(GOLDEN))["cases"]:
        if _num(lib, c["P"], c["T"]) != c["num_max"]:
            return False
    for d in (1, 2, 3):
        for kind in ("normal", "int"):
            for seed in range(3):
                P, T = wl.random_pair(seed, 5 + seed, 7, d, kind=kind, dtype=np.float64)
                if _num(lib, P, T) != orc.brute_force_ddks(P, T)[0]:
                    return False
                if _num(lib, T, P) != _num(lib, P, T):
                    return False
    return True


def test_unmutated_copy_passes(tmp_path):
    lib = _build(tmp_path, "identity", "int oracle_num_threads", "int oracle_num_threads")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"planted mistake {name} went unnoticed"
