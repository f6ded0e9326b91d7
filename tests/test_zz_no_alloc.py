"""ddks_distance_noalloc: the exact distance for callers that cannot allocate
device memory once running (a latency-critical loop that must not pay
cudaMalloc's synchronisation, a process whose device memory another allocator
already holds, code whose device footprint is fixed at start-up).  Its scratch
is one static device array, so two calls in a row reuse it; each call must give
the same result as ddks_distance on the same inputs (bit-exact integers).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import paper_2106_13706_gb300 as pkg
from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2106_13706_gb300 import build as b
    b.build()
    return t


def _key(r):
    return (r["num_max"], r["denom"], r["argmax_origin"], r["argmax_orthant"])


def _noalloc_via_abi(torch, P, T):
    """Call the C entry point directly through ctypes (no binding helpers)."""
    lib = pkg.load()
    r = pkg.binding.ddks_result()
    dt = 1 if P.dtype == torch.float64 else 0
    rc = lib.ddks_distance_noalloc(P.data_ptr(), P.shape[0], T.data_ptr(), T.shape[0], P.shape[1], dt,
                                   torch.cuda.current_stream().cuda_stream, ctypes.byref(r))
    return rc, r.as_dict()


def test_two_calls_in_a_row_match_ddks_distance(torch):
    cases = [wl.gaussian_pair(seed=0, n_p=200, n_t=200, d=3),
             wl.random_pair(7, 5000, 3100, 4, kind="int"),
             wl.random_pair(8, 700, 900, 6, kind="normal", dtype=np.float64)]
    with pkg.Context(device=0) as c:
        for P, T in cases:
            Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
            ref = c.distance(Pd, Td)
            rc1, r1 = _noalloc_via_abi(torch, Pd, Td)
            rc2, r2 = _noalloc_via_abi(torch, Pd, Td)
            assert rc1 == 0 and rc2 == 0
            assert _key(r1) == _key(ref)
            assert _key(r2) == _key(ref)


def _tied_normal(seed, n_p, n_t, d, dtype):
    P, T = wl.random_pair(seed, n_p, n_t, d, kind="normal", dtype=dtype)
    rng = np.random.default_rng(seed + 1)
    k = max(1, n_t // 100)  # 1% of T's rows copy P rows exactly
    T[rng.choice(n_t, k, replace=False)] = P[rng.choice(n_p, k, replace=False)]
    return P, T


@pytest.mark.parametrize("case", ["f32_int_d8_max", "f64_tied_d8_max", "f32_d7"])
def test_at_the_stated_limits_against_the_oracle(torch, case):
    # N = NP + NT = 16384 (the largest shared-memory sort) with d = 8 (the
    # narrowest lane configuration), in both precisions, with many ties
    if case == "f32_int_d8_max":
        P, T = wl.random_pair(21, 8000, 8384, 8, kind="int")
    elif case == "f64_tied_d8_max":
        P, T = _tied_normal(22, 9000, 7384, 8, np.float64)
    else:
        P, T = _tied_normal(23, 5000, 6001, 7, np.float32)
    ref = orc.ddks(P, T)
    Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
    for _ in range(2):
        rc, r = _noalloc_via_abi(torch, Pd, Td)
        assert rc == 0
        assert _key(r) == (ref["num_max"], ref["denom"], ref["argmax_origin"], ref["argmax_orthant"])


def test_limits_and_errors(torch):
    big = torch.zeros((16000, 2), dtype=torch.float32, device="cuda")
    small = torch.zeros((385, 2), dtype=torch.float32, device="cuda")
    rc, _ = _noalloc_via_abi(torch, big, small)          # N = 16385 > 16384
    assert rc == -8
    rc, _ = _noalloc_via_abi(torch, torch.zeros((4, 9), device="cuda"), torch.zeros((4, 9), device="cuda"))
    assert rc == -8                                      # d = 9 > 8
    lib = pkg.load()
    r = pkg.binding.ddks_result()
    host = np.zeros((4, 2), np.float32)
    assert lib.ddks_distance_noalloc(host.ctypes.data, 4, host.ctypes.data, 4, 2, 0, None,
                                     ctypes.byref(r)) == -1  # host inputs are refused
    P, T = wl.random_pair(1, 30, 20, 2)
    P[3, 1] = np.nan
    rc, _ = _noalloc_via_abi(torch, torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda())
    assert rc == -2
    # the NaN flag is cleared by the next call
    P[3, 1] = 0.5
    rc, r = _noalloc_via_abi(torch, torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda())
    assert rc == 0 and r["denom"] == 600
