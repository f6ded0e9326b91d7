"""The LSD radix sort (radix.cu) behind the per-dimension ranks of the exact
paths (K0) and the rdKS distance orders, forced on at small sizes through the
context's radix_min_n and compared with the oracle on every kernel path
(bit-exact num_max, arg-max, per-origin maxima), float32 keys (4 digit passes)
and float64 keys (8), ties, constants, ragged tile tails; and against the
chunk-sort + merge path at sizes where both run.
"""
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


def _dev(torch, A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


CASES = [  # (d, NP, NT, kind, path): paths that read K0's ranks
    (1, 1, 1, "normal", pkg.PATH_AUTO), (1, 3000, 2001, "int", pkg.PATH_AUTO),
    (2, 2047, 2, "normal", pkg.PATH_DOMINANCE), (2, 5000, 3001, "int", pkg.PATH_DOMINANCE),
    (2, 4096, 4096, "const", pkg.PATH_DOMINANCE), (3, 2049, 2047, "int", pkg.PATH_REGISTER),
    (3, 1500, 1200, "normal", pkg.PATH_REGISTER), (4, 700, 900, "int", pkg.PATH_LANE),
    (6, 1500, 1000, "normal", pkg.PATH_WARP), (9, 900, 1100, "int", pkg.PATH_WARP),
    (15, 300, 200, "int", pkg.PATH_SORT), (3, 64, 2000, "shifted", pkg.PATH_AUTO),
]


@pytest.mark.parametrize("d,n_p,n_t,kind,path", CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_distance_with_radix_ranks(torch, d, n_p, n_t, kind, path, dtype):
    P, T = wl.random_pair(31 * d + n_p, n_p, n_t, d, kind=kind, dtype=dtype)
    N = n_p + n_t
    ref = orc.ddks(P, T, origins=(0, N), per_origin=True)
    with pkg.Context(device=0, path=path, radix_min_n=1, rank_kernel=1) as c:
        got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, N, per_origin=True)
    assert (got["num_max"], got["denom"]) == (ref["num_max"], ref["denom"])
    assert (got["argmax_origin"], got["argmax_orthant"]) == (ref["argmax_origin"], ref["argmax_orthant"])
    assert np.array_equal(got["per_origin"][:N], ref["per_origin"][:N])


@pytest.mark.parametrize("kind,dtype", [("int", np.float32), ("normal", np.float32), ("normal", np.float64)])
def test_radix_and_merge_agree_d2_large(torch, kind, dtype):
    # 300k points: 147 tiles per row (the count scan runs as its own kernels)
    P, T = wl.random_pair(77, 160_000, 140_001, 2, kind=kind, dtype=dtype)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    N = P.shape[0] + T.shape[0]
    res = []
    for m in (1, -1):
        with pkg.Context(device=0, path=pkg.PATH_DOMINANCE, radix_min_n=m, rank_kernel=1) as c:
            res.append(c.distance_range(Pd, Td, 0, N, per_origin=True))
    a, b = res
    assert (a["num_max"], a["argmax_origin"], a["argmax_orthant"]) == (b["num_max"], b["argmax_origin"],
                                                                      b["argmax_orthant"])
    assert np.array_equal(a["per_origin"][:N], b["per_origin"][:N])
    # sampled origins against the oracle's definition
    rng = np.random.default_rng(5)
    for o in rng.choice(N, 6, replace=False):
        r = orc.ddks(P, T, origins=(int(o), int(o) + 1), per_origin=True)
        assert a["per_origin"][o] == r["per_origin"][0]


@pytest.mark.parametrize("d,n_p,n_t,kind", [(1, 700, 325, "normal"), (3, 1025, 1024, "int"),
                                            (3, 2500, 2500, "normal"), (5, 3000, 4100, "int"),
                                            (2, 2000, 2000, "const")])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rdks_with_radix_sort(torch, d, n_p, n_t, kind, dtype):
    P, T = wl.random_pair(400 + d, n_p, n_t, d, kind=kind, dtype=dtype)
    ref = orc.rdks(P, T)
    with pkg.Context(device=0, radix_min_n=1, rank_kernel=1) as c:
        got = c.rdks(_dev(torch, P), _dev(torch, T))
    assert (got["num_max"], got["denom"]) == (ref["num_max"], ref["denom"])
    assert np.array_equal(got["per_corner"], ref["per_corner"])
    assert got["argmax_origin"] == int(np.argmax(ref["per_corner"] == ref["num_max"]))


@pytest.mark.parametrize("n_p,n_t", [(100_000, 100_000), (150_000, 150_001)])
def test_rdks_radix_and_merge_agree_large(torch, n_p, n_t):
    # 4 rows of 200k (98 tiles of 2048: counts summed by the scatter CTAs)
    # and of 300k (147 tiles: the count scan kernel)
    P, T = wl.gaussian_pair(8, n_p, n_t, 3, shift=0.05)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    res = []
    for m in (1, -1):
        with pkg.Context(device=0, radix_min_n=m, rank_kernel=1) as c:
            res.append(c.rdks(Pd, Td))
    assert res[0]["num_max"] == res[1]["num_max"]
    assert np.array_equal(res[0]["per_corner"], res[1]["per_corner"])


def test_dominance_partial_ranges_with_radix(torch):
    # the whole range runs the queries in dimension-1 order; partial ranges in origin order
    P, T = wl.random_pair(13, 3000, 2600, 2, kind="int")
    N = 5600
    with pkg.Context(device=0, path=pkg.PATH_DOMINANCE, radix_min_n=1, rank_kernel=1) as c:
        for a, b in [(0, N), (0, 1), (2999, 3001), (4000, N), (1, N)]:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"][: b - a], ref["per_origin"][: b - a])
            assert (got["num_max"], got["argmax_origin"], got["argmax_orthant"]) == (
                ref["num_max"], ref["argmax_origin"], ref["argmax_orthant"])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_radix_special_values(torch, dtype):
    # -0.0 ties with +0.0, infinities sort to the ends, NaN reports ENAN
    rng = np.random.default_rng(21)
    P = rng.choice([0.0, -0.0, 1.5, -np.inf, np.inf, 2.0], size=(3000, 2)).astype(dtype)
    T = rng.choice([0.0, -0.0, -1.5, np.inf, 2.0], size=(2500, 2)).astype(dtype)
    N = 5500
    ref = orc.ddks(P, T, origins=(0, N), per_origin=True)
    for path in (pkg.PATH_DOMINANCE, pkg.PATH_AUTO):
        with pkg.Context(device=0, path=path, radix_min_n=1, rank_kernel=1) as c:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, N, per_origin=True)
            assert (got["num_max"], got["argmax_origin"], got["argmax_orthant"]) == (
                ref["num_max"], ref["argmax_origin"], ref["argmax_orthant"])
            assert np.array_equal(got["per_origin"][:N], ref["per_origin"][:N])
            bad = P.copy()
            bad[7, 1] = np.nan
            with pytest.raises(pkg.DdksError) as e:
                c.distance(_dev(torch, bad), _dev(torch, T))
            assert e.value.code == -2
