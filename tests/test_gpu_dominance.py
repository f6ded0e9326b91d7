"""The d = 2 range-query path (DDKS_PATH_DOMINANCE: quadrant counts from
wavelet-matrix range counts over the rank encoding, O(N log N) work) against
the oracle's exact statistic: bit-exact num_max, denominator, arg-max origin and
orthant, per-origin maxima; ties, constants, float32 and float64, host inputs,
origin ranges, graph replay, and sampled origins of a 2,000,000-point problem.
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


def _same(got, ref):
    assert (got["num_max"], got["denom"]) == (ref["num_max"], ref["denom"])
    assert (got["argmax_origin"], got["argmax_orthant"]) == (ref["argmax_origin"], ref["argmax_orthant"])


@pytest.mark.parametrize("n_p,n_t,kind", [(1, 1, "normal"), (1, 5, "int"), (3, 2, "const"), (31, 33, "int"),
                                          (500, 700, "normal"), (2048, 2048, "int"), (5000, 3001, "normal"),
                                          (9000, 7000, "int"), (40000, 25000, "normal"), (700, 900, "shifted")])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_matches_oracle(torch, n_p, n_t, kind, dtype):
    P, T = wl.random_pair(7 + n_p, n_p, n_t, 2, kind=kind, dtype=dtype)
    ref = orc.ddks(P, T)
    with pkg.Context(device=0, path=pkg.PATH_DOMINANCE) as c:
        _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)
        _same(c.distance(P, T), ref)  # host inputs


def test_ranges_and_per_origin(torch):
    P, T = wl.random_pair(3, 3000, 2600, 2, kind="int")
    N = 5600
    with pkg.Context(device=0, path=pkg.PATH_DOMINANCE) as c:
        for a, b in [(0, N), (0, 1), (2999, 3001), (4000, N), (1234, 1234)]:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"][: b - a], ref["per_origin"][: b - a])
            assert got["num_max"] == ref["num_max"]


def test_other_dimensions_are_refused(torch):
    P, T = wl.random_pair(1, 50, 40, 3)
    with pkg.Context(device=0, path=pkg.PATH_DOMINANCE) as c:
        with pytest.raises(pkg.DdksError) as e:
            c.distance(_dev(torch, P), _dev(torch, T))
        assert e.value.code == -8


def test_auto_path_and_replay(torch):
    # d = 2 with 40,000+ points: the default plan is the range-query path
    P, T = wl.gaussian_pair(11, 30000, 20000, 2, shift=0.1)
    ref = orc.ddks(P, T)
    Pd, Td = _dev(torch, P), _dev(torch, T)
    with pkg.Context(device=0) as c:
        for _ in range(4):
            _same(c.distance(Pd, Td), ref)
        assert c.stats()["graph_replays"] >= 2


def test_two_million_points_sampled_origins(torch):
    # the bench's size: every origin's maximum is checked on sampled ranges
    P, T = wl.gaussian_pair(0, 1_000_000, 1_000_000, 2, shift=0.05)
    N = 2_000_000
    with pkg.Context(device=0, path=pkg.PATH_DOMINANCE) as c:
        full = c.distance(_dev(torch, P), _dev(torch, T))
        assert full["denom"] == 10 ** 12
        best = 0
        for a, b in [(0, 300), (999_850, 1_000_150), (N - 300, N), (full["argmax_origin"], full["argmax_origin"] + 1)]:
            got = c.distance_range(_dev(torch, P), _dev(torch, T), a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True, nthreads=orc.num_threads())
            assert np.array_equal(got["per_origin"][: b - a], ref["per_origin"][: b - a])
            best = max(best, ref["num_max"])
        # the reported maximum is attained at the reported origin
        assert best == full["num_max"]
