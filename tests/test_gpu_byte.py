"""The byte-compare path (count_byte.cu: per-block byte re-ranks, four
dimensions per 32-bit compare, one shared histogram per origin) against the
oracle: bit-exact per-origin maxima, num_max and arg-max on shapes with
several origin blocks of 127 and several rounds per block, ragged tails, ties,
padding dimensions (d not a multiple of 4), origin sub-ranges and config 3."""
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


@pytest.mark.parametrize("d", [2, 4, 5, 7, 8, 9, 12, 13, 15])
@pytest.mark.parametrize("kind", ["normal", "int"])
def test_shapes_against_oracle(torch, d, kind):
    shapes = [(1, 1), (40, 23), (200, 311), (1000, 777)] if d <= 12 else [(40, 23), (300, 200)]
    with pkg.Context(device=0, path=pkg.PATH_BYTE) as c:
        for i, (n_p, n_t) in enumerate(shapes):
            P, T = wl.random_pair(900 + 10 * d + i, n_p, n_t, d, kind=kind)
            ref = orc.ddks(P, T, per_origin=True)
            got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, n_p + n_t, per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"]), (d, n_p, n_t)
            _same(got, ref)


def test_origin_ranges_float64(torch):
    P, T = wl.random_pair(31, 2500, 1800, 11, kind="int", dtype=np.float64)
    N = 4300
    with pkg.Context(device=0, path=pkg.PATH_BYTE) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        for a, b in [(0, 1), (3, 130), (2490, 2640), (N - 300, N)]:
            got = c.distance_range(Pd, Td, a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"]), (a, b)
            _same(got, ref)


def test_config3_full(torch):
    P, T = wl.CONFIGS["cfg3_d12_4096x4096_f64"]()
    ref = orc.ddks(P, T, per_origin=True)
    with pkg.Context(device=0, path=pkg.PATH_BYTE) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        for _ in range(3):  # direct, captured, replayed
            got = c.distance_range(Pd, Td, 0, len(P) + len(T), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"])
            _same(got, ref)
