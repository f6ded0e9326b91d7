"""The two bit-sliced kernels of the register path (d = 2..4) against the
oracle: bit planes built in shared memory by the count kernel (the default)
and bit planes staged in global memory by a pack kernel.  Bit-exact per-origin
maxima, num_max and arg-max, on shapes that span several origin blocks of 127
and batches of 16 groups of 32 points, with ragged tails, ties, tiny samples
and origin sub-ranges."""
import numpy as np
import pytest

import paper_2106_13706_gb300 as pkg
from oracle import oracle as orc
from paper_2106_13706_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4]  # 1: staged by the pack kernel; 2..4: built by the count kernel (three kernel shapes)


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


SHAPES = [(1, 1), (1, 40), (31, 33), (127, 1), (64, 64), (200, 311), (1000, 777), (4097, 2050)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("kind", ["normal", "int"])
def test_shapes_full_range(torch, variant, d, kind):
    with pkg.Context(device=0, path=pkg.PATH_REGISTER, register_variant=variant) as c:
        for i, (n_p, n_t) in enumerate(SHAPES):
            P, T = wl.random_pair(100 * d + i, n_p, n_t, d, kind=kind)
            ref = orc.ddks(P, T, per_origin=True)
            got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, n_p + n_t, per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"]), (n_p, n_t)
            _same(got, ref)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("d", [2, 3, 4])
def test_origin_ranges_with_ties(torch, variant, d):
    rng = np.random.default_rng(7 + d)
    P = rng.integers(0, 40, size=(9000, d)).astype(np.float32)
    T = (rng.integers(0, 40, size=(7300, d)) + (rng.random((7300, d)) < 0.3)).astype(np.float32)
    N = len(P) + len(T)
    cuts = [(0, 1), (0, 127), (5, 900), (8990, 9130), (N - 255, N), (0, N)]
    with pkg.Context(device=0, path=pkg.PATH_REGISTER, register_variant=variant) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        for a, b in cuts:
            got = c.distance_range(Pd, Td, a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"]), (a, b)
            _same(got, ref)


def test_variants_agree_on_the_bench_workload(torch):
    P, T = wl.CONFIGS["cfg2_d4_20000x20000_f32_ties"]()
    ref = orc.ddks(P, T, per_origin=True)
    for variant in VARIANTS:
        with pkg.Context(device=0, path=pkg.PATH_REGISTER, register_variant=variant) as c:
            Pd, Td = _dev(torch, P), _dev(torch, T)
            for _ in range(3):  # direct, captured, replayed
                got = c.distance_range(Pd, Td, 0, len(P) + len(T), per_origin=True)
                assert np.array_equal(got["per_origin"], ref["per_origin"])
                _same(got, ref)


def test_float64_and_large_tables(torch):
    # 150k points: re-rank tables of 4,700 words per dimension
    rng = np.random.default_rng(5)
    P = rng.standard_normal((90000, 3))
    T = rng.standard_normal((60000, 3)) + 0.05
    N = len(P) + len(T)
    with pkg.Context(device=0, path=pkg.PATH_REGISTER) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        for a, b in [(0, 200), (89950, 90100), (N - 300, N)]:
            got = c.distance_range(Pd, Td, a, b, per_origin=True)
            ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"])
            _same(got, ref)
