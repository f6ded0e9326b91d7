"""K0 in one launch (rank_cluster.cu: one thread-block cluster per dimension
sorting in distributed shared memory) against the oracle and against the
multi-launch sorts: bit-exact num_max, arg-max and per-origin maxima on every
kernel path, with sizes that leave cluster segments empty, ragged or exactly
full, ties, signed zeros, infinities, NaN rejection, float32 and float64 up to
the largest sizes the cluster kernel takes."""
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


# pooled sizes: one point per CTA or fewer, segments of 1, ragged, exactly 8 * S
SHAPES = [(1, 1), (3, 4), (7, 2), (8, 1), (9, 9), (100, 37), (4000, 4001), (1024, 1024)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["normal", "int", "const"])
def test_small_shapes_all_paths(torch, dtype, kind):
    for i, (n_p, n_t) in enumerate(SHAPES):
        d = 2 + i % 3
        P, T = wl.random_pair(300 + i, n_p, n_t, d, kind=kind, dtype=dtype)
        ref = orc.ddks(P, T, per_origin=True)
        for path in (pkg.PATH_REGISTER, pkg.PATH_LANE, pkg.PATH_WARP):
            with pkg.Context(device=0, path=path, rank_kernel=2) as c:
                got = c.distance_range(_dev(torch, P), _dev(torch, T), 0, n_p + n_t, per_origin=True)
            assert np.array_equal(got["per_origin"], ref["per_origin"]), (n_p, n_t, path)
            _same(got, ref)


def test_special_values(torch):
    rng = np.random.default_rng(11)
    P = rng.standard_normal((600, 3)).astype(np.float32)
    T = rng.standard_normal((500, 3)).astype(np.float32)
    P[:40, 0] = 0.0
    T[:40, 0] = -0.0
    P[40:50, 1] = np.inf
    T[40:45, 1] = -np.inf
    T[100:300, 2] = P[100:300, 2]  # ties across samples
    ref = orc.ddks(P, T)
    for rk in (0, 1, 2):
        with pkg.Context(device=0, rank_kernel=rk) as c:
            _same(c.distance(_dev(torch, P), _dev(torch, T)), ref)
    P[7, 2] = np.nan
    with pkg.Context(device=0) as c:
        with pytest.raises(pkg.DdksError) as e:
            c.distance(_dev(torch, P), _dev(torch, T))
        assert e.value.code == -2


@pytest.mark.parametrize("dtype,n_p,n_t,d", [(np.float32, 44000, 44000, 4), (np.float64, 30000, 30000, 3),
                                             (np.float32, 40000, 30000, 2)])
def test_largest_cluster_sizes_sampled(torch, dtype, n_p, n_t, d):
    # close to the cluster kernel's shared-memory limit; ties on a grid;
    # d = 2 at 70k points also takes the range-query path, which reads the
    # dimension-1 order the cluster kernel writes
    rng = np.random.default_rng(n_p + d)
    P = rng.integers(0, 5000, size=(n_p, d)).astype(dtype)
    T = (rng.integers(0, 5000, size=(n_t, d)) + (rng.random((n_t, d)) < 0.2)).astype(dtype)
    N = n_p + n_t
    ranges = [(0, 100), (n_p - 50, n_p + 50), (N - 100, N)]
    for rk in (2, 1):
        with pkg.Context(device=0, rank_kernel=rk) as c:
            Pd, Td = _dev(torch, P), _dev(torch, T)
            for a, b in ranges:
                got = c.distance_range(Pd, Td, a, b, per_origin=True)
                ref = orc.ddks(P, T, origins=(a, b), per_origin=True)
                assert np.array_equal(got["per_origin"], ref["per_origin"]), (rk, a, b)
                _same(got, ref)


def test_bench_workload_and_replay(torch):
    P, T = wl.CONFIGS["cfg2_d4_20000x20000_f32_ties"]()
    ref = orc.ddks(P, T)
    with pkg.Context(device=0) as c:
        Pd, Td = _dev(torch, P), _dev(torch, T)
        for _ in range(3):  # direct, captured, replayed
            _same(c.distance(Pd, Td), ref)
