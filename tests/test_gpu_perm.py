"""Permutation test (Sec. 4.2) on the GPU against the oracle: every
relabelling's integer numerator, the observed statistic and the p-value."""
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


def _check(torch, P, T, B, seed):
    ref = orc.permutation_test(P, T, B, seed)
    with pkg.Context(device=0) as c:
        got = c.permutation_test(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), B, seed)
    assert got["observed"]["num_max"] == ref["num_obs"]
    assert np.array_equal(got["perm_num_max"], ref["perm_num_max"])
    assert got["p_value"] == ref["p_value"]
    return got


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 8])
def test_small(torch, d):
    P, T = wl.random_pair(d, 23, 31, d, kind="int")
    _check(torch, P, T, 77, seed=d)
    P, T = wl.random_pair(d + 50, 300, 200, d, kind="normal", dtype=np.float64)
    _check(torch, P, T, 300, seed=99)


def test_edges(torch):
    P, T = wl.random_pair(1, 1, 1, 2)
    _check(torch, P, T, 5, seed=0)
    P, T = wl.random_pair(2, 40, 9, 3, kind="shifted")
    g = _check(torch, P, T, 64, seed=1)
    assert g["observed"]["num_max"] == 40 * 9
    P, T = wl.random_pair(3, 30, 30, 3)
    with pkg.Context(device=0) as c:
        r = c.permutation_test(torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda(), 0, 5)
        assert r["p_value"] == 1.0


def test_config4_mixture_1000(torch):
    P, T = wl.CONFIGS["cfg4_d3_2000x2000_mixture_null"]()
    g = _check(torch, P, T, 1000, seed=2021)
    assert 0.0 < g["p_value"] <= 1.0
    P, T = wl.CONFIGS["cfg4_d3_2000x2000_mixture_alt"]()
    g = _check(torch, P, T, 200, seed=7)
    assert g["p_value"] == 1.0 / 201


def test_large_n_labels(torch):
    # N = 9000 > 256: the label kernel narrows the NP-th key by radix digits
    # before ranking its bucket; the lane-histogram counter takes N > 4096
    P, T = wl.random_pair(11, 5000, 4000, 2, kind="normal")
    _check(torch, P, T, 20, seed=123456789)


@pytest.mark.parametrize("d,kind", [(3, "normal"), (5, "int"), (7, "normal")])
def test_relabelling_ranges_reproduce_the_whole_test(torch, d, kind):
    # shards by relabelling (one per GPU in a multi-GPU run): the ranges'
    # numerators concatenate to the whole test's and their counts give its p
    from paper_2106_13706_gb300 import sharding
    P, T = wl.random_pair(70 + d, 600, 450, d, kind=kind)
    B, seed = 250, 4242
    ref = orc.permutation_test(P, T, B, seed)
    with pkg.Context(device=0) as c:
        Pd, Td = torch.from_numpy(P).cuda(), torch.from_numpy(T).cuda()
        cuts = [0, 1, 97, 97, 200, 250]
        parts = [c.permutation_test_range(Pd, Td, a, b, seed) for a, b in zip(cuts[:-1], cuts[1:])]
        mid = c.permutation_test_range(Pd, Td, 120, 130, seed)
    assert all(p["observed"]["num_max"] == ref["num_obs"] for p in parts)
    assert np.array_equal(np.concatenate([p["perm_num_max"] for p in parts]), ref["perm_num_max"])
    assert np.array_equal(mid["perm_num_max"], ref["perm_num_max"][120:130])
    assert sharding.merge_perm_counts([p["count_ge"] for p in parts], B) == ref["p_value"]
